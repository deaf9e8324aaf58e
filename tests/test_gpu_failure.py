"""Failure path of the tensor-core pipelines, exercised without a GPU fault:
every wait of those kernels is bounded by a device timer; a wait that nothing
completes must give up, record TUCKER_ERR_TIMEOUT in the device error word,
return, and leave the context usable for the next call."""
import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pkg


def test_bounded_wait_gives_up_and_reports_timeout(tk, orc):
    assert tk.tucker_device_status(reset=True) in (0, -5)
    assert tk.tucker_device_status() == 0
    t0 = time.time()
    outcome = tk.tucker_selftest_wait_timeout()
    elapsed = time.time() - t0
    assert outcome == 2                      # the wait gave up
    assert 1.0 < elapsed < 60.0              # after its limit (2 s), not at once
    assert tk.tucker_device_status(reset=True) == -5   # TUCKER_ERR_TIMEOUT recorded
    assert tk.tucker_device_status() == 0              # and cleared
    # the context is still usable: a tensor-core TTM runs and is correct
    X = workloads.random_tensor((2, 64, 256), seed=5, dtype=torch.bfloat16)
    F = workloads.random_factor(64, 16, seed=6, dtype=torch.float32, orthonormal=False)
    Y = torch.empty(2, 16, 256, device="cuda")
    tk.tucker_ttm(X.cuda(), 1, F.cuda(), Y)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    ref = orc.ttm(X.double().numpy(), 1, F.double().numpy().T)
    bound = orc.ttm(np.abs(X.double().numpy()), 1, np.abs(F.double().numpy()).T)
    assert np.all(np.abs(Y.double().cpu().numpy() - ref) <= 2.0 ** -14 * bound + 1e-30)
