"""Auxiliary paths: the finiteness check (NaN / Inf in a tensor returns
TUCKER_ERR_NONFINITE), checkpoint / resume of a decomposition (the factors
are the HOOI state), and the workspace / argument errors of the sweep."""
import math

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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16])
def test_check_finite(tk, dtype):
    x = workloads.random_tensor((37, 29, 11), seed=3, dtype=dtype).cuda()
    tk.tucker_check_finite(x)
    for bad in (float("nan"), float("inf"), -float("inf")):
        y = x.clone()
        y.view(-1)[1234] = bad
        with pytest.raises(tk.TuckerError) as e:
            tk.tucker_check_finite(y)
        assert e.value.code == -6


def test_check_finite_fp8(tk):
    x = workloads.random_tensor((4096 + 7,), seed=4, dtype=torch.float32)
    f8 = tk.tucker_convert_fp8(x.cuda())
    tk.tucker_check_finite(f8)


def test_checkpoint_resume(tk):
    L, K = (28, 22, 19), (5, 4, 6)
    w = workloads.planted_tucker(L, K, 0.6, 91, dtype=torch.float32)
    a = tk.Decomposition(w["T"].cuda(), K)
    a.sthosvd()
    for _ in range(2):
        a.sweep()
    sd = a.state_dict()
    a.sweep()
    b = tk.Decomposition(w["T"].cuda(), K)
    b.load_state_dict(sd)
    b.sweep()
    torch.cuda.synchronize()
    for fa, fb in zip(a.F, b.F):
        assert (fa - fb).abs().max().item() <= 1e-6
    assert abs(a.fit() - b.fit()) <= 1e-9
    with pytest.raises(ValueError):
        c = tk.Decomposition(w["T"].cuda(), (4, 4, 6))
        c.load_state_dict(sd)
