"""tucker_eig_topk_noalloc -- the eigensolver entry point for callers that
must not allocate device memory (its scratch is a fixed array inside the
library).  It must give the same factors as tucker_eig_topk, call after call,
even though every call reuses the one scratch array.

This file is collected last on purpose (test_zz_...), and it also passes on
its own in a fresh process.
"""
import math

import numpy as np
import pytest
import torch

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


def sin_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return math.asin(min(1.0, np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)))


def gram_batch(sizes, seed):
    rng = np.random.default_rng(seed)
    Ws = []
    for L, K in sizes:
        Q, _ = np.linalg.qr(rng.standard_normal((L, L)))
        ev = np.concatenate([1.0 / np.arange(1, K + 1), 1e-3 * rng.random(L - K)])
        Ws.append(torch.tensor((Q * ev) @ Q.T, dtype=torch.float64, device="cuda"))
    return Ws


@pytest.mark.parametrize("fdt", [torch.float32, torch.float64])
def test_noalloc_matches_workspace_entry_point(tk, fdt):
    # two calls in a row with different problems: the second must not be
    # affected by what the first left in the shared scratch
    batches = [[(200, 20), (64, 16), (37, 5)], [(96, 12), (200, 8), (16, 4), (64, 64)]]
    for i, sizes in enumerate(batches):
        Ws = gram_batch(sizes, seed=10 + i)
        F_ref = [torch.empty(L, K, dtype=fdt, device="cuda") for L, K in sizes]
        F_new = [torch.full((L, K), float("nan"), dtype=fdt, device="cuda") for L, K in sizes]
        ws = torch.empty(tk.tucker_eig_ws_bytes([s[0] for s in sizes], [s[1] for s in sizes]),
                         dtype=torch.uint8, device="cuda")
        tk.tucker_eig_topk(Ws, F_ref, ws)
        tk.tucker_eig_topk_noalloc(Ws, F_new)
        torch.cuda.synchronize()
        tol = 1e-12 if fdt == torch.float64 else 1e-6
        for (L, K), a, b in zip(sizes, F_ref, F_new):
            A = a.double().cpu().numpy()
            B = b.double().cpu().numpy()
            assert np.all(np.isfinite(B))
            np.testing.assert_allclose(B, A, rtol=0, atol=tol)
            assert sin_angle(A, B) <= tol + 1e-12
            assert np.abs(B.T @ B - np.eye(K)).max() <= tol


def test_noalloc_allocates_no_device_memory(tk):
    # the entry point's one contract: repeated calls take no device memory
    # from the driver and none from torch's allocator.  A first call of the
    # same problems loads the kernels they use (lazy module loading takes
    # device memory once), so the counters are read after it.
    sizes = [(200, 20), (96, 12), (16, 4)]
    Ws = gram_batch(sizes, seed=30)
    Fs = [torch.empty(L, K, dtype=torch.float32, device="cuda") for L, K in sizes]
    tk.tucker_eig_topk_noalloc(Ws, Fs)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        tk.tucker_eig_topk_noalloc(Ws, Fs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    assert all(bool(torch.isfinite(F).all()) for F in Fs)


def test_noalloc_rejects_beyond_the_fixed_scratch(tk):
    W = torch.zeros(256, 256, dtype=torch.float64, device="cuda")
    F = torch.empty(256, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_eig_topk_noalloc([W], [F])
    assert e.value.code == -2
    Ws = [torch.eye(8, dtype=torch.float64, device="cuda") for _ in range(9)]
    Fs = [torch.empty(8, 2, dtype=torch.float32, device="cuda") for _ in range(9)]
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_eig_topk_noalloc(Ws, Fs)
    assert e.value.code == -2
