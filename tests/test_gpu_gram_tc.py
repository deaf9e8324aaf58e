"""The Gram of a mode-n unfolding on the tensor cores (Sec. 5: the SVD of
Z_(n) from its Gram W = Z_(n) Z_(n)^T and an EVD) against the FP64 oracle's
Gram, and against the CUDA-core Gram (kernel policy bit 9).

Error bound of the tensor-core Gram, derived from its arithmetic: each value
is split into x_hi + x_lo, both rounded to 11 significant bits, which hold x
to 2^-22 |x|; of the four products the tensor core forms three, and the
dropped x_lo y_lo is below 2^-22 |x y|, so a product is off by at most
3 * 2^-22 |x y|.  A 32-column stage takes 12 MMAs into a fresh accumulator,
each adding at most two units of 2^-23 of the stage's sum of |x y| (the
bound measured for the TF32 TTM's accumulation); the stage sum enters an
FP32 running sum (at most 16 additions before it is folded into the second
level) and the second level takes at most ceil(Q / 16) folds, Q the chunks
of 32 columns; the last step to FP64 is exact.  Bound used:
(12 + 48 + 16 + ceil(Q / 16) + 2) * 2^-24 * sum |x_i x_j|.
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

U24 = 2.0 ** -24


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pkg


def status_ok(tk):
    import ctypes
    st = ctypes.c_int(-99)
    assert tk.lib().tucker_device_status(ctypes.byref(st), 1) == 0
    return st.value == 0


def view3(shape, n):
    R = int(np.prod(shape[:n], dtype=np.int64))
    C = int(np.prod(shape[n + 1:], dtype=np.int64))
    return R, shape[n], C


def tc_bound(shape, n):
    R, _, C = view3(shape, n)
    Q = R * math.ceil(C / 32)
    return (12 + 48 + 16 + math.ceil(Q / 16) + 2) * U24


def gram_gpu(tk, Z, n, policy=0):
    L = Z.shape[n]
    W = torch.full((L, L), float("nan"), dtype=torch.float64, device="cuda")
    tk.lib().tucker_set_kernel_policy(policy)
    try:
        tk.tucker_gram(Z, n, W)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    return W.cpu().numpy()


# (shape, mode): one block (L <= 128) and block pairs up to four blocks,
# ragged L against 16 and 128, C a multiple of 32 or with a ragged last chunk,
# one row r or many
TC_CASES = [
    ((7, 16), 0), ((20, 36), 0), ((64, 4096), 0), ((100, 1000), 0), ((128, 96), 0),
    ((129, 64), 0), ((200, 2000), 0), ((255, 100), 0), ((256, 320), 0), ((300, 48), 0),
    ((512, 40), 0), ((3, 37, 64), 1), ((17, 200, 20), 1), ((5, 129, 4, 8), 1),
    ((1, 1, 16), 1), ((9, 64, 1000), 1),
]


@pytest.mark.parametrize("shape,n", TC_CASES)
def test_tc_gram_matches_oracle(tk, orc, shape, n):
    Z = workloads.random_tensor(shape, seed=sum(shape) + n, dtype=torch.float32)
    Zd = Z.double().numpy()
    ref = orc.gram(Zd, n)
    mag = orc.gram(np.abs(Zd), n)
    W = gram_gpu(tk, Z.cuda(), n)
    err = np.abs(W - ref)
    bound = tc_bound(shape, n) * mag
    assert np.all(err <= bound + 1e-300), (err / (mag + 1e-300)).max()
    # symmetric up to the order of the FP64 atomic additions
    assert np.all(np.abs(W - W.T) <= 2 * bound + 1e-300)
    # far inside the bound in practice: the split holds FP32 inputs to 2^-22
    rel = float((err / (mag + 1e-300)).max())
    print(f"{shape} mode {n}: max |err| / sum|x y| = {rel:.3g} (bound {tc_bound(shape, n):.3g})")


@pytest.mark.parametrize("shape,n", [((200, 2000), 0), ((17, 200, 20), 1)])
def test_tc_gram_no_worse_than_cuda_cores(tk, orc, shape, n):
    """Against the oracle, the tensor-core Gram's largest error relative to
    sum |x_i x_j| is within 4x of the CUDA-core Gram's (FP32 products summed
    in FP32 runs of 256 columns, runs in FP64), and its mean signed error --
    where a bias of the tensor core's round-toward-zero accumulation would
    show -- is below 2^-24 of sum |x_i x_j|."""
    Z = workloads.random_tensor(shape, seed=11, dtype=torch.float32)
    Zd = Z.double().numpy()
    ref = orc.gram(Zd, n)
    mag = orc.gram(np.abs(Zd), n)
    Wt = gram_gpu(tk, Z.cuda(), n, policy=0)
    Ws = gram_gpu(tk, Z.cuda(), n, policy=512)
    et = float((np.abs(Wt - ref) / mag).max())
    es = float((np.abs(Ws - ref) / mag).max())
    bias = float(np.mean((Wt - ref) / mag))
    print(f"tensor cores {et:.3g}, CUDA cores {es:.3g}, tensor-core mean signed {bias:.3g}")
    assert et <= 4 * es + 4 * U24
    assert abs(bias) <= U24


@pytest.mark.parametrize("L,K,rho", [((200, 60, 50), (10, 8, 6), 1e-2), ((96, 64, 80), (12, 10, 8), 0.3)])
def test_tc_gram_leading_subspace(tk, orc, L, K, rho):
    """What the method uses of the Gram: its leading K_n eigenvectors
    (Sec. 5).  On planted low-rank + noise tensors, for every mode with a
    tensor-core Gram, the angle between the leading subspaces of the GPU Gram
    and of the oracle's is within the Davis-Kahan bound ||E||_F / gap, with
    E the bound matrix of the module docstring and gap = lambda_K -
    lambda_{K+1} of the oracle's Gram."""
    w = workloads.planted_tucker(L, K, rho, 7, dtype=torch.float32)
    T = w["T"]
    Td = T.double().numpy()
    for n in range(len(L)):
        R, Ln, C = view3(L, n)
        if C < 16 or C % 4:
            continue
        ref = orc.gram(Td, n)
        E = tc_bound(L, n) * orc.gram(np.abs(Td), n)
        W = gram_gpu(tk, T.cuda(), n)
        ev, V = np.linalg.eigh(ref)
        _, Vg = np.linalg.eigh(W)
        k = K[n]
        gap = ev[-k] - ev[-k - 1]
        Q0, Q1 = V[:, -k:], Vg[:, -k:]
        sin = np.linalg.norm(Q1 - Q0 @ (Q0.T @ Q1), 2)
        assert sin <= np.linalg.norm(E) / gap, (n, sin, np.linalg.norm(E) / gap)
        assert sin <= 1e-4, (n, sin)


def test_tc_gram_in_sthosvd_matches_oracle(tk, orc):
    """STHOSVD whose Grams run on the tensor cores (every mode but the last
    here) against the oracle's STHOSVD: factors, core and fit."""
    L, K = (128, 96, 64, 40), (8, 8, 6, 5)
    w = workloads.planted_tucker(L, K, 1e-2, 5, dtype=torch.float32)
    T = w["T"].cuda()
    plan = tk.tucker_plan(L, K, tk.TUCKER_F32)
    ws = torch.empty(tk.tucker_plan_cost(plan)["ws_bytes"], dtype=torch.uint8, device="cuda")
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(len(L))]
    G = torch.empty(*K, device="cuda")
    tk.tucker_sthosvd(plan, T, F, G, ws)
    torch.cuda.synchronize()
    assert status_ok(tk)
    Tn = w["T"].numpy()
    Fo, Go = orc.sthosvd(Tn, K)
    nT2 = orc.norm2(Tn)
    fit_o = orc.fit(nT2, orc.norm2(Go))
    fit_g = orc.fit(nT2, orc.norm2(G.double().cpu().numpy()))
    assert abs(fit_g - fit_o) <= 1e-6 * fit_o
    for n in range(len(L)):
        Fg = F[n].double().cpu().numpy()
        Qa, _ = np.linalg.qr(Fo[n])
        s = np.linalg.norm(Fg - Qa @ (Qa.T @ Fg), 2)
        assert s <= 1e-4, (n, s)


def test_tc_gram_scaled_rows(tk, orc):
    """Rows whose magnitudes span 1e-10 .. 1e10, zero rows, and values
    spread over 2^10 inside a row (every product stays in FP32's normal
    range, as both FP32 Gram paths need): within the bound of the module
    docstring, and exactly zero for the zero rows."""
    L, C = 40, 1000
    rng = np.random.default_rng(17)
    Z = rng.standard_normal((L, C)) * np.exp2(rng.uniform(-10, 0, (L, C)))
    Z *= (10.0 ** np.linspace(-10, 10, L))[:, None]
    Z[[3, 17, 29]] = 0.0
    Z = Z.astype(np.float32)
    Zd = Z.astype(np.float64)
    ref = orc.gram(Zd, 0)
    mag = orc.gram(np.abs(Zd), 0)
    W = gram_gpu(tk, torch.from_numpy(Z).cuda(), 0)
    assert np.all(np.isfinite(W))
    err = np.abs(W - ref)
    bound = tc_bound((L, C), 0) * mag
    assert np.all(err <= bound + 1e-300), np.max(err / (mag + 1e-300))
    assert np.all(W[[3, 17, 29]] == 0.0) and np.all(W[:, [3, 17, 29]] == 0.0)
