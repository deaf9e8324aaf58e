"""FP32 TTMs on the tensor cores against the FP64 oracle's TTM (Sec. 2.1),
one mode at a time and as the L2-blocked pair of a sweep's two root
children: the exact-slice kernel (kernel policy bit 32) and the TF32 split
kernel (bit 64).

Error bound of the exact-slice kernel, derived from its arithmetic: per
64-l chunk c the slices hold x to 2^-17 of 2^6 / s (s < 2 m_x(c), m_x the
chunk's largest |x| of this position) and f to the same with m_f(c); the
four product groups are exact; the dropped slice product 2^-32 x2 f2 and
the epilogue's FP32 roundings (three per chunk, one per chunk sum) add at
most (3 nk + 2) 2^-24 sum |x f| + 2^-26 m_x m_f per term.  Bound used:
sum_l 2^-22 (m_x |f| + |x| m_f + m_x m_f / 16) + (3 nk + 4) 2^-24 sum |x f|.

Error bound of the TF32 split contraction, derived from its arithmetic: with
x = x_hi + x_lo and f = f_hi + f_lo (x_hi, f_hi exact TF32 values, the
remainders read by the tensor core to 11 significant bits), the three
products x_hi f_hi + x_hi f_lo + x_lo f_hi differ from x f by at most
10 * 2^-23 |x f|; each of the 2 * ceil(L / 8) MMAs of a 64-l chunk adds at
most two units of 2^-23 of the chunk's sum of |x f|, and the epilogue's
FP32 sum of the chunk sums one more per chunk.  Bound used:
(12 + 4 * ceil(L / 8) + ceil(L / 64)) * 2^-23 * sum |x f|.
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

U23 = 2.0 ** -23


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


def tf32_bound(L):
    return (12 + 4 * math.ceil(L / 8) + math.ceil(L / 64)) * U23


def x3_bound(Xd, n, Fd):
    """The exact-slice kernel's error bound per output (module docstring):
    chunk maxima of |x| per position and of |f| per factor column."""
    L = Xd.shape[n]
    Xm = np.moveaxis(np.abs(Xd), n, 0)            # L x rest
    Fa = np.abs(Fd)                               # L x K
    nk = (L + 63) // 64
    mx = np.empty_like(Xm)
    mf = np.empty_like(Fa)
    for c in range(nk):
        sl = slice(64 * c, min(L, 64 * c + 64))
        mx[sl] = Xm[sl].max(axis=0, keepdims=True)
        mf[sl] = Fa[sl].max(axis=0, keepdims=True)
    t = np.einsum("l...,lk->k...", mx, Fa) + np.einsum("l...,lk->k...", Xm, mf) + \
        np.einsum("l...,lk->k...", mx, mf) / 16
    s = np.einsum("l...,lk->k...", Xm, Fa)
    b = 2.0 ** -22 * t + (3 * nk + 4) * 2.0 ** -24 * s
    return np.moveaxis(b, 0, n), s


def check_x3(orc, X, n, F, Y):
    Xd = X.double().cpu().numpy()
    Fd = F.double().cpu().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound, _ = x3_bound(Xd, n, Fd)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(np.isfinite(Y.cpu().numpy()))
    assert np.all(err <= bound), (err / bound).max()


def check_ttm(orc, X, n, F, Y):
    Xd = X.double().cpu().numpy()
    Fd = F.double().cpu().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    mag = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    ratio = (err / (mag + 1e-300)).max()
    assert ratio <= tf32_bound(X.shape[n]), ratio
    return ratio


TF32_CASES = [
    # column case (C % 4 == 0, C >= 64): ragged tiles against 128 positions,
    # L past 64-l chunks (and a last chunk of fewer than 8 l), K up to 32
    ((5, 200, 136), 1, 20), ((3, 37, 64), 1, 5), ((2, 64, 1000), 1, 16), ((130, 72), 0, 1),
    ((64, 64, 64, 64), 2, 16), ((4, 256, 128), 1, 32), ((96, 512), 0, 32), ((7, 300, 68), 1, 17),
    ((1, 1000, 100), 1, 3), ((200, 13, 204), 0, 20), ((3, 9, 65, 76), 2, 9),
]


@pytest.mark.parametrize("shape,n,K", TF32_CASES)
@pytest.mark.parametrize("policy", [64, 192])
def test_ttm_tf32_matches_oracle(tk, orc, shape, n, K, policy):
    """policy 64 (TF32 path): fresh accumulator per 64-l chunk; 192: one
    accumulator per tile."""
    X = workloads.random_tensor(shape, seed=sum(shape) + 3 * n, dtype=torch.float32)
    F = workloads.random_factor(shape[n], K, seed=K + 5, dtype=torch.float32, orthonormal=False)
    out = list(shape)
    out[n] = K
    Y = torch.full(out, float("nan"), dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(policy) == 0
    try:
        tk.tucker_ttm(X.cuda(), n, F.cuda(), Y)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    bound = tf32_bound(shape[n]) if policy == 64 else (12 + 8 * math.ceil(shape[n] / 8)) * U23
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    mag = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(np.isfinite(Y.cpu().numpy()))
    assert (err / (mag + 1e-300)).max() <= bound


PAIR_CASES = [
    # (shape, a, Ka, Kb): b = a + 2, blocked by mode a + 1
    ((200, 13, 64, 68), 0, 20, 16),
    ((3, 40, 7, 36, 64), 1, 9, 32),
    ((70, 5, 96, 132), 0, 1, 7),
    ((64, 64, 64, 64), 0, 16, 16),
]


@pytest.mark.parametrize("shape,a,Ka,Kb", PAIR_CASES)
@pytest.mark.parametrize("policy", [32, 64])
def test_ttm_pair_matches_oracle_and_single_ttms(tk, orc, shape, a, Ka, Kb, policy):
    """Both root children from one pass over T blocked by mode a + 1 (policy
    32: exact slices; 64: TF32): each within the bound of the oracle's TTM,
    and the same bits as the single tensor-core TTM of each mode (every
    output position is computed by the same MMAs whichever tile holds it)."""
    b = a + 2
    X = workloads.random_tensor(shape, seed=sum(shape) + a, dtype=torch.float32).cuda()
    Fa = workloads.random_factor(shape[a], Ka, seed=Ka + 1, dtype=torch.float32, orthonormal=False).cuda()
    Fb = workloads.random_factor(shape[b], Kb, seed=Kb + 2, dtype=torch.float32, orthonormal=False).cuda()
    oa, ob = list(shape), list(shape)
    oa[a], ob[b] = Ka, Kb
    Ya = torch.full(oa, float("nan"), dtype=torch.float32, device="cuda")
    Yb = torch.full(ob, float("nan"), dtype=torch.float32, device="cuda")
    Ya1 = torch.full(oa, float("nan"), dtype=torch.float32, device="cuda")
    Yb1 = torch.full(ob, float("nan"), dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(policy) == 0
    try:
        tk.tucker_ttm_pair(X, a, Fa, Ya, b, Fb, Yb)
        tk.tucker_ttm(X, a, Fa, Ya1)
        tk.tucker_ttm(X, b, Fb, Yb1)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    assert torch.equal(Ya, Ya1)
    assert torch.equal(Yb, Yb1)
    for n, F, Y in ((a, Fa, Ya), (b, Fb, Yb)):
        if policy == 32:
            check_x3(orc, X, n, F, Y)
        else:
            check_ttm(orc, X, n, F, Y)


@pytest.mark.parametrize("shape,n,K", TF32_CASES)
def test_ttm_exact_slices_match_oracle(tk, orc, shape, n, K):
    """The exact-slice FP32 column TTM (policy bit 32) within its derived
    bound, including a tensor whose magnitudes
    span many binades (the per-chunk scaling must hold each position's
    small values to its own chunk's scale)."""
    X = workloads.random_tensor(shape, seed=sum(shape) + 3 * n, dtype=torch.float32)
    F = workloads.random_factor(shape[n], K, seed=K + 5, dtype=torch.float32, orthonormal=False)
    out = list(shape)
    out[n] = K
    for scale in (None, "wide"):
        Xs = X
        if scale == "wide":
            g = torch.Generator().manual_seed(9)
            Xs = X * torch.exp2(torch.randint(-30, 30, X.shape, generator=g).float())
        Y = torch.full(out, float("nan"), dtype=torch.float32, device="cuda")
        assert tk.lib().tucker_set_kernel_policy(32) == 0
        try:
            tk.tucker_ttm(Xs.cuda(), n, F.cuda(), Y)
            torch.cuda.synchronize()
        finally:
            tk.lib().tucker_set_kernel_policy(0)
        assert status_ok(tk)
        check_x3(orc, Xs, n, F, Y)


def test_ttm_exact_slices_have_no_bias(tk, orc):
    """Over many outputs of an L = 200 contraction the exact-slice kernel's
    mean signed error (signed toward each output's sign) is a small fraction
    of its mean absolute error: no rounding toward zero anywhere.  The TF32
    kernel (policy 64) fails the same check: its accumulation rounds toward
    zero (measured mean signed error about 0.8 of the mean absolute one)."""
    X = workloads.random_tensor((200, 20000), seed=77, dtype=torch.float32)
    F = workloads.random_factor(200, 20, seed=78, dtype=torch.float32, orthonormal=True)
    ref = orc.ttm(X.double().numpy(), 0, F.double().numpy().T)
    ratios = {}
    for policy in (32, 64):
        Y = torch.empty(20, 20000, dtype=torch.float32, device="cuda")
        assert tk.lib().tucker_set_kernel_policy(policy) == 0
        try:
            tk.tucker_ttm(X.cuda(), 0, F.cuda(), Y)
            torch.cuda.synchronize()
        finally:
            tk.lib().tucker_set_kernel_policy(0)
        d = Y.double().cpu().numpy() - ref
        ratios[policy] = abs(np.mean(d * np.sign(ref))) / np.mean(np.abs(d))
    assert ratios[32] <= 0.1, ratios
    assert ratios[64] >= 0.3, ratios


def sin_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return math.asin(min(1.0, s))


@pytest.mark.parametrize("L,K,rho,seed", [
    ((48, 40, 32, 24), (8, 6, 6, 4), 1e-2, 61),     # the low-noise case the TF32 bias fails
    ((72, 64, 68, 64), (8, 8, 8, 8), 1e-2, 62),     # root pair on the tensor cores (modes 0, 2)
    ((30, 30, 30), (6, 4, 5), 1.0, 8),              # hard case: the fit moves across sweeps
])
def test_sweeps_with_exact_slices_match_oracle(tk, orc, L, K, rho, seed):
    """STHOSVD + 3 HOOI sweeps with every FP32 column TTM on the tensor cores
    (exact slices, policy bit 32; the root pair where the plan has one): fit
    within 1e-5 relative and factor subspaces within 1e-4 rad of the FP64
    oracle at every sweep, the FP32 path's bars."""
    w = workloads.planted_tucker(L, K, rho, seed, dtype=torch.float32)
    assert tk.lib().tucker_set_kernel_policy(32) == 0
    try:
        d = tk.Decomposition(w["T"].cuda(), K)
        d.sthosvd()
        gpu = []
        for _ in range(3):
            d.sweep()
            gpu.append(([f.double().cpu().numpy() for f in d.F], d.fit()))
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    Tn = w["T"].numpy()
    nT2 = orc.norm2(Tn)
    Fo, Go = orc.sthosvd(Tn, K)
    for s in range(3):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
        fit_o = orc.fit(nT2, orc.norm2(Go))
        Fg, fit_g = gpu[s]
        assert abs(fit_g - fit_o) <= 1e-5 * fit_o, (s, fit_g, fit_o)
        for n in range(len(L)):
            assert sin_angle(Fg[n], Fo[n]) <= 1e-4, (s, n)


BF16_PAIR_CASES = [
    ((64, 64, 64, 64), 0, 16, 16),
    ((3, 40, 7, 36, 64), 1, 9, 32),
    ((70, 5, 96, 136), 0, 20, 7),
    ((8, 64, 64, 64, 64), 1, 16, 5),
]


@pytest.mark.parametrize("shape,a,Ka,Kb", BF16_PAIR_CASES)
@pytest.mark.parametrize("ydt", [torch.bfloat16, torch.float32])
def test_bf16_tensor_core_pair_equals_single_ttms(tk, orc, shape, a, Ka, Kb, ydt):
    """The BF16 root pair (policy bit 256) from one pass over T blocked by mode a + 1 gives the
    bits of the two single tensor-core TTMs (policy 16: tensor cores wherever
    the shape allows; each output position is summed by the same MMAs in the
    same order whichever tile holds it), and those are within the BF16
    tensor-core bound of the oracle used for the single TTM (F carried as
    [F_hi | F_lo], FP32 accumulation in TMEM):
    (2^-15 + (L + 2) 2^-23) * sum |x f|."""
    b = a + 2
    X = workloads.random_tensor(shape, seed=sum(shape) + 17 * a, dtype=torch.bfloat16).cuda()
    Fa = workloads.random_factor(shape[a], Ka, seed=Ka + 3, dtype=torch.float32, orthonormal=False).cuda()
    Fb = workloads.random_factor(shape[b], Kb, seed=Kb + 4, dtype=torch.float32, orthonormal=False).cuda()
    oa, ob = list(shape), list(shape)
    oa[a], ob[b] = Ka, Kb
    Ya, Yb = torch.empty(oa, dtype=ydt, device="cuda"), torch.empty(ob, dtype=ydt, device="cuda")
    Ya1, Yb1 = torch.empty(oa, dtype=torch.float32, device="cuda"), torch.empty(ob, dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(256) == 0  # the BF16 pair is opt-in
    try:
        tk.tucker_ttm_pair(X, a, Fa, Ya, b, Fb, Yb)
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert tk.lib().tucker_set_kernel_policy(16) == 0
    try:
        tk.tucker_ttm(X, a, Fa, Ya1)
        tk.tucker_ttm(X, b, Fb, Yb1)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    if ydt == torch.float32:
        assert torch.equal(Ya, Ya1) and torch.equal(Yb, Yb1)
    else:
        assert torch.equal(Ya, Ya1.to(torch.bfloat16)) and torch.equal(Yb, Yb1.to(torch.bfloat16))
    Xd = X.double().cpu().numpy()
    for n, F, Y in ((a, Fa, Ya1), (b, Fb, Yb1)):
        Fd = F.double().cpu().numpy()
        ref = orc.ttm(Xd, n, Fd.T)
        mag = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
        bound = (2.0 ** -15 + (shape[n] + 2) * 2.0 ** -23) * mag
        assert np.all(np.abs(Y.double().cpu().numpy() - ref) <= bound)
