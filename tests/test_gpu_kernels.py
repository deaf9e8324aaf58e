"""Parity of the individual CUDA kernels (through the C ABI) with the FP64
oracle: TTM (Sec. 2.1), Gram (Sec. 5), leading eigenvectors (Sec. 5 EVD).

Tolerances are rounding-error bounds of the arithmetic, not fitted numbers:
an FP32 dot product of length L accumulated with fused multiply-adds is within
(L + 2) * 2^-24 * sum |a_i b_i| of the exact value (FP64: 2^-53).
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53


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
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return math.asin(min(1.0, s))


TTM_CASES = [
    # shape, mode, K -- ragged tails, C == 1, odd C, K > 32 (k-blocking), L > 64 (l-chunks)
    ((37, 29, 11), 0, 5), ((37, 29, 11), 1, 7), ((37, 29, 11), 2, 3),
    ((5, 200, 12), 1, 20), ((300, 65), 1, 16), ((3, 7, 5, 6), 2, 2),
    ((257, 33), 0, 40), ((1, 130, 1), 1, 8), ((9, 8, 7, 6, 5), 3, 6),
    ((200, 4, 50), 0, 24), ((13, 1, 17), 1, 1), ((64, 64, 64), 2, 8),
]


@pytest.mark.parametrize("shape,n,K", TTM_CASES)
@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_ttm_matches_oracle(tk, orc, shape, n, K, dtype):
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[dtype]
    X = workloads.random_tensor(shape, seed=sum(shape) + n, dtype=tdt)
    fdt = torch.float64 if dtype == "f64" else torch.float32
    F = workloads.random_factor(shape[n], K, seed=K, dtype=fdt, orthonormal=False)
    out_shape = list(shape)
    out_shape[n] = K
    Y = torch.empty(out_shape, dtype=fdt, device="cuda")
    # the CUDA-core kernels (policy 1): exact FMA accumulation bound
    assert tk.lib().tucker_set_kernel_policy(1) == 0
    try:
        tk.tucker_ttm(X.cuda(), n, F.cuda(), Y)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    u = U64 if dtype == "f64" else U32
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= (shape[n] + 2) * u * bound + 1e-300), err.max()


SLAB_CASES = [
    # C == 1 rows: L a multiple of 8 (vector reads for both types), of 4 only
    # (vector FP32, scalar BF16), odd L; R ragged against the 256-row block;
    # K over every rank class (2 .. 32)
    ((300, 24), 1, 6), ((1000, 24), 1, 8), ((257, 20), 1, 5), ((513, 7), 1, 3), ((64, 3, 32), 2, 32),
    ((91, 17), 1, 1), ((40, 33), 1, 13), ((5, 7, 9, 63), 3, 17), ((2, 300, 16), 2, 24),
    # 1 < C < 64: slabs of L x C per block, positions 256 apart
    ((77, 32, 24), 1, 8), ((50, 40, 2), 1, 4), ((33, 9, 63), 1, 16), ((5, 17, 3), 1, 2),
    ((64, 56, 48, 40, 3), 3, 10), ((129, 31, 5), 1, 32), ((7, 24, 33), 1, 20),
    # C % 4 == 0 and K <= 16
    ((300, 12, 8), 1, 3), ((40, 20, 60), 1, 13), ((9, 33, 4), 1, 16), ((1001, 7, 28), 1, 5),
]


@pytest.mark.parametrize("shape,n,K", SLAB_CASES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("offset", [0, 1])
def test_ttm_short_rows_match_oracle(tk, orc, shape, n, K, dtype, offset):
    """Short rows after mode n (C < 64): runs of whole slabs staged in shared
    memory by 16-byte cp.async (offset 0), or by element copies when the
    tensor does not start on a 16-byte boundary (offset 1: the tensor is a
    view one element into a larger buffer).  FP32 FMA accumulation of exact
    inputs: bound (L + 2) 2^-24 sum |x f|, as for the other CUDA-core TTMs."""
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    X = workloads.random_tensor(shape, seed=sum(shape) * 7 + n, dtype=tdt)
    m = X.numel()
    buf = torch.zeros(m + 8, dtype=tdt, device="cuda")
    buf[offset:offset + m] = X.reshape(-1).cuda()
    Xg = buf[offset:offset + m].view(shape)
    F = workloads.random_factor(shape[n], K, seed=K + 11, dtype=torch.float32, orthonormal=False)
    out_shape = list(shape)
    out_shape[n] = K
    Y = torch.full(out_shape, float("nan"), dtype=torch.float32, device="cuda")
    tk.tucker_ttm(Xg, n, F.cuda(), Y)
    torch.cuda.synchronize()
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= (shape[n] + 2) * U32 * bound + 1e-300), (err / (bound + 1e-300)).max()


# C == 1 with many FP32 rows: the staged row-tile kernel where L % 8 == 0,
# the multi-row kernel for long rows otherwise; R ragged against the rows of
# a block, L over one F chunk of 128 or two, K over the rank classes and
# above 32 (two k blocks)
MULTI_ROW_CASES = [
    ((311302, 128), 1, 20), ((311300, 200), 1, 5), ((160001, 136), 1, 24), ((160003, 128), 1, 33),
    ((2, 160000, 132), 2, 16), ((311301, 124), 1, 20),
    # staged row tiles (L % 8 == 0, at least a block of rows per SM): two
    # stages of columns, K above 32 (two k blocks)
    ((80001, 16), 1, 5), ((40000, 64), 1, 33), ((3, 30000, 200), 2, 20),
]


@pytest.mark.parametrize("shape,n,K", MULTI_ROW_CASES)
def test_ttm_many_rows_match_oracle(tk, orc, shape, n, K):
    X = workloads.random_tensor(shape, seed=sum(shape) + 3 * n, dtype=torch.float32)
    F = workloads.random_factor(shape[n], K, seed=K + 5, dtype=torch.float32, orthonormal=False)
    out_shape = list(shape)
    out_shape[n] = K
    Y = torch.full(out_shape, float("nan"), dtype=torch.float32, device="cuda")
    tk.tucker_ttm(X.cuda(), n, F.cuda(), Y)
    torch.cuda.synchronize()
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= (shape[n] + 2) * U32 * bound + 1e-300), (err / (bound + 1e-300)).max()


TC_CASES = [
    # column case (mode not last; C % 8 == 0, C >= 64): ragged tiles, l chunks
    ((5, 200, 136), 1, 20), ((3, 37, 64), 1, 5), ((2, 64, 1000), 1, 16), ((130, 72), 0, 1),
    ((64, 64, 64, 64), 2, 16), ((4, 256, 128), 1, 33), ((96, 512), 0, 64),
    # C == 64: two r per tile (odd R leaves the last tile half empty)
    ((7, 64, 64), 1, 16), ((4, 100, 64), 1, 20), ((3, 5, 40, 64), 2, 7),
    # row case (last mode; L % 8 == 0)
    ((300, 64), 1, 16), ((257, 200), 1, 20), ((1000, 24), 1, 8), ((7, 9, 128), 2, 64),
]


def status_ok(tk):
    import ctypes
    st = ctypes.c_int(-99)
    assert tk.lib().tucker_device_status(ctypes.byref(st), 1) == 0
    return st.value == 0


@pytest.mark.parametrize("shape,n,K", TC_CASES)
@pytest.mark.parametrize("policy", [16, 1])
def test_ttm_bf16_tensor_cores(tk, orc, shape, n, K, policy):
    """BF16 tensor, FP32 factor: the tcgen05 path (policy 16: tensor cores
    wherever the shape allows) splits F into two BF16 parts (error <= 2^-16
    |f| per product) and accumulates in FP32 in TMEM; the CUDA-core path
    (policy 1) converts exactly and accumulates with FMAs.  Bound:
    (2^-15 + (L + 2) * 2^-23) * sum |x f|."""
    X = workloads.random_tensor(shape, seed=sum(shape) * 3 + n, dtype=torch.bfloat16)
    F = workloads.random_factor(shape[n], K, seed=K + 1, dtype=torch.float32, orthonormal=False)
    out_shape = list(shape)
    out_shape[n] = K
    Y = torch.full(out_shape, float("nan"), dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(policy) == 0
    try:
        tk.tucker_ttm(X.cuda(), n, F.cuda(), Y)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    tol = (2.0 ** -15 + (shape[n] + 2) * 2.0 ** -23) * bound + 1e-30
    assert np.all(err <= tol), (err / (bound + 1e-30)).max()


F32_TC_CASES = [
    # column case (C % 4 == 0, C >= 64): ragged tiles (C not a multiple of 128),
    # l chunks (L > 64, L not a multiple of 64), K > 16 and K = 64
    ((5, 200, 136), 1, 20), ((2, 64, 1000), 1, 16), ((130, 72), 0, 1), ((200, 4, 200), 0, 20),
    ((4, 256, 128), 1, 32), ((96, 512), 0, 17), ((3, 37, 68), 1, 5), ((40, 40, 40, 40), 1, 20),
]


@pytest.mark.parametrize("shape,n,K", F32_TC_CASES)
def test_ttm_f32_tensor_cores(tk, orc, shape, n, K):
    """FP32 tensor, FP32 factor on tcgen05: tile and factor split into three
    BF16 parts each (24 significant bits); the six products x_i f_j with
    i + j <= 4 accumulate in FP32 in TMEM.  The parts reproduce x and f to
    2^-24 relative and the omitted products are below 2^-24 |x f|, hence
    the bound (2^-21 + (L + 2) * 2^-22) * sum |x f| (tensor-core FP32
    accumulation counted at twice the FMA rounding)."""
    X = workloads.random_tensor(shape, seed=sum(shape) * 5 + n, dtype=torch.float32)
    F = workloads.random_factor(shape[n], K, seed=K + 3, dtype=torch.float32, orthonormal=False)
    out_shape = list(shape)
    out_shape[n] = K
    Y = torch.full(out_shape, float("nan"), dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(4) == 0
    try:
        tk.tucker_ttm(X.cuda(), n, F.cuda(), Y)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert status_ok(tk)
    Xd = X.double().numpy()
    Fd = F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    # also the mean signed error relative to the bound: a bias of the
    # accumulation shows here, a random rounding error averages out
    bias = float(np.mean((Y.double().cpu().numpy() - ref) / (bound + 1e-30)))
    print("f32 tensor-core TTM mean signed error / bound:", bias)
    tol = (2.0 ** -21 + (shape[n] + 2) * 2.0 ** -22) * bound + 1e-30
    assert np.all(err <= tol), (err / (bound + 1e-30)).max()


@pytest.mark.parametrize("shape,n", [((37, 29, 11), 0), ((37, 29, 11), 1), ((37, 29, 11), 2),
                                     ((130, 700), 0), ((700, 130), 1), ((3, 200, 41), 1),
                                     ((20, 20, 20, 200), 3), ((5, 6, 7), 1)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_gram_matches_oracle(tk, orc, shape, n, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Z = workloads.random_tensor(shape, seed=len(shape) * 7 + n, dtype=tdt)
    L = shape[n]
    W = torch.empty(L, L, dtype=torch.float64, device="cuda")
    tk.tucker_gram(Z.cuda(), n, W)
    torch.cuda.synchronize()
    Zd = Z.double().numpy()
    ref = orc.gram(Zd, n)
    bound = orc.gram(np.abs(Zd), n)
    # FP32 products summed in FP32 runs of 256 columns, runs summed in FP64
    u = U64 * (Zd.size // L + 2) if dtype == "f64" else U32 * (256 + 2) + U64 * (Zd.size // L)
    err = np.abs(W.cpu().numpy() - ref)
    assert np.all(err <= u * bound + 1e-300), (err / (bound + 1e-300)).max()
    # split-K partials are added with FP64 atomics, whose order differs between
    # W[a, b] and W[b, a]: symmetric up to that rounding
    Wc = W.cpu().numpy()
    assert np.all(np.abs(Wc - Wc.T) <= 2 * u * bound + 1e-300)


def spectrum_matrix(L, evals, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((L, L)))
    return (Q * evals) @ Q.T


EIG_CASES = [
    (16, 4, "rand"), (37, 5, "rand"), (64, 8, "rand"), (64, 16, "decay"), (96, 12, "decay"),
    (200, 20, "decay"), (50, 10, "cluster"), (20, 20, "rand"), (1, 1, "rand"), (2, 1, "rand"),
    (128, 64, "rand"), (33, 3, "lowrank"),
]


@pytest.mark.parametrize("L,K,kind", EIG_CASES)
@pytest.mark.parametrize("fdt", [torch.float32, torch.float64])
def test_eig_topk_matches_oracle(tk, orc, L, K, kind, fdt):
    rng = np.random.default_rng(L * 100 + K)
    if kind == "rand":
        M = rng.standard_normal((L, L + 3))
        W = M @ M.T
    elif kind == "decay":
        ev = np.concatenate([1.0 / np.arange(1, K + 1) ** 2, 1e-6 * rng.random(L - K)])
        W = spectrum_matrix(L, ev, L)
    elif kind == "cluster":
        ev = np.concatenate([[3, 2, 2, 2, 2, 1, 1, 1, 0.5, 0.4], 0.01 * rng.random(L - 10)])
        W = spectrum_matrix(L, ev, L)
    else:  # rank 5 < L
        M = rng.standard_normal((L, 5))
        W = M @ M.T
    W = 0.5 * (W + W.T)
    evals, V, _ = orc.jacobi_eig(W)
    Wg = torch.tensor(W, dtype=torch.float64, device="cuda")
    F = torch.empty(L, K, dtype=fdt, device="cuda")
    ws = torch.empty(tk.tucker_eig_ws_bytes([L], [K]), dtype=torch.uint8, device="cuda")
    tk.tucker_eig_topk([Wg], [F], ws)
    torch.cuda.synchronize()
    Fc = F.double().cpu().numpy()
    orth = 1e-12 if fdt == torch.float64 else 1e-6
    assert np.abs(Fc.T @ Fc - np.eye(K)).max() <= orth
    gap = evals[K - 1] - (evals[K] if K < L else -np.inf)
    if gap > 1e-6 * evals[0]:
        # subspace of the leading K eigenvectors (unique when the gap is open).
        # Error model of the method: the FP32 stage leaves ~n*eps32*lambda_1/gap,
        # each FP64 subspace-iteration step multiplies it by lambda_{K+1}/lambda_K
        # (one step for FP32 factors, two for FP64), and the output rounding adds
        # its own floor.
        ratio = evals[K] / evals[K - 1] if K < L else 0.0
        steps = 2 if fdt == torch.float64 else 1
        stage1 = L * U32 * evals[0] / gap
        floor = 1e-12 if fdt == torch.float64 else 4 * U32
        assert sin_angle(Fc, V[:, :K]) <= stage1 * max(ratio, 0.0) ** steps + floor
        # individual columns where the eigenvalue is simple: same vector incl. sign
        for j in range(K):
            lo = evals[j - 1] - evals[j] if j > 0 else np.inf
            hi = evals[j] - evals[j + 1] if j + 1 < L else np.inf
            if min(lo, hi) > 1e-3 * evals[0]:
                assert np.abs(Fc[:, j] - V[:, j]).max() <= 1e-4, j
    # Rayleigh quotients equal the leading eigenvalues
    rq = np.einsum("ij,ij->j", Fc, W @ Fc)
    u = 1e-12 if fdt == torch.float64 else 8 * U32
    np.testing.assert_allclose(rq, evals[:K], rtol=0, atol=u * evals[0] + 1e-300)


def test_eig_batch_of_uneven_sizes(tk, orc):
    rng = np.random.default_rng(5)
    sizes = [(16, 4), (96, 16), (37, 9), (64, 8), (50, 6)]
    Ws, Fs, refs = [], [], []
    for L, K in sizes:
        M = rng.standard_normal((L, L))
        W = M @ M.T
        Ws.append(torch.tensor(W, device="cuda"))
        Fs.append(torch.empty(L, K, dtype=torch.float32, device="cuda"))
        refs.append(orc.jacobi_eig(W)[1][:, :K])
    ws = torch.empty(tk.tucker_eig_ws_bytes([s[0] for s in sizes], [s[1] for s in sizes]),
                     dtype=torch.uint8, device="cuda")
    tk.tucker_eig_topk(Ws, Fs, ws)
    torch.cuda.synchronize()
    for F, R in zip(Fs, refs):
        assert sin_angle(F.double().cpu().numpy(), R) <= 1e-4


def test_eig_rejects_oversize(tk):
    W = torch.zeros(256, 256, dtype=torch.float64, device="cuda")
    F = torch.empty(256, 4, dtype=torch.float32, device="cuda")
    ws = torch.empty(tk.tucker_eig_ws_bytes([256], [4]), dtype=torch.uint8, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_eig_topk([W], [F], ws)
    assert e.value.code == -2
