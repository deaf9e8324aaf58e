"""The fused root: both root children of the TTM-tree from one read of T.

tucker_ttm_pair (the kernel alone) is checked element by element against the
oracle's literal TTM (Sec. 2.1) with the FP32 FMA accumulation bound, on
shapes covering every layout of T as [A][La][M][Lb][B] and on a tensor that
does not start on a 16-byte boundary.  Whole sweeps with a fused root are
checked against the same sweeps with fusion turned off (plan flag) and against
the FP64 oracle with the FP32 bars (relative fit difference <= 1e-5, largest
principal angle <= 1e-4 rad); the BF16 form against the unfused BF16 form.
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


PAIR_CASES = [
    # dims, a, b, Ka, Kb: (A, M, B) = (1,1,>1), (1,>1,1), (1,>1,>1), (>1,1,1),
    # (>1,1,>1), (>1,>1,1), (>1,>1,>1); the 6-way workload's pair at a smaller A;
    # ranks over the 8 / 16 / 32 classes
    ((8, 4, 4), 0, 1, 3, 2),
    ((11, 9, 20), 0, 2, 10, 10),
    ((22, 7, 5, 2), 0, 2, 3, 2),
    ((300, 13, 7), 1, 2, 6, 3),
    ((26, 39, 2, 30, 4), 2, 3, 1, 2),
    ((5, 18, 3, 24), 1, 3, 1, 7),
    ((3, 13, 4, 3, 2), 1, 3, 3, 1),
    ((7, 5, 3, 32, 24), 3, 4, 8, 6),
    ((513, 40, 48), 1, 2, 17, 32),
    ((1000, 16, 8), 1, 2, 16, 5),
]


@pytest.mark.parametrize("dims,a,b,Ka,Kb", PAIR_CASES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("offset", [0, 1])
def test_ttm_pair_matches_oracle(tk, orc, dims, a, b, Ka, Kb, dtype, offset):
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    X = workloads.random_tensor(dims, seed=sum(dims) + 31 * a + b, dtype=tdt)
    m = X.numel()
    buf = torch.zeros(m + 8, dtype=tdt, device="cuda")
    buf[offset:offset + m] = X.reshape(-1).cuda()
    Xg = buf[offset:offset + m].view(dims)
    Fa = workloads.random_factor(dims[a], Ka, seed=Ka + 5, dtype=torch.float32, orthonormal=False)
    Fb = workloads.random_factor(dims[b], Kb, seed=Kb + 7, dtype=torch.float32, orthonormal=False)
    sa, sb = list(dims), list(dims)
    sa[a], sb[b] = Ka, Kb
    Ya = torch.full(sa, float("nan"), dtype=torch.float32, device="cuda")
    Yb = torch.full(sb, float("nan"), dtype=torch.float32, device="cuda")
    tk.tucker_ttm_pair(Xg, a, Fa.cuda(), Ya, b, Fb.cuda(), Yb)
    torch.cuda.synchronize()
    Xd = X.double().numpy()
    for n, F, Y in ((a, Fa, Ya), (b, Fb, Yb)):
        Fd = F.double().numpy()
        ref = orc.ttm(Xd, n, Fd.T)
        bound = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
        err = np.abs(Y.double().cpu().numpy() - ref)
        assert np.all(err <= (dims[n] + 2) * U32 * bound + 1e-300), (n, (err / (bound + 1e-300)).max())


def test_ttm_pair_rejects_what_does_not_fit(tk):
    X = torch.zeros(4, 64, 64, device="cuda")  # trailing block 16 KB in FP32
    Fa = torch.zeros(64, 4, device="cuda")
    Ya = torch.empty(4, 4, 64, device="cuda")
    Yb = torch.empty(4, 64, 4, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_ttm_pair(X, 1, Fa, Ya, 2, Fa, Yb)
    assert e.value.code == -2


SWEEP_CASES = [
    # L, K, rho, seed: plans whose root is fused (checked below); the first
    # two fuse the last two modes, as the 6-way workload does
    ((12, 28, 12, 13, 9), (4, 7, 4, 3, 2), 1e-2, 41),
    ((40, 21, 10, 18), (20, 10, 2, 4), 0.1, 46),
    ((30, 30, 30), (6, 4, 5), 1.0, 8),
    ((22, 7, 5, 2), (3, 4, 2, 2), 0.2, 42),
    ((26, 3, 2, 16, 21), (5, 1, 2, 3, 12), 0.3, 43),
    ((11, 9, 20), (10, 9, 10), 0.3, 44),
]


def gpu_sweeps(tk, T, L, K, dtype, fuse, sweeps, Tcopy=None):
    p = tk.tucker_plan(L, K, dtype, fuse_root=fuse)
    p32 = tk.tucker_plan(L, K, tk.TUCKER_F32)
    ws = torch.empty(max(tk.tucker_plan_cost(p)["ws_bytes"], tk.tucker_plan_cost(p32)["ws_bytes"]),
                     dtype=torch.uint8, device="cuda")
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(len(L))]
    F2 = [torch.empty_like(f) for f in F]
    G = torch.empty(*K, device="cuda")
    tk.tucker_sthosvd(p32, T if Tcopy is None else Tcopy, F, G, ws)
    for _ in range(sweeps):
        tk.tucker_hooi_sweep_core(p, T, F, F2, G, ws)
        F, F2 = F2, F
    torch.cuda.synchronize()
    return p, [f.double().cpu().numpy() for f in F], G.double().cpu().numpy()


@pytest.mark.parametrize("L,K,rho,seed", SWEEP_CASES)
def test_fused_sweeps_match_unfused_and_oracle(tk, orc, L, K, rho, seed):
    w = workloads.planted_tucker(L, K, rho, seed, dtype=torch.float32, build_dtype=torch.float64)
    T = w["T"].cuda()
    S = 3
    p, Ff, Gf = gpu_sweeps(tk, T, L, K, tk.TUCKER_F32, True, S)
    assert tk.tucker_plan_fused_root(p) is not None
    _, Fu, Gu = gpu_sweeps(tk, T, L, K, tk.TUCKER_F32, False, S)
    # G is the core of the factors the last sweep started from: the same in both
    assert np.abs(Gf - Gu).max() <= 1e-5 * np.abs(Gu).max()
    Tn = w["T"].double().numpy()
    Fo, Go = orc.sthosvd(Tn, K)
    for _ in range(S):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
    nt = orc.norm2(Tn)
    fit_o = orc.fit(nt, orc.norm2(Go))
    for Fg in (Ff, Fu):
        for n in range(len(L)):
            if K[n] < L[n]:
                assert sin_angle(Fg[n], Fo[n]) <= 1e-4, n
        fit_final = orc.fit(nt, orc.norm2(orc.core(Tn, Fg)))
        assert abs(fit_final - fit_o) <= 1e-5 * fit_o, (fit_final, fit_o)
    for n in range(len(L)):
        assert np.abs(Ff[n] - Fu[n]).max() <= 1e-5, n


def test_fused_bf16_form_matches_unfused(tk):
    L, K = (12, 28, 12, 13, 9), (4, 7, 4, 3, 2)
    w = workloads.planted_tucker(L, K, 1e-2, 45, dtype=torch.float32, build_dtype=torch.float64)
    T32 = w["T"].cuda()
    T16 = torch.empty(T32.shape, dtype=torch.bfloat16, device="cuda")
    tk.tucker_convert_bf16(T32, T16)
    p, Ff, _ = gpu_sweeps(tk, T16, L, K, tk.TUCKER_BF16, True, 3, Tcopy=T32)
    assert tk.tucker_plan_fused_root(p) is not None
    _, Fu, _ = gpu_sweeps(tk, T16, L, K, tk.TUCKER_BF16, False, 3, Tcopy=T32)
    for n in range(len(L)):
        if K[n] < L[n]:
            assert sin_angle(Ff[n], Fu[n]) <= 1e-3, n
