"""FP8 variant of the precision form: the tensor stored as E4M3 codes with one
FP32 scale per 64 elements.  The conversion must match the oracle's
quantisation bit for bit; the TTM and the norm that read FP8 must match the
oracle applied to the dequantised values within FP32 rounding; FP8 sweeps
followed by FP32 polish sweeps meet the precision form's bar (relative fit
difference <= 1e-3 against the FP64 oracle on the FP32 tensor)."""
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


def sin_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return math.asin(min(1.0, np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)))


def spread_values(n, seed):
    """Gaussian values whose magnitude changes by orders of magnitude from one
    64-slab to the next, with an all-zero slab and exact E4M3 midpoints."""
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(n, generator=g, dtype=torch.float64)
    mag = 10.0 ** (torch.rand((n + 63) // 64, generator=g, dtype=torch.float64) * 8 - 4)
    x = (x * mag.repeat_interleave(64)[:n]).float()
    if n >= 192:
        x[64:128] = 0.0
        x[128:192] = torch.tensor([448.0, 1.0625 * 448 / 448] + [1.0] * 62)
    return x


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4096 * 64 + 17, 1 << 22])
def test_convert_fp8_matches_oracle_bit_for_bit(tk, orc, n):
    x = spread_values(n, seed=n)
    f8 = tk.tucker_convert_fp8(x.cuda())
    torch.cuda.synchronize()
    q_ref, s_ref = orc.fp8_quantize(x.numpy())
    q = f8.codes().cpu().numpy()
    s = f8.scales().cpu().numpy()
    assert np.array_equal(s.view(np.uint32), s_ref.view(np.uint32))
    assert np.array_equal(q, q_ref)


TTM_CASES = [
    ((64, 48, 40), 0, 16),      # column case, C % 256 != 0: CUDA-core columns kernel
    ((64, 48, 40), 1, 9),       # C = 40 < 64: CUDA-core columns kernel (C % 4 == 0)
    ((30, 20, 64), 2, 16),      # last mode, L % 4 == 0: rows kernel
    ((30, 20, 63), 2, 7),       # last mode, L odd: any-shape kernel
    ((13, 7, 9), 1, 5),         # C odd: any-shape kernel
    ((40, 36, 32, 30), 2, 20),  # C = 30: two K blocks on the CUDA cores
    ((30, 70, 192), 1, 16),     # C % 256 != 0: CUDA cores
    ((30, 70, 256), 1, 16),     # tensor cores: C = 256, two tiles per row, L ragged past 64
    ((5, 130, 768), 1, 32),     # tensor cores: three l chunks (last ragged, its scale rows
                                # run into the next row's), tiles at scale columns 0 and 2 of a box
    ((2, 100, 512), 1, 20),     # tensor cores: two l chunks, K = 20 (two 16-column groups)
    ((30, 70, 80), 1, 16),      # C % 64 != 0 (scale blocks straddle tile halves): CUDA cores
    ((3, 40, 2048), 1, 1),      # tensor cores: K = 1
    ((2, 64, 64, 16), 1, 20),   # tensor cores: C = 1024, K = 20 (two 16-column groups)
]


@pytest.mark.parametrize("dims,n,K", TTM_CASES)
@pytest.mark.parametrize("policy", [0, 1])
def test_ttm_fp8_matches_oracle_on_dequantised_values(tk, orc, dims, n, K, policy):
    """CUDA cores (policy 1): the dequantised values s * E4M3(q) in FP32 and
    FMA accumulation, within 5e-6 of sum |x f|.  Tensor cores (policy 0, the
    column shapes they take): each dequantised value rounded to BF16
    (relative 2^-9, a 32nd of the E4M3 step), F as a BF16 hi + lo pair, FP32
    accumulation in TMEM: within (2^-8 + (L + 2) 2^-23) sum |x f|."""
    x = spread_values(int(np.prod(dims)), seed=7 * n + K)
    f8 = tk.tucker_convert_fp8(x.cuda())
    f8.shape = tuple(dims)
    F = workloads.random_factor(dims[n], K, seed=3 + n, dtype=torch.float32)
    out = list(dims)
    out[n] = K
    Y = torch.full(out, float("nan"), dtype=torch.float32, device="cuda")
    assert tk.lib().tucker_set_kernel_policy(policy) == 0
    try:
        tk.tucker_ttm(f8, n, F.cuda(), Y)
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert tk.tucker_device_status() == 0
    q, s = orc.fp8_quantize(x.numpy())
    xd = orc.fp8_dequantize(q, s).reshape(dims)
    Fd = F.double().numpy()
    ref = orc.ttm(xd, n, Fd.T)
    bound = orc.ttm(np.abs(xd), n, np.abs(Fd).T)
    err = np.abs(Y.double().cpu().numpy() - ref)
    tol = 5e-6 if policy == 1 else 2.0 ** -8 + (dims[n] + 2) * 2.0 ** -23
    assert np.all(err <= tol * bound + 1e-30), float(np.max(err / (bound + 1e-30)))


def test_norm2_fp8(tk, orc):
    L = (50, 40, 36)
    x = spread_values(int(np.prod(L)), seed=11)
    f8 = tk.tucker_convert_fp8(x.cuda())
    f8.shape = L
    p = tk.tucker_plan(L, (5, 4, 3), tk.TUCKER_FP8_E4M3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    tk.tucker_norm2(p, f8, out)
    torch.cuda.synchronize()
    q, s = orc.fp8_quantize(x.numpy())
    ref = orc.norm2(orc.fp8_dequantize(q, s))
    assert abs(out.item() - ref) <= 1e-6 * ref


def test_fp8_plan_rejects_sthosvd(tk):
    L, K = (16, 12, 8), (3, 3, 2)
    x = torch.randn(int(np.prod(L)), device="cuda")
    f8 = tk.tucker_convert_fp8(x)
    f8.shape = L
    p = tk.tucker_plan(L, K, tk.TUCKER_FP8_E4M3)
    ws = tk.workspace(p)
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(3)]
    G = torch.empty(*K, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_sthosvd(p, f8, F, G, ws)
    assert e.value.code == -2


CASES = [
    ((24, 20, 18), (4, 3, 5), 0.3, 61),
    ((64, 64, 64, 64), (16, 16, 16, 16), 1e-2, 62),   # tensor-core shapes below the root
    ((32, 28, 24, 20, 16), (6, 5, 4, 4, 3), 5e-2, 63),
    ((72, 64, 40), (8, 6, 5), 0.5, 64),
]


@pytest.mark.parametrize("L,K,rho,seed", CASES)
def test_fp8_sweeps_then_fp32_polish(tk, orc, L, K, rho, seed):
    w = workloads.planted_tucker(L, K, rho, seed, spectrum=("geom", 0.8), dtype=torch.float32)
    T32 = w["T"].cuda()
    f8 = tk.tucker_convert_fp8(T32.reshape(-1))
    f8.shape = tuple(L)
    p8 = tk.tucker_plan(L, K, tk.TUCKER_FP8_E4M3)
    p32 = tk.tucker_plan(L, K, tk.TUCKER_F32)
    ws = torch.empty(max(tk.tucker_plan_cost(p8)["ws_bytes"], tk.tucker_plan_cost(p32)["ws_bytes"]),
                     dtype=torch.uint8, device="cuda")
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(len(L))]
    F2 = [torch.empty_like(f) for f in F]
    G = torch.empty(*K, device="cuda")
    tk.tucker_sthosvd(p32, T32, F, G, ws)
    for _ in range(6):
        tk.tucker_hooi_sweep_core(p8, f8, F, F2, G, ws)
        F, F2 = F2, F
    for _ in range(2):
        tk.tucker_hooi_sweep(p32, T32, F, F2, ws)
        F, F2 = F2, F
    tk.tucker_core(p32, T32, F, G, ws)
    nt = torch.empty(1, dtype=torch.float64, device="cuda")
    fo = torch.empty(2, dtype=torch.float64, device="cuda")
    tk.tucker_norm2(p32, T32, nt)
    tk.tucker_fit(p32, G, nt, fo)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    fit_g = fo[0].item()
    Tn = w["T"].numpy()
    Fo, Go = orc.sthosvd(Tn, K)
    for _ in range(8):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
    fit_o = orc.fit(orc.norm2(Tn), orc.norm2(Go))
    assert abs(fit_g - fit_o) <= 1e-3 * fit_o, (fit_g, fit_o)
    for n in range(len(L)):
        Fg = F[n].double().cpu().numpy()
        assert np.abs(Fg.T @ Fg - np.eye(K[n])).max() <= 1e-6
        assert sin_angle(Fg, Fo[n]) <= 1e-2
