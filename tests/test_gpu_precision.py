"""Precision form: the tensor stored in BF16 (conversion kernel), HOOI sweeps
on it with BF16 intermediates (tensor-core TTMs where the shape allows), then
FP32 polish sweeps on the FP32 tensor.  Bar after polish: relative fit
difference <= 1e-3 against the FP64 oracle run on the FP32 tensor."""
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


@pytest.mark.parametrize("n", [1, 7, 8, 4096 + 5, 1 << 20])
def test_convert_bf16_is_round_to_nearest_even(tk, n):
    x = workloads.random_tensor((n,), seed=n, dtype=torch.float32) * 37.0
    x[: min(n, 4)] = torch.tensor([0.0, -0.0, 1e-40, 3.0e38][: min(n, 4)])
    xg = x.cuda()
    hi = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    lo = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    tk.tucker_convert_bf16(xg, hi, lo)
    torch.cuda.synchronize()
    ref_hi = x.to(torch.bfloat16)                       # torch rounds to nearest even
    ref_lo = (x - ref_hi.float()).to(torch.bfloat16)
    assert torch.equal(hi.cpu().view(torch.int16), ref_hi.view(torch.int16))
    assert torch.equal(lo.cpu().view(torch.int16), ref_lo.view(torch.int16))
    # hi + lo reproduces x to ~2^-16 relative
    rec = hi.cpu().double() + lo.cpu().double()
    ok = torch.isfinite(x.double()) & (x.double().abs() < 1e38)
    rel = ((rec - x.double()).abs() / x.double().abs().clamp_min(1e-30))[ok & (x != 0)]
    if rel.numel():
        assert rel.max().item() <= 2.0 ** -16


CASES = [
    ((24, 20, 18), (4, 3, 5), 0.3, 51),
    ((12, 10, 16, 9, 8), (3, 3, 4, 2, 2), 0.2, 52),
    ((64, 64, 64, 64), (16, 16, 16, 16), 1e-2, 53),   # tensor-core shapes (C, L % 8 == 0)
    ((72, 64, 40), (8, 6, 5), 0.5, 54),
]


@pytest.mark.parametrize("L,K,rho,seed", CASES)
def test_bf16_sweeps_then_fp32_polish(tk, orc, L, K, rho, seed):
    w = workloads.planted_tucker(L, K, rho, seed, spectrum=("geom", 0.8), dtype=torch.float32)
    T32 = w["T"].cuda()
    T16 = torch.empty(T32.shape, dtype=torch.bfloat16, device="cuda")
    tk.tucker_convert_bf16(T32, T16)
    p16 = tk.tucker_plan(L, K, tk.TUCKER_BF16)
    p32 = tk.tucker_plan(L, K, tk.TUCKER_F32)
    ws = torch.empty(max(tk.tucker_plan_cost(p16)["ws_bytes"], tk.tucker_plan_cost(p32)["ws_bytes"]),
                     dtype=torch.uint8, device="cuda")
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(len(L))]
    F2 = [torch.empty_like(f) for f in F]
    G = torch.empty(*K, device="cuda")
    tk.tucker_sthosvd(p16, T16, F, G, ws)
    for _ in range(6):
        tk.tucker_hooi_sweep(p16, T16, F, F2, ws)
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
