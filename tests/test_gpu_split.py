"""Split BF16 storage (TUCKER_BF16_SPLIT): an FP32 tensor held as hi = bf16(x)
and lo = bf16(x - hi), read by the tensor-core TTM as A_hi [F_hi | F_lo] +
A_lo F_hi (the split first TTM of the precision form), against the FP64
oracle on the FP32 values (Sec. 2.1 TTM, Fig. 2 sweeps).

Error bound of one split TTM, derived from its arithmetic: hi + lo holds x
to 2^-18 |x| (two round-to-nearest BF16 steps of 2^-9 each), [F_hi | F_lo]
holds f to 2^-18 |f|, the dropped product lo * f_lo is at most 2^-18 |x f|,
and each of the 2 ceil(L / 16) MMAs accumulating into an output adds at
most 2^-23 of the running sum of |x f|.  Bound used:
(3 * 2^-18 + (2 ceil(L / 16) + 4) * 2^-23) * sum |x f|.
"""
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


def test_split_layout_and_norm(tk, orc):
    """The buffer holds hi, then lo from the 256-byte boundary at or after
    2n bytes; hi and lo are the round-to-nearest-even BF16 steps; the squared
    norm of the split tensor is that of hi + lo."""
    for n in (1, 100, 4099):
        assert tk.lib().tucker_bf16_split_lo_offset(n) == (2 * n + 255) // 256 * 256
        assert tk.lib().tucker_bf16_split_bytes(n) == (2 * n + 255) // 256 * 256 + 2 * n
    x = workloads.random_tensor((33, 17, 40), seed=3, dtype=torch.float32)
    xs = tk.tucker_bf16_split(x.cuda())
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    torch.cuda.synchronize()
    assert torch.equal(xs.hi().cpu().view(torch.int16), hi.view(torch.int16))
    assert torch.equal(xs.lo().cpu().view(torch.int16), lo.view(torch.int16))
    # the norm of a split tensor (64^3 takes the tensor-core TTM in every
    # mode, so a split plan exists for it)
    xs2 = tk.tucker_bf16_split(workloads.random_tensor((64, 64, 64), seed=4, dtype=torch.float32).cuda())
    plan = tk.tucker_plan((64, 64, 64), (4, 4, 4), tk.TUCKER_BF16_SPLIT)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    tk.tucker_norm2(plan, xs2, out)
    torch.cuda.synchronize()
    h2 = xs2.hi().cpu().double().numpy() + xs2.lo().cpu().double().numpy()
    assert abs(out.item() - orc.norm2(h2)) <= 1e-12 * orc.norm2(h2)


SPLIT_CASES = [
    # column case (C % 8 == 0, C >= 64): ragged tiles, l chunks; row case (L % 8 == 0)
    ((5, 200, 136), 1, 20), ((3, 37, 64), 1, 5), ((2, 64, 1000), 1, 16), ((64, 64, 64, 64), 2, 16),
    ((4, 256, 128), 1, 33), ((300, 64), 1, 16), ((257, 200), 1, 20), ((7, 9, 128), 2, 64),
]


@pytest.mark.parametrize("shape,n,K", SPLIT_CASES)
def test_split_ttm_matches_oracle(tk, orc, shape, n, K):
    X = workloads.random_tensor(shape, seed=sum(shape) + n, dtype=torch.float32)
    F = workloads.random_factor(shape[n], K, seed=K + 3, dtype=torch.float32, orthonormal=False)
    Xs = tk.tucker_bf16_split(X.cuda())
    out = list(shape)
    out[n] = K
    Y = torch.full(out, float("nan"), dtype=torch.float32, device="cuda")
    tk.tucker_ttm(Xs, n, F.cuda(), Y)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    Xd, Fd = X.double().numpy(), F.double().numpy()
    ref = orc.ttm(Xd, n, Fd.T)
    mag = orc.ttm(np.abs(Xd), n, np.abs(Fd).T)
    L = shape[n]
    bound = (3 * 2.0 ** -18 + (2 * math.ceil(L / 16) + 4) * 2.0 ** -23) * mag
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= bound), (err / (mag + 1e-300)).max()
    # the split is far closer to x than a single BF16 rounding (2^-9)
    assert (err / (mag + 1e-300)).max() <= 2.0 ** -14


def test_split_plan_needs_tensor_core_shapes(tk):
    # mode 1 of (72, 64, 40) has 40 trailing elements: no tensor-core tile
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_plan((72, 64, 40), (8, 6, 5), tk.TUCKER_BF16_SPLIT)
    assert e.value.code == -2
    tk.tucker_plan((96, 64, 72), (8, 6, 5), tk.TUCKER_BF16_SPLIT)


@pytest.mark.parametrize("L,K,rho,seed", [
    ((64, 64, 64, 64), (16, 16, 16, 16), 1e-2, 53),
    ((96, 64, 72), (8, 6, 5), 0.5, 55),
])
def test_split_sweeps_match_oracle(tk, orc, L, K, rho, seed):
    """STHOSVD on the FP32 tensor, then HOOI sweeps that read the split
    tensor in every TTM of T (FP32 intermediates), core and fit of the split
    tensor: against the oracle's STHOSVD + sweeps on the FP32 values.  The
    split holds T to ~2^-18, so the result is far inside the BF16 form's bar
    (1e-3) without FP32 polish sweeps."""
    w = workloads.planted_tucker(L, K, rho, seed, spectrum=("geom", 0.8), dtype=torch.float32)
    T32 = w["T"].cuda()
    Ts = tk.tucker_bf16_split(T32)
    ps = tk.tucker_plan(L, K, tk.TUCKER_BF16_SPLIT)
    p32 = tk.tucker_plan(L, K, tk.TUCKER_F32)
    ws = torch.empty(max(tk.tucker_plan_cost(ps)["ws_bytes"], tk.tucker_plan_cost(p32)["ws_bytes"]),
                     dtype=torch.uint8, device="cuda")
    F = [torch.empty(L[n], K[n], device="cuda") for n in range(len(L))]
    F2 = [torch.empty_like(f) for f in F]
    G = torch.empty(*K, device="cuda")
    tk.tucker_sthosvd(p32, T32, F, G, ws)
    sweeps = 3
    for _ in range(sweeps):
        tk.tucker_hooi_sweep(ps, Ts, F, F2, ws)
        F, F2 = F2, F
    tk.tucker_core(ps, Ts, F, G, ws)
    nt = torch.empty(1, dtype=torch.float64, device="cuda")
    fo = torch.empty(2, dtype=torch.float64, device="cuda")
    tk.tucker_norm2(ps, Ts, nt)
    tk.tucker_fit(ps, G, nt, fo)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    fit_g = fo[0].item()
    Tn = w["T"].numpy()
    Fo, Go = orc.sthosvd(Tn, K)
    for _ in range(sweeps):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
    fit_o = orc.fit(orc.norm2(Tn), orc.norm2(Go))
    assert abs(fit_g - fit_o) <= 1e-4 * fit_o, (fit_g, fit_o)
    for n in range(len(L)):
        Fg = F[n].double().cpu().numpy()
        assert np.abs(Fg.T @ Fg - np.eye(K[n])).max() <= 1e-6
        assert sin_angle(Fg, Fo[n]) <= 1e-3
