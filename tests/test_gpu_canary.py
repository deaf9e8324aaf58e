"""NaN canary for the workspaces (a stand-in for a memory checker): the
workspace and 64 KiB of guard bytes after it are filled with 0xFF bytes --
NaN in FP32, FP64 and BF16 -- before STHOSVD, HOOI sweeps (plain and with the
core of the input factors), the Gauss-Seidel sweep, the core and the fit run
on ragged shapes.  A read of a workspace word that no kernel wrote first
would carry a NaN into the factors, core or fit; a write past the workspace
would change the guard bytes.  Both are checked after every call."""
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

GUARD = 1 << 16


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pkg


def guarded(nbytes):
    buf = torch.full((nbytes + GUARD,), 0xFF, dtype=torch.uint8, device="cuda")
    return buf, buf[:nbytes]


def guard_intact(buf, nbytes):
    return bool((buf[nbytes:] == 0xFF).all())


CASES = [
    # L, K, storage: ragged against every tile size, N = 2 .. 6, each type
    ((37, 29, 11), (5, 7, 3), "f32"),
    ((9, 8, 7, 6, 5), (3, 3, 2, 2, 2), "f32"),
    ((33, 45), (7, 7), "f64"),
    ((20, 17, 15, 6), (5, 4, 6, 3), "f64"),
    ((72, 64, 40), (8, 6, 5), "bf16"),
    ((64, 48, 40, 24), (8, 8, 6, 4), "fp8"),
    ((16, 14, 12, 10, 8, 6), (4, 4, 3, 3, 2, 2), "bf16"),   # fused root
]


@pytest.mark.parametrize("L,K,kind", CASES)
def test_workspace_canary(tk, L, K, kind):
    dt = torch.float64 if kind == "f64" else torch.float32
    w = workloads.planted_tucker(L, K, 0.3, sum(L), dtype=dt)
    T = w["T"].cuda()
    code = {"f32": tk.TUCKER_F32, "f64": tk.TUCKER_F64, "bf16": tk.TUCKER_BF16, "fp8": tk.TUCKER_FP8_E4M3}[kind]
    if kind == "bf16":
        Ts = torch.empty(T.shape, dtype=torch.bfloat16, device="cuda")
        tk.tucker_convert_bf16(T, Ts)
    elif kind == "fp8":
        Ts = tk.tucker_convert_fp8(T)
    else:
        Ts = T
    plan = tk.tucker_plan(L, K, code)
    p32 = plan if kind in ("f32", "f64") else tk.tucker_plan(L, K, tk.TUCKER_F32)
    nbytes = tk.tucker_plan_cost(plan)["ws_bytes"]
    buf, ws = guarded(nbytes)
    fdt = torch.float64 if kind == "f64" else torch.float32
    F = [torch.empty(L[n], K[n], dtype=fdt, device="cuda") for n in range(len(L))]
    F2 = [torch.empty_like(f) for f in F]
    G = torch.empty(*K, dtype=fdt, device="cuda")
    nt = torch.empty(1, dtype=torch.float64, device="cuda")
    fo = torch.empty(2, dtype=torch.float64, device="cuda")

    def finite(*ts):
        return all(bool(torch.isfinite(t.float()).all()) for t in ts)

    # STHOSVD runs on the FP32 (FP64) tensor, in its own guarded workspace
    nb32 = tk.tucker_plan_cost(p32)["ws_bytes"]
    buf32, ws32 = guarded(nb32)
    tk.tucker_sthosvd(p32, T, F, G, ws32)
    torch.cuda.synchronize()
    assert guard_intact(buf32, nb32) and finite(*F, G)
    calls = [
        lambda: tk.tucker_hooi_sweep(plan, Ts, F, F2, ws),
        lambda: tk.tucker_hooi_sweep_core(plan, Ts, F2, F, G, ws),
        lambda: tk.tucker_hooi_sweep_gs(plan, Ts, F, F2, G, ws),
        lambda: tk.tucker_core(plan, Ts, F2, G, ws),
    ]
    for i, call in enumerate(calls):
        buf.fill_(0xFF)
        call()
        torch.cuda.synchronize()
        assert guard_intact(buf, nbytes), i
        assert finite(*F, *F2, G), i
    tk.tucker_norm2(plan, Ts, nt)
    tk.tucker_fit(plan, G, nt, fo)
    torch.cuda.synchronize()
    assert finite(fo) and 0.0 <= fo[0].item() <= 1.0
    assert tk.tucker_device_status() == 0


def test_batch_workspace_canary(tk):
    """The batched form: its work tables are prepared into a NaN-filled
    guarded workspace, then norms, STHOSVD, direct sweeps, graph-replayed
    sweeps and the residual fit run in it."""
    wb = workloads.planted_batch(24, 4, rho=1e-3)
    T = wb["T"].cuda()
    d = tk.BatchDecomposition(T, wb["dims"], wb["ranks"])
    nbytes = d.b.ws_bytes
    buf, ws = guarded(nbytes)
    d.ws = ws
    tk.tucker_batch_prepare(d.b, ws)
    tk.tucker_batch_norm2(d.b, T, d.normT2, ws)
    d.sthosvd()
    for _ in range(2):
        d.sweep(graph=False)
    for _ in range(2):
        d.sweep(graph=True)
    torch.cuda.synchronize()
    assert guard_intact(buf, nbytes)
    assert bool(torch.isfinite(d.factors()).all()) and bool(torch.isfinite(d.fit_out).all())
    assert bool((d.fit_out > 0.99).all())
    assert tk.tucker_device_status() == 0
