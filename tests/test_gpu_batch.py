"""Parity of the batched form (many small independent tensors per launch) with
the FP64 oracle run on every tensor in turn, and with the single-tensor GPU
path.  Inputs: prefixes of the 4096-tensor batch recipe (3-way, lengths on
[16, 96], ranks on [4, 16], 1e-3 relative noise) plus hand-picked edge
batches (N = 2 and 4, length 200 with rank 32, ragged tile tails).

Bars as for single tensors on the FP32 path: relative fit difference <= 1e-5,
largest principal angle <= 1e-4 rad.  The batched fit is computed from the
residual ||T - G x F|| itself, so it is also checked against the oracle's
residual of the GPU's own factors and cores.
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
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return math.asin(min(1.0, s))


def edge_batch(seed=31):
    """Hand-picked shapes: N = 3 with length 200 / rank 32, odd sizes whose
    tile tails are ragged, and a rank-1 mode."""
    dims = [(200, 12, 10), (17, 9, 23), (5, 7, 3), (96, 96, 16), (33, 1 + 32, 65)]
    ranks = [(32, 8, 6), (5, 3, 4), (2, 2, 1), (16, 16, 4), (6, 7, 9)]
    return dims, ranks


def pack(dims, ranks, seed, rho, device="cpu"):
    Ts = []
    for i, (L, K) in enumerate(zip(dims, ranks)):
        w = workloads.planted_tucker(L, K, rho, 1000 * seed + i, dtype=torch.float32,
                                     build_dtype=torch.float64)
        Ts.append(w["T"].reshape(-1))
    return torch.cat(Ts).to(device)


def oracle_run(orc, Tn, K, sweeps):
    F, G = orc.sthosvd(Tn, K)
    out = [(F, G)]
    for _ in range(sweeps):
        F, G = orc.hooi_sweep(Tn, F, K)
        out.append((F, G))
    return out


def check_against_oracle(tk, orc, dims, ranks, T, sweeps=3):
    d = tk.BatchDecomposition(T.cuda(), dims, ranks)
    b = d.b
    d.sthosvd()
    hist = [(d.factors().cpu().double().numpy().copy(), d.fit_out.cpu().numpy().copy())]
    for _ in range(sweeps):
        d.sweep(graph=True)
        # G / fit now describe the factors the sweep started from
        hist[-1] = (hist[-1][0], d.fit_out.cpu().numpy().copy())
        hist.append((d.factors().cpu().double().numpy().copy(), None))
    torch.cuda.synchronize()
    nT2 = d.normT2.cpu().numpy()
    Tc = T.cpu()
    for i in range(b.count):
        L, K = dims[i], ranks[i]
        Tn = b.tensor(Tc, i).numpy()
        ref = oracle_run(orc, Tn, K, sweeps)
        assert abs(nT2[i] - orc.norm2(Tn)) <= 1e-12 * orc.norm2(Tn)
        for s, ((Fg, fit_g), (Fo, Go)) in enumerate(zip(hist, ref)):
            for n in range(len(L)):
                Fi = b.factor(torch.from_numpy(Fg), i, n).numpy()
                assert np.abs(Fi.T @ Fi - np.eye(K[n])).max() <= 1e-6, (i, s, n)
                if K[n] < L[n]:
                    assert sin_angle(Fi, Fo[n]) <= 1e-4, (i, s, n, sin_angle(Fi, Fo[n]))
            if fit_g is not None:
                fit_o = orc.fit(orc.norm2(Tn), orc.norm2(Go))
                assert abs(fit_g[i] - fit_o) <= 1e-5 * abs(fit_o), (i, s, fit_g[i], fit_o)


def test_batch_prefix_of_4096_matches_oracle(tk, orc):
    w = workloads.planted_batch(12, 4, rho=1e-3)
    check_against_oracle(tk, orc, w["dims"], w["ranks"], w["T"], sweeps=3)


def test_batch_edge_shapes_match_oracle(tk, orc):
    dims, ranks = edge_batch()
    T = pack(dims, ranks, 31, 0.05)
    check_against_oracle(tk, orc, dims, ranks, T, sweeps=2)


@pytest.mark.parametrize("dims,ranks", [
    ([(30, 20), (12, 40), (64, 9)], [(5, 5), (4, 4), (9, 9)]),                 # N = 2
    ([(12, 10, 9, 8), (7, 16, 5, 11)], [(3, 4, 2, 3), (2, 5, 3, 4)]),          # N = 4
])
def test_batch_other_orders_match_oracle(tk, orc, dims, ranks):
    T = pack(dims, ranks, 41 + len(dims[0]), 0.1)
    check_against_oracle(tk, orc, dims, ranks, T, sweeps=2)


def test_batch_fit_is_the_residual_of_the_decomposition(tk, orc):
    """fit_i = 1 - ||T_i - G_i x F_i|| / ||T_i||, the oracle evaluating the
    residual of the GPU's own STHOSVD factors and cores in FP64."""
    dims, ranks = edge_batch()
    w = workloads.planted_batch(10, 4, rho=1e-3)
    dims, ranks = dims + w["dims"], ranks + w["ranks"]
    T = torch.cat([pack(dims[:5], ranks[:5], 31, 1e-3), w["T"]])
    d = tk.BatchDecomposition(T.cuda(), dims, ranks)
    d.sthosvd()
    torch.cuda.synchronize()
    b = d.b
    F, G, fit = d.factors().cpu(), d.G.cpu(), d.fit_out.cpu().numpy()
    for i in range(b.count):
        Tn = b.tensor(T, i).numpy()
        Fi = [b.factor(F, i, n).double().numpy() for n in range(3)]
        Gi = b.core(G, i).double().numpy()
        ref = 1 - orc.residual(Tn, Gi, Fi) / math.sqrt(orc.norm2(Tn))
        assert abs(fit[i] - ref) <= 1e-8 * abs(ref), (i, fit[i], ref)


def test_batch_sweep_matches_single_tensor_path(tk):
    """One batched sweep from given factors equals tucker_hooi_sweep_core on
    each tensor (same method, different kernels: FP32 rounding only)."""
    w = workloads.planted_batch(24, 4, rho=1e-3)
    dims, ranks = w["dims"], w["ranks"]
    T = w["T"].cuda()
    b = tk.BatchPlan(dims, ranks)
    ws = torch.empty(b.ws_bytes, dtype=torch.uint8, device="cuda")
    tk.tucker_batch_prepare(b, ws)
    F0 = torch.empty(b.f_elems, dtype=torch.float32, device="cuda")
    G0 = torch.empty(b.g_elems, dtype=torch.float32, device="cuda")
    tk.tucker_batch_sthosvd(b, T, F0, G0, ws)
    F1 = torch.empty_like(F0)
    G1 = torch.empty_like(G0)
    tk.tucker_batch_sweep(b, T, F0, F1, G1, ws)
    torch.cuda.synchronize()
    for i in range(b.count):
        L, K = dims[i], ranks[i]
        plan = tk.tucker_plan(L, K)
        pws = tk.workspace(plan)
        Fin = [b.factor(F0, i, n).contiguous() for n in range(3)]
        Fout = [torch.empty_like(f) for f in Fin]
        G = torch.empty(*K, dtype=torch.float32, device="cuda")
        tk.tucker_hooi_sweep_core(plan, b.tensor(T, i), Fin, Fout, G, pws)
        torch.cuda.synchronize()
        Gb = b.core(G1, i)
        assert (Gb - G).abs().max().item() <= 1e-5 * G.abs().max().item(), i
        for n in range(3):
            A = b.factor(F1, i, n).double().cpu().numpy()
            B = Fout[n].double().cpu().numpy()
            if K[n] < L[n]:
                assert sin_angle(A, B) <= 2e-5, (i, n)
            # same sign convention (largest-magnitude entry of a column positive)
            j = np.abs(B).argmax(axis=0)
            assert np.all(np.sign(A[j, range(K[n])]) == np.sign(B[j, range(K[n])])), (i, n)


def test_batch_graph_equals_direct_calls(tk):
    w = workloads.planted_batch(40, 4, rho=1e-3)
    T = w["T"].cuda()
    a = tk.BatchDecomposition(T, w["dims"], w["ranks"])
    c = tk.BatchDecomposition(T, w["dims"], w["ranks"])
    a.sthosvd()
    c.sthosvd()
    n0 = tk.tucker_launch_count()
    for _ in range(3):
        a.sweep(graph=True)
    per_graph = (tk.tucker_launch_count() - n0) / 3
    for _ in range(3):
        c.sweep(graph=False)
    torch.cuda.synchronize()
    assert per_graph >= 5
    assert (a.factors() - c.factors()).abs().max().item() <= 1e-6
    assert (a.G - c.G).abs().max().item() <= 1e-6 * c.G.abs().max().item()
    assert (a.fit_out - c.fit_out).abs().max().item() <= 1e-12
    # fits of a well-conditioned planted batch are close to 1 - 1e-3
    assert float(a.fit_out.min()) > 0.99


def test_batch_fit_is_monotone(tk):
    w = workloads.planted_batch(16, 7, rho=0.3)
    d = tk.BatchDecomposition(w["T"].cuda(), w["dims"], w["ranks"])
    d.sthosvd()
    prev = d.fit_out.clone()
    for _ in range(4):
        d.sweep()
        cur = d.fit_out.clone()
        assert torch.all(cur >= prev - 1e-6), (cur - prev).min().item()
        prev = cur


def test_batch_workspace_errors(tk):
    dims, ranks = [(10, 9, 8)], [(2, 3, 2)]
    b = tk.BatchPlan(dims, ranks)
    T = torch.zeros(720, dtype=torch.float32, device="cuda")
    F = torch.zeros(b.f_elems, dtype=torch.float32, device="cuda")
    G = torch.zeros(b.g_elems, dtype=torch.float32, device="cuda")
    ws = torch.empty(b.ws_bytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_batch_sthosvd(b, T, F, G, ws)
    assert "prepare" in str(e.value)
    with pytest.raises(tk.TuckerError):
        tk.tucker_batch_prepare(b, ws[: b.ws_bytes // 2])
    tk.tucker_batch_prepare(b, ws)
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_batch_sweep(b, T, F, F, G, ws)
    assert "alias" in str(e.value)


def _sthosvd_start(tk, dims, ranks, T):
    d = tk.BatchDecomposition(T.cuda(), dims, ranks, fused=False)
    d.sthosvd()
    torch.cuda.synchronize()
    return d


def test_fused_sweep_equals_per_site_launches(tk):
    """The persistent fused sweep runs the per-site kernels' tile and matrix
    code tensor by tensor: from the same factors its new factors and cores
    are bit-identical to tucker_batch_sweep's, and its fits equal
    tucker_batch_fit's up to the order of the per-tensor FP64 sum."""
    wb = workloads.planted_batch(96, 4, rho=1e-3)
    dims, ranks = wb["dims"], wb["ranks"]
    d = _sthosvd_start(tk, dims, ranks, wb["T"])
    F0 = d.factors().clone()
    T = d.T
    Fa, Fb = torch.empty_like(F0), torch.empty_like(F0)
    Ga, Gb = torch.empty_like(d.G), torch.empty_like(d.G)
    fa, fb = torch.empty_like(d.fit_out), torch.empty_like(d.fit_out)
    tk.tucker_batch_sweep(d.b, T, F0, Fa, Ga, d.ws)
    tk.tucker_batch_fit(d.b, T, F0, Ga, d.normT2, fa, d.ws)
    tk.tucker_batch_sweep_fused(d.b, T, F0, Fb, Gb, d.normT2, fb, d.ws)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    assert torch.equal(Fa, Fb)
    assert torch.equal(Ga, Gb)
    assert torch.allclose(fa, fb, rtol=0, atol=1e-12)
    # a second fused sweep from the new factors (the queue was reset)
    Fc = torch.empty_like(F0)
    tk.tucker_batch_sweep(d.b, T, Fa, Fc, Ga, d.ws)
    tk.tucker_batch_sweep_fused(d.b, T, Fb, Fa, Gb, d.normT2, fb, d.ws)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    assert torch.equal(Fc, Fa)


def test_fused_sweep_edge_shapes_and_graph(tk):
    """Edge shapes (length 200 with rank 32, ragged tails, a rank-1 mode, the
    staged short-row tiles): the fused sweep recorded in a graph equals the
    per-site launches."""
    dims, ranks = edge_batch()
    T = pack(dims, ranks, 5, 1e-2)
    d = _sthosvd_start(tk, dims, ranks, T)
    F0 = d.factors().clone()
    Fa, Fb = torch.empty_like(F0), torch.empty_like(F0)
    Ga = torch.empty_like(d.G)
    tk.tucker_batch_sweep(d.b, d.T, F0, Fa, Ga, d.ws)
    tk.tucker_batch_set_fused(d.b, True)
    g = tk.BatchGraph(d.b, d.T, F0, Fb, d.G, d.normT2, d.fit_out, d.ws)
    g.launch()
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    assert torch.equal(Fa, Fb)
    assert torch.equal(Ga, d.G)


def test_fused_sweep_detects_a_corrupted_queue(tk):
    """Failure detection without a GPU fault: the host poisons the fused
    sweep's work queue (the 'next tensor' counter already at the end), so no
    CTA takes a tensor; the last CTA sees that fewer tensors than the batch
    were taken, records TUCKER_ERR_INCOMPLETE in the device error word and
    resets the queue, and the next sweep runs normally."""
    wb = workloads.planted_batch(40, 4, rho=1e-3)
    dims, ranks = wb["dims"], wb["ranks"]
    d = _sthosvd_start(tk, dims, ranks, wb["T"])
    F0 = d.factors().clone()
    off = tk.tucker_batch_queue_offset(d.b)
    q = d.ws[off:off + 12].view(torch.int32)
    q[0] = d.b.count
    Fb = torch.full_like(F0, float("nan"))
    tk.tucker_batch_sweep_fused(d.b, d.T, F0, Fb, d.G, d.normT2, d.fit_out, d.ws)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == tk.TUCKER_ERR_INCOMPLETE
    assert bool(torch.isnan(Fb).all())  # no tensor was processed
    assert q.tolist() == [0, 0, 0]
    tk.tucker_batch_sweep_fused(d.b, d.T, F0, Fb, d.G, d.normT2, d.fit_out, d.ws)
    Fa = torch.empty_like(F0)
    tk.tucker_batch_sweep(d.b, d.T, F0, Fa, None, d.ws)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    assert torch.equal(Fa, Fb)
