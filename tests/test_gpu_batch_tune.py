"""The batched form's autotuner (tucker_batch_autotune) and its launch
configurations.  Every configuration only changes how positions are mapped
to threads and tiles (positions per thread, which rows are staged through
shared memory, the order of a launch's nodes), never the order in which any
output's terms are summed, so a sweep gives the same bits under every
configuration; the fit's per-tensor sums are added atomically and agree to
rounding of the last addition.  Variants: 1, 2 (or 4) positions per thread,
or one position per thread with its input rows copied by cp.async.  The
batches mix the 4096-tensor recipe's shapes with hand-picked ragged ones
whose row lengths C fall on every side of the staging thresholds (C < 16,
16 <= C < 32, 32 <= C < 64, C >= 64).
"""
import itertools

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


def mixed_batch(seed, small_ranks=False):
    w = workloads.planted_batch(20, seed, rho=1e-3)
    dims, ranks = list(w["dims"]), list(w["ranks"])
    extra_d = [(200, 12, 10), (17, 9, 23), (5, 7, 3), (96, 96, 16), (33, 33, 65), (40, 20, 50)]
    extra_r = [(32, 8, 6), (5, 3, 4), (2, 2, 1), (16, 16, 4), (6, 7, 9), (12, 9, 10)]
    if small_ranks:
        ranks = [tuple(min(k, 8) for k in r) for r in ranks]
        extra_r = [tuple(min(k, 8) for k in r) for r in extra_r]
    Ts = [w["T"]]
    for i, (L, K) in enumerate(zip(extra_d, extra_r)):
        p = workloads.planted_tucker(L, K, 0.05, 900 + i, dtype=torch.float32,
                                     build_dtype=torch.float64)
        Ts.append(p["T"].reshape(-1))
    # the planted tensors of the recipe were made with their own ranks; with
    # the ranks capped the decomposition is of lower rank than planted, which
    # is still a valid problem
    return dims + extra_d, ranks + extra_r, torch.cat(Ts).cuda()


class Run:
    def __init__(self, tk, dims, ranks, T):
        self.tk = tk
        self.b = tk.BatchPlan(dims, ranks)
        self.T = T
        self.ws = torch.empty(self.b.ws_bytes, dtype=torch.uint8, device="cuda")
        tk.tucker_batch_prepare(self.b, self.ws)
        self.F0 = torch.empty(self.b.f_elems, dtype=torch.float32, device="cuda")
        G = torch.empty(self.b.g_elems, dtype=torch.float32, device="cuda")
        tk.tucker_batch_sthosvd(self.b, T, self.F0, G, self.ws)
        self.nT2 = torch.empty(self.b.count, dtype=torch.float64, device="cuda")
        tk.tucker_batch_norm2(self.b, T, self.nT2, self.ws)

    def sweep(self):
        tk, b = self.tk, self.b
        F1 = torch.empty_like(self.F0)
        G = torch.empty(b.g_elems, dtype=torch.float32, device="cuda")
        fit = torch.empty(b.count, dtype=torch.float64, device="cuda")
        tk.tucker_batch_sweep(b, self.T, self.F0, F1, G, self.ws)
        tk.tucker_batch_fit(b, self.T, self.F0, G, self.nT2, fit, self.ws)
        torch.cuda.synchronize()
        return F1, G, fit


def uniform(sites, ppt, stage_c, order, asyn):
    return [dict(s, ppt=ppt, stage_c=stage_c, order=order, **{"async": asyn if s["site"] != "fit" else 0})
            for s in sites]


@pytest.mark.parametrize("small_ranks", [False, True])
def test_every_configuration_gives_the_same_bits(tk, small_ranks):
    dims, ranks, T = mixed_batch(21, small_ranks)
    r = Run(tk, dims, ranks, T)
    F_ref, G_ref, fit_ref = r.sweep()
    sites = tk.tucker_batch_tuning(r.b)
    variants = [(1, 1)] + [(p, 0) for p in ((1, 2, 4) if small_ranks else (1, 2))]
    for (ppt, asyn), sc, order in itertools.product(variants, (0, 16, 32, 64), (0, 1)):
        tk.tucker_batch_set_tuning(r.b, uniform(sites, ppt, sc, order, asyn))
        tk.tucker_batch_prepare(r.b, r.ws)
        F1, G, fit = r.sweep()
        assert torch.equal(F1, F_ref), (ppt, asyn, sc, order)
        assert torch.equal(G, G_ref), (ppt, asyn, sc, order)
        assert torch.allclose(fit, fit_ref, rtol=0, atol=1e-12), (ppt, asyn, sc, order)
    assert tk.tucker_device_status() == 0


def test_autotune_keeps_results_and_refuses_stale_graphs(tk):
    dims, ranks, T = mixed_batch(22)
    r = Run(tk, dims, ranks, T)
    b = r.b
    F_ref, G_ref, fit_ref = r.sweep()
    F1 = torch.empty_like(r.F0)
    G = torch.empty(b.g_elems, dtype=torch.float32, device="cuda")
    fit = torch.empty(b.count, dtype=torch.float64, device="cuda")
    old = tk.BatchGraph(b, T, r.F0, F1, G, r.nT2, fit, r.ws)
    old.launch()
    torch.cuda.synchronize()
    assert torch.equal(F1, F_ref) and torch.equal(G, G_ref)
    Gt = torch.empty_like(G)
    tk.tucker_batch_autotune(b, T, r.F0, Gt, r.ws, reps=2)
    torch.cuda.synchronize()
    assert torch.equal(Gt, G_ref)  # the tuning runs leave the core of F0 in G
    sites = tk.tucker_batch_tuning(b)
    for s in sites:
        assert s["ms_default"] > 0 and 0 < s["ms_tuned"] <= s["ms_default"]
        assert s["ppt"] in (1, 2) and s["order"] in (0, 1) and s["async"] in (0, 1)
    with pytest.raises(tk.TuckerError) as e:
        old.launch()
    assert "autotune" in str(e.value)
    F1.zero_()
    G.zero_()
    new = tk.BatchGraph(b, T, r.F0, F1, G, r.nT2, fit, r.ws)
    new.launch()
    torch.cuda.synchronize()
    assert torch.equal(F1, F_ref)
    assert torch.equal(G, G_ref)
    assert torch.allclose(fit, fit_ref, rtol=0, atol=1e-12)
    # the tuning carries over to another batch of the same shapes
    r2 = Run(tk, dims, ranks, T)
    tk.tucker_batch_set_tuning(r2.b, sites)
    tk.tucker_batch_prepare(r2.b, r2.ws)
    F2, G2, _ = r2.sweep()
    assert torch.equal(F2, F_ref) and torch.equal(G2, G_ref)


def test_decomposition_autotune_then_graph_sweeps(tk):
    dims, ranks, T = mixed_batch(23)
    a = tk.BatchDecomposition(T, dims, ranks)
    c = tk.BatchDecomposition(T, dims, ranks)
    a.sthosvd()
    c.sthosvd()
    a.sweep(graph=True)  # records graphs with the default configuration
    c.sweep(graph=True)
    sites = a.autotune(reps=2)
    assert len(sites) == len(tk.tucker_batch_tuning(c.b))
    # both forms were timed; the faster is kept
    assert set(a.form_ms) == {"fused", "per_site"}
    assert a.fused == (a.form_ms["fused"] < a.form_ms["per_site"])
    # 23 tensors: the size heuristic takes the per-site launches
    assert c.fused is False
    for _ in range(3):
        a.sweep(graph=True)
        c.sweep(graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a.factors(), c.factors())
    assert torch.equal(a.G, c.G)
    assert torch.allclose(a.fit_out, c.fit_out, rtol=0, atol=1e-12)


@pytest.mark.parametrize("fused", [False, True])
def test_decomposition_either_form_after_autotune(tk, fused):
    """Whichever form a decomposition sweeps by, after autotune() (which
    switches forms while it times them and restores the factors) its sweeps
    equal those of one that never tuned, set to the same form."""
    dims, ranks, T = mixed_batch(29)
    a = tk.BatchDecomposition(T, dims, ranks, fused=fused)
    c = tk.BatchDecomposition(T, dims, ranks, fused=fused)
    a.sthosvd()
    c.sthosvd()
    a.autotune(reps=1)
    a.set_fused(fused)
    for _ in range(2):
        a.sweep(graph=True)
        c.sweep(graph=False)
    torch.cuda.synchronize()
    assert tk.tucker_device_status() == 0
    assert torch.equal(a.factors(), c.factors())
    assert torch.equal(a.G, c.G)
    assert torch.allclose(a.fit_out, c.fit_out, rtol=0, atol=1e-12)
