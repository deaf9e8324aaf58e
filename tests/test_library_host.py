"""CPU-side checks of the library: it loads, exports every symbol declared in
include/tucker.h, and its host planner (no device work) agrees with the
planner oracle.  No kernel is launched here."""
import math
import os
import random
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    return pkg


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tucker.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tucker_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(tk):
    import ctypes
    L = ctypes.CDLL(tk.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n


def test_version_and_error_text(tk):
    assert tk.tucker_version() >= 100
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_plan((4, 4), (5, 2))
    assert "K_n" in str(e.value)
    assert e.value.code == -1


@pytest.mark.parametrize("L,K,msg", [((4,), (2,), "N must"), ((4, 4), (0, 2), "K_n"),
                                     ((6, 6, 6), (6, 1, 1), "product of the other"),
                                     ((2 ** 14, 2 ** 14, 2 ** 13), (2, 2, 2), "2^40")])
def test_plan_validation(tk, L, K, msg):
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_plan(L, K)
    assert msg in str(e.value)


def tree_of(tk, plan):
    nodes = tk.tucker_plan_nodes(plan)
    return [n["label"] for n in nodes], [n["parent"] for n in nodes], nodes


def test_optimal_tree_matches_oracle_dp_and_bruteforce(tk, orc):
    rnd = random.Random(3)
    for trial in range(120):
        N = rnd.choice([2, 3, 4, 5])
        L = [rnd.choice([2, 3, 5, 8, 20, 50]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        try:
            plan = tk.tucker_plan(L, K)
        except tk.TuckerError:
            continue  # rank-deficient core (K_n > prod of the others)
        labels, parents, nodes = tree_of(tk, plan)
        cost = orc.tree_cost(L, K, labels, parents)
        assert cost is not None, (L, K, labels, parents)
        assert cost == tk.tucker_plan_cost(plan)["tree_macs"]
        assert cost == orc.tree_dp(L, K), (L, K)
        if N <= 4:
            assert cost == orc.tree_bruteforce(L, K)[1]
        # every internal node has at most 2 children (Lemma 3.1 trees are binary)
        for i in range(len(labels)):
            assert sum(1 for p in parents if p == i) <= 2


def check_memory_plan(tk, plan, inter_bytes):
    """Simulates the depth-first execution of the plan's tree: when node v
    runs, the outputs of its ancestors are live (each is read by a later
    descendant), and with a fused root the second root child's output is live
    from the moment the first one runs until its own subtree ends.  No two
    buffers live at the same time may overlap, and all lie in the workspace."""
    nodes = tk.tucker_plan_nodes(plan)
    ws = tk.tucker_plan_cost(plan)["ws_bytes"]
    n = len(nodes)
    end = list(range(1, n + 1))  # subtree of u = [u, end[u]) in pre-order
    for v in range(n - 1, 0, -1):
        p = nodes[v]["parent"]
        end[p] = max(end[p], end[v])
    fused = tk.tucker_plan_fused_root(plan)
    buf = {u: (nd["ws_offset"], nd["ws_offset"] + nd["out_elems"] * inter_bytes)
           for u, nd in enumerate(nodes) if nd["label"] >= 0}
    for u, (a, b) in buf.items():
        assert 0 <= a < b <= ws, (u, a, b, ws)
    for v in buf:
        live = set()
        w = nodes[v]["parent"]
        while w > 0:
            live.add(w)
            w = nodes[w]["parent"]
        if fused:
            u1, u2 = fused
            if u1 <= v < end[u2] and v != u2:
                live.add(u2)
            if v == u2:
                live.discard(u1)
        a, b = buf[v]
        for w in live:
            c, d = buf[w]
            assert b <= c or d <= a, ("overlap", v, w, buf[v], buf[w])


def test_memory_plan_has_no_live_overlap(tk):
    """The stack memory plan (Sec. 3.1: live intermediates bounded by the tree
    depth) never places two simultaneously live outputs on the same bytes:
    every tree kind, with and without the fused root, several dtypes."""
    shapes = [((200,) * 4, (20,) * 4), ((64,) * 5, (16,) * 5),
              ((64, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)),
              ((16, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)),
              ((12, 28, 12, 13, 9), (4, 7, 4, 3, 2)), ((40, 21, 10, 18), (20, 10, 2, 4))]
    rnd = random.Random(17)
    for _ in range(60):
        N = rnd.choice([2, 3, 4, 5, 6, 7, 8])
        L = [rnd.choice([2, 3, 5, 8, 13, 24, 40]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        if all(K[n] <= math.prod(K) // K[n] for n in range(N)):
            shapes.append((L, K))
    fused_seen = 0
    for L, K in shapes:
        for dtype, ib in ((tk.TUCKER_F32, 4), (tk.TUCKER_BF16, 2), (tk.TUCKER_F64, 8)):
            for tree in (tk.TREE_OPTIMAL, tk.TREE_CHAIN, tk.TREE_BALANCED):
                for fuse in (True, False):
                    p = tk.tucker_plan(L, K, dtype, tree, fuse_root=fuse)
                    fused_seen += tk.tucker_plan_fused_root(p) is not None
                    check_memory_plan(tk, p, ib)
    assert fused_seen >= 4


def test_core_chain_order_matches_bruteforce(tk, orc):
    """The new-core chain's mode order (a DP over the set of modes applied)
    reaches the least multiply-adds over all N! orders."""
    shapes = [((200,) * 4, (20,) * 4), ((64,) * 5, (16,) * 5),
              ((64, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)), ((40, 12, 30, 25), (3, 10, 4, 20))]
    rnd = random.Random(23)
    for _ in range(80):
        N = rnd.choice([2, 3, 4, 5, 6, 7])
        L = [rnd.choice([2, 3, 5, 8, 13, 40, 97]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        if all(K[n] <= math.prod(K) // K[n] for n in range(N)):
            shapes.append((L, K))
    for L, K in shapes:
        assert tk.tucker_plan_cost(tk.tucker_plan(L, K))["core_macs"] == orc.core_chain_bruteforce(L, K), (L, K)


def test_elems_tree_matches_bruteforce(tk, orc):
    """The planner's DP under the elements-moved node cost (COST_ELEMS) reaches
    the least cost over every TTM-tree of any arity (explicit enumeration of
    the planner oracle), and the tree it returns is a valid TTM-tree whose
    elements-moved cost the oracle recomputes to the reported tree_elems."""
    rnd = random.Random(5)
    checked = 0
    for trial in range(200):
        N = rnd.choice([2, 3, 4, 4])
        L = [rnd.choice([2, 3, 5, 8, 20, 50]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        try:
            plan = tk.tucker_plan(L, K, cost_model=tk.COST_ELEMS)
        except tk.TuckerError:
            continue  # rank-deficient core (K_n > prod of the others)
        labels, parents, _ = tree_of(tk, plan)
        cost = orc.tree_cost(L, K, labels, parents, elems=True)
        assert cost is not None, (L, K, labels, parents)
        assert cost == tk.tucker_plan_cost(plan)["tree_elems"]
        assert cost == orc.tree_bruteforce(L, K, elems=True)[1], (L, K)
        checked += 1
    assert checked >= 80
    L, K = (13, 7, 20, 5, 9), (4, 7, 3, 2, 5)  # one N = 5 case
    plan = tk.tucker_plan(L, K, cost_model=tk.COST_ELEMS)
    assert tk.tucker_plan_cost(plan)["tree_elems"] == orc.tree_bruteforce(L, K, elems=True)[1]


@pytest.mark.parametrize("tree,fn", [(1, "chain"), (2, "chain_k"), (3, "chain_h"), (4, "balanced")])
def test_prior_scheme_trees_match_oracle(tk, orc, tree, fn):
    rnd = random.Random(11 + tree)
    for trial in range(40):
        N = rnd.choice([3, 4, 5, 6])
        L = [rnd.choice([3, 5, 20, 50, 100]) for _ in range(N)]
        K = [max(1, l // rnd.choice([1, 2, 5, 10])) for l in L]
        try:
            plan = tk.tucker_plan(L, K, tree=tree)
        except tk.TuckerError:
            continue
        labels, parents, _ = tree_of(tk, plan)
        cost = orc.tree_cost(L, K, labels, parents)
        assert cost is not None
        if fn == "chain":
            ref = orc.chain_cost(L, K)
        elif fn == "chain_k":
            ref = orc.chain_cost(L, K, orc.k_order(L, K))
        elif fn == "chain_h":
            ref = orc.chain_cost(L, K, orc.h_order(L, K))
        else:
            ref = orc.balanced_cost(L, K)
        assert cost == ref
        assert cost >= orc.tree_dp(L, K)


def test_workload_tree_costs(tk, orc):
    # the benchmark shapes: the planner's optimum equals the oracle DP, and the
    # chain/optimal load ratios are those of the enumeration
    cases = [((200,) * 4, (20,) * 4), ((64,) * 5, (16,) * 5),
             ((64, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)), ((64,) * 3, (8,) * 3)]
    for L, K in cases:
        plan = tk.tucker_plan(L, K)
        c = tk.tucker_plan_cost(plan)
        assert c["tree_macs"] == orc.tree_dp(L, K)
        labels, parents, _ = tree_of(tk, plan)
        assert orc.tree_cost(L, K, labels, parents) == c["tree_macs"]


def test_memory_plan_is_a_stack(tk):
    """A node's output buffer must not overlap any buffer on its root path
    (they are all live while the node runs)."""
    for L, K in [((200,) * 4, (20,) * 4), ((64,) * 5, (16,) * 5), ((9, 8, 7, 6, 5), (3, 2, 4, 1, 2))]:
        plan = tk.tucker_plan(L, K, dtype=tk.TUCKER_F32)
        _, _, nodes = tree_of(tk, plan)
        ws = tk.tucker_plan_cost(plan)["ws_bytes"]
        for i, nd in enumerate(nodes):
            if nd["label"] < 0:
                continue
            a0, a1 = nd["ws_offset"], nd["ws_offset"] + 4 * nd["out_elems"]
            assert a1 <= ws
            p = nd["parent"]
            while p > 0:
                q = nodes[p]
                b0, b1 = q["ws_offset"], q["ws_offset"] + 4 * q["out_elems"]
                assert a1 <= b0 or b1 <= a0, (i, p)
                p = q["parent"]


FUSED_SHAPES = [
    # (L, K): shapes whose first two root children fuse, covering every layout
    # of T as [A][La][M][Lb][B] (A, M, B each 1 or more) and both orders of
    # the two children in the tree
    ((64, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)),
    ((8, 4, 4), (3, 2, 2)), ((11, 9, 20), (10, 9, 10)), ((22, 7, 5, 2), (3, 4, 2, 2)),
    ((21, 13, 7, 11, 21), (8, 3, 6, 1, 2)), ((13, 32, 14, 37, 4), (7, 8, 6, 7, 1)),
    ((26, 39, 2, 30, 4), (12, 3, 1, 2, 2)), ((4, 31, 5, 13, 5, 16), (4, 9, 5, 3, 2, 6)),
    ((5, 18, 3, 24), (4, 1, 3, 7)), ((13, 4, 32, 16), (3, 1, 3, 2)),
    ((26, 3, 2, 16, 21), (5, 1, 2, 3, 12)), ((3, 13, 4, 3, 2), (2, 3, 3, 1, 2)),
]


@pytest.mark.parametrize("L,K", FUSED_SHAPES)
def test_fused_root_plan(tk, L, K):
    """A fused root names the first two root children (depth-first order);
    the second one's buffer overlaps no buffer of the first one's subtree
    (it is written with the first one and read after that subtree); without
    fusion (plan flag) the plan is the plain stack plan.  The trailing block
    from the smaller of the two modes fits in 8 KB (host only)."""
    import math
    for dtype, es in ((tk.TUCKER_F32, 4), (tk.TUCKER_BF16, 2)):
        p = tk.tucker_plan(L, K, dtype)
        nodes = tk.tucker_plan_nodes(p)
        roots = [i for i, nd in enumerate(nodes) if nd["parent"] == 0 and nd["label"] >= 0]
        f = tk.tucker_plan_fused_root(p)
        a = min(nodes[roots[0]]["label"], nodes[roots[1]]["label"])
        fits = math.prod(L[a:]) * es <= 8192
        if dtype == tk.TUCKER_F32:
            assert f is not None or not fits
        if f is None:
            continue
        assert f == (roots[0], roots[1])
        u1, u2 = f
        sub = {u1}
        for i, nd in enumerate(nodes):
            if nd["parent"] in sub:
                sub.add(i)
        b0 = nodes[u2]["ws_offset"]
        b1 = b0 + es * nodes[u2]["out_elems"]
        for i in sub:
            if nodes[i]["label"] < 0:
                continue
            a0 = nodes[i]["ws_offset"]
            a1 = a0 + es * nodes[i]["out_elems"]
            assert a1 <= b0 or b1 <= a0, (L, i)
        assert b1 <= tk.tucker_plan_cost(p)["ws_bytes"]
        q = tk.tucker_plan(L, K, dtype, fuse_root=False)
        assert tk.tucker_plan_fused_root(q) is None
        assert tk.tucker_plan_cost(q)["tree_macs"] == tk.tucker_plan_cost(p)["tree_macs"]


def test_plan_flags_validated(tk):
    import ctypes
    h = ctypes.c_void_p()
    L = (tk._i64((8, 4, 4)))
    K = (tk._i64((3, 2, 2)))
    opts = tk.PlanOpts(tk.TUCKER_F32, tk.TREE_OPTIMAL, tk.COST_MACS, 4)
    assert tk.lib().tucker_plan(3, L, K, ctypes.byref(opts), ctypes.byref(h)) == -1
    # the trailing block of 200^4 (64 MB) is too large for the fused kernel:
    # by default its plans keep the root children apart; made under the
    # tensor-core pair policy bits (32 for FP32, 256 for BF16) they take the
    # L2-blocked pair (modes 0 and 2, blocked by mode 1); FP8 plans never do
    for dt in (tk.TUCKER_F32, tk.TUCKER_BF16, tk.TUCKER_FP8_E4M3):
        assert tk.tucker_plan_fused_root(tk.tucker_plan((200,) * 4, (20,) * 4, dt)) is None
    for dt, pol in ((tk.TUCKER_F32, 32), (tk.TUCKER_BF16, 256), (tk.TUCKER_FP8_E4M3, 32 | 256)):
        assert tk.lib().tucker_set_kernel_policy(pol) == 0
        try:
            p = tk.tucker_plan((200,) * 4, (20,) * 4, dt)
            f = tk.tucker_plan_fused_root(p)
            if dt == tk.TUCKER_FP8_E4M3:
                assert f is None
                continue
            assert f is not None
            nodes = tk.tucker_plan_nodes(p)
            assert sorted(nodes[u]["label"] for u in f) == [0, 2]
            # the pair needs a 16-byte row stride and K within the kernel's
            # accumulators (32 for FP32, 64 for BF16)
            kbig = 40 if dt == tk.TUCKER_F32 else 80
            assert tk.tucker_plan_fused_root(tk.tucker_plan((200,) * 4, (kbig,) * 4, dt)) is None
            assert tk.tucker_plan_fused_root(tk.tucker_plan((200, 200, 200, 201), (20,) * 4, dt)) is None
        finally:
            tk.lib().tucker_set_kernel_policy(0)


def test_elems_cost_model(tk, orc):
    # the elements-moved objective never moves more elements than the MAC tree
    for L, K in [((672, 672, 627, 16), (279, 279, 153, 14)),
                 ((500, 500, 500, 11, 10), (81, 129, 127, 7, 6))]:
        pm = tk.tucker_plan(L, K)
        pe = tk.tucker_plan(L, K, cost_model=tk.COST_ELEMS)
        cm, ce = tk.tucker_plan_cost(pm), tk.tucker_plan_cost(pe)
        assert ce["tree_elems"] <= cm["tree_elems"]
        assert cm["tree_macs"] <= ce["tree_macs"]
        labels, parents, _ = tree_of(tk, pe)
        assert orc.tree_cost(L, K, labels, parents) == ce["tree_macs"]


def test_sthosvd_order_matches_bruteforce(tk, orc):
    """The planner's STHOSVD order (DP over the set of truncated modes) reaches
    the least cost of all N! orders, under both objectives; its reported cost
    is the oracle's cost of the order it returns; natural order whenever that
    is optimal, and always without the flag."""
    # shapes the planner accepts (K_n <= product of the other K); the brute
    # force itself is pinned to hand-derived costs in the planner-oracle tests
    cases = [((10, 2, 10), (2, 1, 2)), ((10, 2, 10, 7), (6, 1, 2, 3)), ((40, 12, 30, 25), (3, 10, 4, 20)),
             ((672, 672, 33, 627), (279, 279, 29, 153)), ((200,) * 4, (20,) * 4)]
    rnd = random.Random(11)
    for _ in range(60):
        N = rnd.choice([2, 3, 4, 5, 6])
        L = [rnd.choice([2, 3, 5, 8, 13, 40, 97]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        if all(K[n] <= math.prod(K) // K[n] for n in range(N)):
            cases.append((L, K))
    for L, K in cases:
        for cm, elems in ((tk.COST_MACS, False), (tk.COST_ELEMS, True)):
            best, _, nat = orc.sthosvd_order_bruteforce(L, K, elems)
            order, cost = tk.tucker_plan_sthosvd(tk.tucker_plan(L, K, cost_model=cm, sthosvd_order=True))
            assert sorted(order) == list(range(len(L)))
            assert cost == best == orc.sthosvd_order_cost(L, K, order, elems), (L, K, elems)
            if nat == best:
                assert order == list(range(len(L))), (L, K, elems, order)
            order0, cost0 = tk.tucker_plan_sthosvd(tk.tucker_plan(L, K, cost_model=cm))
            assert order0 == list(range(len(L))) and cost0 == nat
    assert sum(1 for L, K in cases if orc.sthosvd_order_bruteforce(L, K)[2] >
               orc.sthosvd_order_bruteforce(L, K)[0]) >= 10


def test_plan_sthosvd_rejects_null(tk):
    import ctypes
    order = (ctypes.c_int * 4)()
    assert tk.lib().tucker_plan_sthosvd(None, order, None) == -1
    p = tk.tucker_plan((10, 2, 10, 7), (6, 1, 2, 3))
    assert tk.lib().tucker_plan_sthosvd(p.handle, None, None) == -1
    assert tk.lib().tucker_plan_sthosvd(p.handle, order, None) == 0 and list(order) == [0, 1, 2, 3]


def test_sthosvd_order_workspace_covers_the_order(tk):
    """The workspace of a plan with an optimised STHOSVD order holds two
    buffers of the largest tensor after any step of that order."""
    L, K = (10, 2, 10, 7), (6, 1, 2, 3)
    p = tk.tucker_plan(L, K, sthosvd_order=True)
    order, _ = tk.tucker_plan_sthosvd(p)
    assert order != [0, 1, 2, 3]
    mx, P = 0, set()
    for m in order[:-1]:
        P.add(m)
        mx = max(mx, math.prod(K[n] if n in P else L[n] for n in range(4)))
    assert tk.tucker_plan_cost(p)["ws_bytes"] >= 2 * 4 * mx


def test_batch_plan_layout(tk):
    """The batched form packs tensors, factors and cores back to back in the
    order of the batch (host only)."""
    import math

    import workloads
    dims, ranks = workloads.batch_shapes(37, 4)
    b = tk.BatchPlan(dims, ranks)
    sizes = [math.prod(d) for d in dims]
    assert b.t_elems == sum(sizes)
    assert b.t_off == [sum(sizes[:i]) for i in range(37)]
    fs = [dims[i][n] * ranks[i][n] for i in range(37) for n in range(3)]
    assert b.f_off == [sum(fs[:j]) for j in range(len(fs))]
    assert b.f_elems == sum(fs)
    gs = [math.prod(r) for r in ranks]
    assert b.g_off == [sum(gs[:i]) for i in range(37)] and b.g_elems == sum(gs)
    assert b.ws_bytes > 4 * b.t_elems // 10


def test_batch_tuning_defaults_before_autotune(tk):
    """Before tucker_batch_autotune every sweep site holds the default launch
    configuration (one position per thread, rows shorter than 32 staged, plan
    order) and no timings; the sites are the tree levels, the core step and
    the N reconstruction steps of the fit (host only)."""
    import workloads
    dims, ranks = workloads.batch_shapes(19, 4)
    b = tk.BatchPlan(dims, ranks)
    sites = tk.tucker_batch_tuning(b)
    kinds = [s["site"] for s in sites]
    assert kinds.count("core") == 1 and kinds.count("fit") == 3
    assert kinds == ["level"] * kinds.count("level") + ["core"] + ["fit"] * 3
    assert 1 <= kinds.count("level") <= 2  # 3-way trees: depth 2 at most below the root
    for s in sites:
        assert (s["ppt"], s["stage_c"], s["order"], s["async"]) == (1, 32, 0, 0)
        assert s["ms_default"] == -1.0 and s["ms_tuned"] == -1.0


def test_batch_set_tuning_round_trip_and_validation(tk):
    """Configurations set through tucker_batch_set_tuning read back the same;
    out-of-order sites and out-of-range values are refused (host only)."""
    import copy

    import workloads
    dims, ranks = workloads.batch_shapes(11, 5)
    b = tk.BatchPlan(dims, ranks)
    sites = tk.tucker_batch_tuning(b)
    new = copy.deepcopy(sites)
    for i, s in enumerate(new):
        s["ppt"] = 2
        s["order"] = i % 2
        if s["site"] != "fit":
            s["stage_c"] = (0, 16, 64)[i % 3]
            if i % 2:
                s["ppt"], s["async"] = 1, 1
    tk.tucker_batch_set_tuning(b, new)
    got = tk.tucker_batch_tuning(b)
    for s, g in zip(new, got):
        assert (g["ppt"], g["order"], g["async"]) == (s["ppt"], s["order"], s["async"])
        assert g["stage_c"] == (s["stage_c"] if s["site"] != "fit" else 32)
    for bad in ({"ppt": 3}, {"ppt": 4}, {"stage_c": 65}, {"order": 2}, {"index": 7},
                {"async": 2}, {"async": 1, "ppt": 2}):
        wrong = copy.deepcopy(sites)
        wrong[0].update(bad)
        with pytest.raises(tk.TuckerError) as e:
            tk.tucker_batch_set_tuning(b, wrong)
        assert e.value.code == -1
    with pytest.raises(tk.TuckerError):
        tk.tucker_batch_set_tuning(b, sites[:-1])
    fit = copy.deepcopy(sites)
    fit[-1]["async"] = 1  # reconstruction steps have no cp.async variant
    with pytest.raises(tk.TuckerError):
        tk.tucker_batch_set_tuning(b, fit)


@pytest.mark.parametrize("dims,ranks,msg", [
    ([(20, 20, 201)], [(4, 4, 4)], "L_n <= 200"),
    ([(40, 40, 40)], [(33, 33, 33)], "K_n <= 32"),
    ([(10, 10, 10)], [(9, 1, 1)], "product of the other"),
])
def test_batch_plan_validation(tk, dims, ranks, msg):
    with pytest.raises(tk.TuckerError) as e:
        tk.BatchPlan(dims, ranks)
    assert msg in str(e.value)


def test_optimal_tree_never_above_prior_trees_on_benchmark_metadata(tk):
    """Sec. 6 benchmark metadata (L_n in {20, 50, 100, 400}, K_n = L_n / c,
    c in {1.25, 2, 5, 10}): the optimal tree's load is at most that of the
    chain (K-order, h-order) and balanced trees of Sec. 3.2, on a seeded
    sample of 5-D and 6-D inputs."""
    import math
    modes = [(L, int(round(L / c))) for L in (20, 50, 100, 400) for c in (1.25, 2, 5, 10)]
    rng = random.Random(7)
    checked = 0
    while checked < 150:
        N = rng.choice((5, 6))
        pick = [rng.choice(modes) for _ in range(N)]
        L = [p[0] for p in pick]
        K = [p[1] for p in pick]
        if math.prod(L) > 8e9:
            continue
        try:
            opt = tk.tucker_plan_cost(tk.tucker_plan(L, K))["tree_macs"]
        except tk.TuckerError:
            continue
        for tree in (tk.TREE_CHAIN_K, tk.TREE_CHAIN_H, tk.TREE_BALANCED, tk.TREE_CHAIN):
            other = tk.tucker_plan_cost(tk.tucker_plan(L, K, tree=tree))["tree_macs"]
            assert opt <= other, (L, K, tree)
        checked += 1


def test_eig_wrappers_reject_bad_factor_types(tk):
    # the C entry points see only raw pointers: the binding must refuse a
    # factor type the solver does not write, a mixed list, a non-double W and
    # a factor whose row count is not W's size, before anything is launched
    import torch
    W = torch.eye(8, dtype=torch.float64)
    cases = [
        ([W], [torch.empty(8, 2, dtype=torch.bfloat16)], TypeError),
        ([W, W], [torch.empty(8, 2, dtype=torch.float32), torch.empty(8, 2, dtype=torch.float64)],
         TypeError),
        ([W.float()], [torch.empty(8, 2, dtype=torch.float32)], TypeError),
        ([W], [torch.empty(7, 2, dtype=torch.float32)], ValueError),
        ([W, W], [torch.empty(8, 2, dtype=torch.float32)], ValueError),
    ]
    ws = torch.empty(256, dtype=torch.uint8)
    for Ws, Fs, exc in cases:
        with pytest.raises(exc):
            tk.tucker_eig_topk(Ws, Fs, ws)
        with pytest.raises(exc):
            tk.tucker_eig_topk_noalloc(Ws, Fs)


def test_eig_entry_points_reject_unknown_factor_dtype(tk):
    # the host-side check of the C ABI runs before any device work
    import ctypes
    L = tk.lib()
    Ls, Ks = tk._i64([8]), tk._i64([2])
    ptrs = (ctypes.c_void_p * 1)(ctypes.c_void_p(256))
    for code in (tk.TUCKER_BF16, tk.TUCKER_FP8_E4M3, 7):
        rc = L.tucker_eig_topk(1, Ls, Ks, ptrs, ptrs, code, ctypes.c_void_p(256), 4096, None)
        assert rc == -1
        assert b"f_dtype" in L.tucker_last_error()
        rc = L.tucker_eig_topk_noalloc(1, Ls, Ks, ptrs, ptrs, code, None)
        assert rc == -1


def test_workspace_cap_trades_fused_root_then_sthosvd_order(tk):
    """A workspace cap gives up the fused root first (the 6-way workload's
    plan fuses its root and needs more workspace for it), then the least-cost
    STHOSVD order, and otherwise fails with TUCKER_ERR_WORKSPACE; the tree
    and its cost never change."""
    L, K = (64, 56, 48, 40, 32, 24), (16, 14, 12, 10, 8, 6)
    full = tk.tucker_plan(L, K, sthosvd_order=True)
    nofuse = tk.tucker_plan(L, K, fuse_root=False, sthosvd_order=True)
    natural = tk.tucker_plan(L, K, fuse_root=False)
    w_full, w_nf, w_nat = (tk.tucker_plan_cost(p)["ws_bytes"] for p in (full, nofuse, natural))
    assert tk.tucker_plan_fused_root(full) is not None and w_full > w_nf
    # a cap at or above the full plan's need changes nothing
    p = tk.tucker_plan(L, K, sthosvd_order=True, ws_cap=w_full)
    assert tk.tucker_plan_fused_root(p) is not None
    assert tk.tucker_plan_cost(p)["ws_bytes"] == w_full
    # just below: the fused root goes, the STHOSVD order stays
    p = tk.tucker_plan(L, K, sthosvd_order=True, ws_cap=w_full - 1)
    assert tk.tucker_plan_fused_root(p) is None
    assert tk.tucker_plan_cost(p)["ws_bytes"] == w_nf
    assert tk.tucker_plan_sthosvd(p)[0] == tk.tucker_plan_sthosvd(nofuse)[0]
    assert tk.tucker_plan_cost(p)["tree_macs"] == tk.tucker_plan_cost(full)["tree_macs"]
    # the STHOSVD order is given up when only that meets the cap
    if w_nat < w_nf:
        p = tk.tucker_plan(L, K, sthosvd_order=True, ws_cap=w_nf - 1)
        assert tk.tucker_plan_sthosvd(p)[0] == list(range(len(L)))
        assert tk.tucker_plan_cost(p)["ws_bytes"] == w_nat
    # below every layout: TUCKER_ERR_WORKSPACE naming the smallest size
    with pytest.raises(tk.TuckerError) as e:
        tk.tucker_plan(L, K, sthosvd_order=True, ws_cap=min(w_nf, w_nat) - 1)
    assert e.value.code == -3
    assert str(min(w_nf, w_nat)) in str(e.value)


def test_workspace_cap_gives_up_the_sthosvd_order(tk):
    """On 64 x 64 x 32 with ranks 16 the least-cost STHOSVD order takes mode 2
    first, whose ping-pong buffers are larger than the natural order's: a cap
    between the two sizes keeps the plan with the natural order."""
    L, K = (64, 64, 32), (16, 16, 16)
    opt = tk.tucker_plan(L, K, sthosvd_order=True)
    nat = tk.tucker_plan(L, K)
    w_opt, w_nat = tk.tucker_plan_cost(opt)["ws_bytes"], tk.tucker_plan_cost(nat)["ws_bytes"]
    assert w_nat < w_opt and tk.tucker_plan_sthosvd(opt)[0] != [0, 1, 2]
    p = tk.tucker_plan(L, K, sthosvd_order=True, ws_cap=w_opt - 1)
    assert tk.tucker_plan_sthosvd(p)[0] == [0, 1, 2]
    assert tk.tucker_plan_cost(p)["ws_bytes"] == w_nat <= w_opt - 1
