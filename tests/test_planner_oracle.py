"""Pins of the planner oracle (Sec. 3): hand-derived costs, hand-counted
trees, exhaustive enumeration of every TTM-tree against the recurrence, and
the Remark that always reusing a mode is not optimal."""
import json
import os
import random

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "planner_costs.json")


def test_hand_derived_costs(orc):
    data = json.load(open(GOLD))
    for case in data["cases"]:
        L, K = case["L"], case["K"]
        assert orc.chain_cost(L, K) == case["chain_natural"]
        assert orc.balanced_cost(L, K) == case["balanced"]
        assert orc.tree_dp(L, K) == case["optimal"]
        cnt, mn, mx = orc.tree_bruteforce(L, K)
        assert mn == case["optimal"]
        assert mx >= case["chain_natural"]


def test_hand_derived_ordered_chains(orc):
    # Sec. 3.2 mode orderings: K-order by increasing K_n, h-order by
    # increasing K_n / L_n; the chain costs under each were worked by hand
    data = json.load(open(GOLD))["ordered_chains"]
    for case in data["cases"]:
        L, K = case["L"], case["K"]
        assert orc.k_order(L, K) == case["k_order"]
        assert orc.h_order(L, K) == case["h_order"]
        assert orc.chain_cost(L, K, orc.k_order(L, K)) == case["chain_k_order"]
        assert orc.chain_cost(L, K, orc.h_order(L, K)) == case["chain_h_order"]
        assert orc.chain_cost(L, K) == case["chain_natural"]
        if "chain_k_reversed" in case:
            assert orc.chain_cost(L, K, orc.k_order(L, K)[::-1]) == case["chain_k_reversed"]
            assert orc.chain_cost(L, K, orc.h_order(L, K)[::-1]) == case["chain_h_reversed"]


def test_hand_counted_tree_numbers(orc):
    data = json.load(open(GOLD))["tree_counts"]
    for n_str, count in data.items():
        if n_str.startswith("_"):
            continue
        N = int(n_str)
        cnt, _, _ = orc.tree_bruteforce([3] * N, [2] * N)
        assert cnt == count


def test_bruteforce_equals_dp_random_small(orc):
    rnd = random.Random(7)
    for trial in range(150):
        N = rnd.choice([2, 3, 4])
        L = [rnd.choice([2, 3, 5, 8, 20, 50]) for _ in range(N)]
        K = [rnd.randint(1, l) for l in L]
        cnt, mn, mx = orc.tree_bruteforce(L, K)
        assert mn == orc.tree_dp(L, K), (L, K)
        # the chain and balanced trees are TTM-trees, so they cost at least the optimum
        assert orc.chain_cost(L, K) >= mn
        assert orc.balanced_cost(L, K) >= mn
        assert orc.chain_cost(L, K, orc.k_order(L, K)) >= mn
        assert orc.chain_cost(L, K, orc.h_order(L, K)) >= mn
        if N == 4:
            assert cnt == 4092


@pytest.mark.slow
def test_bruteforce_equals_dp_five_modes(orc):
    # N = 5 has tens of millions of trees; two instances keep the run short.
    for L, K in [((8, 12, 6, 10, 9), (3, 5, 2, 7, 4)), ((20, 50, 20, 100, 400), (10, 25, 16, 20, 40))]:
        cnt, mn, _ = orc.tree_bruteforce(L, K)
        assert cnt == 40241424
        assert mn == orc.tree_dp(L, K)


def test_always_reuse_is_not_optimal(orc):
    # Remark after the recurrence (Sec. 3.3): the optimal tree may decline a
    # reusable mode.  This 5-mode instance shows it; the DP without that
    # restriction agrees with exhaustive enumeration.
    L, K = (8, 400, 8, 64, 400), (5, 378, 8, 3, 302)
    opt = orc.tree_dp(L, K)
    greedy = orc.tree_dp(L, K, greedy=True)
    assert greedy > opt
    assert opt == 270174029056
    assert greedy == 270194130176


def test_balanced_and_chain_counts_match_section_3_2(orc):
    # chain trees perform N(N-1) TTMs; with all K_n = L_n every TTM costs
    # L*|T|, which exposes the TTM count directly.
    for N in (2, 3, 4, 5):
        L = [3] * N
        cost = orc.chain_cost(L, L)
        assert cost == N * (N - 1) * 3 * 3 ** N
    # balanced tree for N = 4 has 8 internal nodes (Fig. "Example TTM-trees" (c))
    assert orc.balanced_cost([3] * 4, [3] * 4) == 8 * 3 * 3 ** 4


def test_tree_validator(orc):
    # the N = 3 optimal tree for L=(2,3,4), K=(1,2,3), written out by hand
    #  0 root; 1: x2 (mode 1); 2: x3 under 1 -> leaf F1; 3: x1 under 1 -> leaf F3
    #  4: x1 under root; 5: x3 under 4 -> leaf F2
    labels = [-1, 1, 2, 0, 0, 2, -2, -4, -3]
    parents = [-1, 0, 1, 1, 0, 4, 2, 3, 5]
    assert orc.tree_cost((2, 3, 4), (1, 2, 3), labels, parents) == 172
    bad = list(parents)
    bad[7] = 2  # leaf F3 under a path that lacks mode 1
    assert orc.tree_cost((2, 3, 4), (1, 2, 3), labels, bad) is None


# ----------------------------------------------------- STHOSVD mode order ----
GOLD_STH = os.path.join(os.path.dirname(__file__), "golden", "sthosvd_order_costs.json")


def test_sthosvd_order_hand_derived_costs(orc):
    """Every order of three hand-worked cases (multiply-adds and elements
    moved), and the brute-force optimum, against the written-out derivations;
    the third case has different optima under the two objectives."""
    for case in json.load(open(GOLD_STH))["cases"]:
        L, K = case["L"], case["K"]
        for key, elems in (("macs", False), ("elems", True)):
            for order, cost in case[key].items():
                assert orc.sthosvd_order_cost(L, K, [int(m) for m in order.split(",")], elems) == cost
            best, arg, nat = orc.sthosvd_order_bruteforce(L, K, elems)
            assert [best, arg] == case["best_" + key]
            assert nat == case[key][",".join(str(n) for n in range(len(L)))]


def test_sthosvd_order_cost_properties(orc):
    """Symmetric shapes cost the same in every order; a non-permutation is
    rejected; the step cost is the sum of a Gram and a TTM, so with K = L (no
    truncation) every order costs N * 2 * L * |T| when all L are equal."""
    import itertools
    L, K = (6, 6, 6, 6), (2, 2, 2, 2)
    costs = {orc.sthosvd_order_cost(L, K, p) for p in itertools.permutations(range(4))}
    assert len(costs) == 1
    assert orc.sthosvd_order_cost(L, K, [0, 0, 1, 2]) == 2 ** 64 - 1
    assert orc.sthosvd_order_cost((5, 5, 5), (5, 5, 5), [2, 0, 1]) == 3 * 2 * 5 * 125


# -------------------------------------------- elements-moved node cost -------
def test_elems_model_hand_derived(orc):
    """Elements moved (|In| + |Out| per internal node) on 4^3, K = 2: a first
    TTM moves 64 + 32 = 96, a second 32 + 16 = 48.  Chain trees: 3 chains of
    96 + 48 = 432 (the most any of the 14 trees moves).  Optimal: the root's
    output is read by at least two first-level TTMs (96 each) and each of the
    3 leaves needs one more TTM (48 each): 2*96 + 3*48 = 336, reached by the
    balanced tree."""
    cnt, mn, mx = orc.tree_bruteforce((4, 4, 4), (2, 2, 2), elems=True)
    assert (cnt, mn, mx) == (14, 336, 432)
    # balanced tree of Sec. 3.2 as (label, parent): root; x0 -> {x1 -> F2, x2 -> F1}; x1 -> x2 -> F0
    labels = [-1, 0, 1, -4, 2, -3, 1, 2, -2]
    parents = [-1, 0, 1, 2, 1, 4, 0, 6, 7]
    assert orc.tree_cost((4, 4, 4), (2, 2, 2), labels, parents, elems=True) == 336
    assert orc.tree_cost((4, 4, 4), (2, 2, 2), labels, parents) == 448


def test_elems_model_scales_on_uniform_shapes(orc):
    """With every L_n = L and K_n = K a node moves |In| (1 + K / L) elements
    for K |In| multiply-adds, so every tree's two costs differ by the factor
    (L + K) / (L K): the least and the largest costs scale exactly."""
    rnd = random.Random(3)
    for _ in range(12):
        N = rnd.choice([2, 3, 4])
        l = rnd.choice([3, 5, 8, 20])
        k = rnd.randint(1, l)
        _, mn_m, mx_m = orc.tree_bruteforce([l] * N, [k] * N)
        _, mn_e, mx_e = orc.tree_bruteforce([l] * N, [k] * N, elems=True)
        assert mn_m * (l + k) == mn_e * l * k and mx_m * (l + k) == mx_e * l * k


# --------------------------------------------------- new-core chain order ----
def test_core_chain_hand_derived_costs(orc):
    """Every order of three hand-worked new-core chains and the least cost."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "core_chain_costs.json")))
    for case in gold["cases"]:
        L, K = case["L"], case["K"]
        for order, cost in case["orders"].items():
            assert orc.core_chain_cost(L, K, [int(m) for m in order.split(",")]) == cost
        assert orc.core_chain_bruteforce(L, K) == case["best"]
    assert orc.core_chain_cost((4, 4, 4), (2, 2, 2), [0, 0, 1]) == 2 ** 64 - 1
