"""Host checks of bench.py's analysis code: the fit of measured sweep times
against tree costs (used by --planner-gpu) recovers an exact linear law."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    return pkg


def test_tree_time_fit_recovers_a_bytes_law(tk):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    trees = {"opt": tk.TREE_OPTIMAL, "chain_k": tk.TREE_CHAIN_K, "balanced": tk.TREE_BALANCED}
    rows = []
    for L, K in [((50,) * 5, (25, 5, 5, 5, 5)), ((20, 50, 50, 100, 100), (4, 40, 40, 20, 20))]:
        ms = {}
        for name, tree in trees.items():
            c = tk.tucker_plan_cost(tk.tucker_plan(L, K, tk.TUCKER_F32, tree))
            ms[name] = 0.4 * c["tree_elems"] * 4 / 1e9  # exactly 0.4 ms per GB moved
        rows.append({"L": list(L), "K": list(K), "ms_per_sweep": ms})
    fit = bench.tree_time_fit(rows, trees)
    assert fit["pairs"] == 6
    assert fit["gb_moved"]["rms_rel_err"] < 1e-9
    assert math.isclose(fit["gb_moved"]["ms_per_unit"][0], 0.4, rel_tol=1e-6)
    assert fit["gmacs"]["rms_rel_err"] > 0.01  # multiply-adds do not follow this law
    assert bench.tree_time_fit(rows[:1][:0], trees) is None
