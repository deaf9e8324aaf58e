import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _debug_build_index_check(request):
    """Under the index-checked debug build (TUCKER_LIB_VARIANT=debug), every
    GPU test also asserts that no kernel recorded an out-of-range index."""
    yield
    if os.environ.get("TUCKER_LIB_VARIANT", "") != "debug" or request.node.get_closest_marker("gpu") is None:
        return
    import paper_1707_05594_gb300 as tk
    if tk._lib is None:
        return
    rec = tk.tucker_debug_check(reset=True)
    assert rec["count"] == 0, f"out-of-range global index in the debug build: {rec}"
