"""The index-checked debug build (the library compiled with -DTUCKER_DEBUG;
tucker_debug_build / tucker_debug_check in include/tucker.h).

On the CPU: it compiles, exports every symbol the header declares, reports
itself as the debug build, and the normal build reports no records without
touching a device.  On the GPU: the ragged-shape parity suites run again
against the debug build in a child process; tests/conftest.py then asserts
after every GPU test that no kernel recorded an out-of-range index, and the
parity assertions themselves still hold with the checks compiled in."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "tests"))
from test_library_host import declared_symbols  # noqa: E402


@pytest.fixture(scope="module")
def debug_lib():
    from paper_1707_05594_gb300 import build
    return build.build(debug=True)


def test_debug_build_exports_and_identifies_itself(debug_lib):
    L = ctypes.CDLL(debug_lib)
    for n in declared_symbols():
        assert hasattr(L, n), n
    assert L.tucker_debug_build() == 1


def test_normal_build_has_no_records():
    from paper_1707_05594_gb300 import build
    L = ctypes.CDLL(build.build())
    assert L.tucker_debug_build() == 0
    idx, bnd, line = ctypes.c_int64(7), ctypes.c_int64(7), ctypes.c_int(7)
    buf = ctypes.create_string_buffer(8)
    # the normal build answers without a device: zero records, outputs cleared
    assert L.tucker_debug_check(ctypes.byref(idx), ctypes.byref(bnd), ctypes.byref(line), buf, 8, 1) == 0
    assert (idx.value, bnd.value, line.value, buf.value) == (0, 0, 0, b"")


# ragged shapes of every kernel family: CUDA-core and tensor-core TTMs (all
# storage types), Grams, short-row and fused-root kernels, FP8, the split
# storage, the batched form, and the workspace canary's sweeps
SUITES = ["tests/test_gpu_kernels.py", "tests/test_gpu_gram_tc.py", "tests/test_gpu_fused_root.py",
          "tests/test_gpu_fp8.py", "tests/test_gpu_split.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_canary.py", "tests/test_gpu_f32_tc.py"]


@pytest.mark.gpu
def test_parity_suites_under_the_debug_build(debug_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, TUCKER_LIB_VARIANT="debug")
    suites = [s for s in SUITES if os.path.exists(os.path.join(ROOT, s))]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        *suites], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
