"""Plain FP64 CPU oracle for dense Tucker decomposition (STHOSVD + HOOI) and
for the TTM-tree planner.

TEST INFRASTRUCTURE ONLY: this package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` -- nothing else.  It shares no code with the CUDA path
(``paper_1707_05594_gb300``) and never imports it.

The arithmetic lives in ``oracle.c`` / ``planner_oracle.c`` / ``fp8_oracle.c``
(plain C, double precision, naive loops); this module only marshals numpy
arrays.

Citations are to the paper: Sec. 1 (STHOSVD, and that the tree ideas carry
over to it: its mode order), Sec. 2.1 (TTM, TTM-chain), Sec. 2.2 and Fig. 2
(Tucker model, HOOI, new core), Sec. 3.1-3.3 (TTM-trees, cost, recurrence),
Sec. 5 (SVD via Gram + EVD).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "planner_oracle.c"),
         os.path.join(_HERE, "fp8_oracle.c")]

_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_u64 = ctypes.c_ulonglong
ORC_INF = 0xFFFFFFFFFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``_liboracle.so`` (gcc, -fopenmp)."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    lib.orc_ttm_d.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, _dp, ctypes.c_int64, _dp]
    lib.orc_ttm_f.argtypes = [ctypes.c_int, _i64p, ctypes.c_void_p, ctypes.c_int, _dp,
                              ctypes.c_int64, _dp]
    lib.orc_gram.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, _dp]
    lib.orc_jacobi_eig.argtypes = [ctypes.c_int64, _dp, _dp, _dp]
    lib.orc_jacobi_eig.restype = ctypes.c_int
    lib.orc_hooi_sweep.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.POINTER(_dp), ctypes.POINTER(_dp), _dp, ctypes.c_int]
    lib.orc_hooi_sweep.restype = ctypes.c_int
    lib.orc_core.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_void_p, ctypes.c_int,
                             ctypes.POINTER(_dp), _dp]
    lib.orc_sthosvd.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_void_p, ctypes.c_int,
                                ctypes.POINTER(_dp), _dp, _dp]
    lib.orc_sthosvd.restype = ctypes.c_int
    lib.orc_sthosvd_order.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_dp), _dp, _dp]
    lib.orc_sthosvd_order.restype = ctypes.c_int
    lib.orc_norm2_d.argtypes = [ctypes.c_int64, _dp]
    lib.orc_norm2_d.restype = ctypes.c_double
    lib.orc_norm2_f.argtypes = [ctypes.c_int64, ctypes.c_void_p]
    lib.orc_norm2_f.restype = ctypes.c_double
    lib.orc_fit.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_fit.restype = ctypes.c_double
    lib.orc_reconstruct.argtypes = [ctypes.c_int, _i64p, _i64p, _dp, ctypes.POINTER(_dp), _dp]
    lib.orc_residual.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_void_p, ctypes.c_int, _dp,
                                 ctypes.POINTER(_dp)]
    lib.orc_residual.restype = ctypes.c_double
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    # planner oracle
    lib.orc_tree_bruteforce.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(_u64),
                                        ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
    lib.orc_tree_bruteforce.restype = ctypes.c_int
    lib.orc_tree_bruteforce_model.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, ctypes.POINTER(_u64),
                                              ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
    lib.orc_tree_bruteforce_model.restype = ctypes.c_int
    lib.orc_tree_cost_model.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.orc_tree_cost_model.restype = _u64
    lib.orc_tree_dp.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int]
    lib.orc_tree_dp.restype = _u64
    lib.orc_chain_cost.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.orc_chain_cost.restype = _u64
    lib.orc_balanced_cost.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.orc_balanced_cost.restype = _u64
    lib.orc_tree_cost.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.orc_tree_cost.restype = _u64
    lib.orc_core_chain_cost.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.orc_core_chain_cost.restype = _u64
    lib.orc_core_chain_bruteforce.argtypes = [ctypes.c_int, _i64p, _i64p]
    lib.orc_core_chain_bruteforce.restype = _u64
    lib.orc_sthosvd_order_cost.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_int]
    lib.orc_sthosvd_order_cost.restype = _u64
    lib.orc_sthosvd_order_bruteforce.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_u64),
                                                 ctypes.POINTER(_u64)]
    lib.orc_sthosvd_order_bruteforce.restype = ctypes.c_int
    # FP8 E4M3 storage with per-64 scales
    lib.orc_e4m3_decode.argtypes = [ctypes.c_int]
    lib.orc_e4m3_decode.restype = ctypes.c_double
    lib.orc_e4m3_encode.argtypes = [ctypes.c_float]
    lib.orc_e4m3_encode.restype = ctypes.c_int
    lib.orc_fp8_quantize.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    lib.orc_fp8_dequantize.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, _dp]
    _lib = lib
    return lib


def _i64(a: Sequence[int]):
    arr = (ctypes.c_int64 * len(a))(*[int(x) for x in a])
    return arr


def _dptr(x: np.ndarray):
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(_dp)


def _tensor_arg(T: np.ndarray):
    T = np.ascontiguousarray(T)
    if T.dtype == np.float32:
        return T, T.ctypes.data_as(ctypes.c_void_p), 1
    if T.dtype == np.float64:
        return T, T.ctypes.data_as(ctypes.c_void_p), 0
    raise TypeError("oracle tensors are float32 or float64")


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


# --------------------------------------------------------------------------
# Sec. 2.1 TTM
# --------------------------------------------------------------------------
def ttm(X: np.ndarray, n: int, A: np.ndarray) -> np.ndarray:
    """Z = X x_n A with A of size Kout x L_n (Sec. 2.1)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    dims = list(X.shape)
    assert A.shape[1] == dims[n]
    out_dims = dims.copy()
    out_dims[n] = A.shape[0]
    Y = np.empty(out_dims, dtype=np.float64)
    Xc, xp, is_f = _tensor_arg(X)
    if is_f:
        lib.orc_ttm_f(len(dims), _i64(dims), xp, n, _dptr(A), A.shape[0], _dptr(Y))
    else:
        lib.orc_ttm_d(len(dims), _i64(dims), Xc.ctypes.data_as(_dp), n, _dptr(A), A.shape[0],
                      _dptr(Y))
    return Y


def gram(Z: np.ndarray, n: int) -> np.ndarray:
    """W = Z_(n) Z_(n)^T (Sec. 5)."""
    lib = _load()
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    L = Z.shape[n]
    W = np.empty((L, L), dtype=np.float64)
    lib.orc_gram(Z.ndim, _i64(Z.shape), _dptr(Z), n, _dptr(W))
    return W


def jacobi_eig(A: np.ndarray):
    """All eigenpairs of a symmetric matrix by cyclic Jacobi: (evals desc,
    V with eigenvectors in columns, sweeps).  Sign: largest |entry| positive."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    ev = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.float64)
    sweeps = lib.orc_jacobi_eig(n, _dptr(A), _dptr(ev), _dptr(V))
    return ev, V, sweeps


def _fptrs(Fs):
    arr = (_dp * len(Fs))(*[_dptr(F) for F in Fs])
    return arr


def hooi_sweep(T: np.ndarray, Fs: Sequence[np.ndarray], K: Sequence[int],
               gauss_seidel: bool = False):
    """One HOOI invocation (Fig. 2) with chain trees.  Returns (F_new, G_new)."""
    lib = _load()
    L = list(T.shape)
    Fin = [np.ascontiguousarray(F, dtype=np.float64) for F in Fs]
    Fout = [np.empty((L[n], K[n]), dtype=np.float64) for n in range(len(L))]
    G = np.empty(list(K), dtype=np.float64)
    Tc, tp, is_f = _tensor_arg(T)
    rc = lib.orc_hooi_sweep(len(L), _i64(L), _i64(K), tp, is_f, _fptrs(Fin), _fptrs(Fout),
                            _dptr(G), 1 if gauss_seidel else 0)
    if rc < 0:
        raise RuntimeError("oracle Jacobi eigensolver did not converge")
    return Fout, G


def core(T: np.ndarray, Fs: Sequence[np.ndarray]) -> np.ndarray:
    """New core G = T x_1 F_1^T ... x_N F_N^T (Fig. 2)."""
    lib = _load()
    L = list(T.shape)
    K = [F.shape[1] for F in Fs]
    Fin = [np.ascontiguousarray(F, dtype=np.float64) for F in Fs]
    G = np.empty(K, dtype=np.float64)
    Tc, tp, is_f = _tensor_arg(T)
    lib.orc_core(len(L), _i64(L), _i64(K), tp, is_f, _fptrs(Fin), _dptr(G))
    return G


def sthosvd(T: np.ndarray, K: Sequence[int], return_evals: bool = False,
            order: Sequence[int] | None = None):
    """STHOSVD, the modes taken in natural order or in `order` (a permutation).

    Returns (F list, G[, per-mode eigenvalues]); mode n's eigenvalues are those
    of the Gram its factor came from, whatever the order."""
    lib = _load()
    L = list(T.shape)
    Fout = [np.empty((L[n], K[n]), dtype=np.float64) for n in range(len(L))]
    G = np.empty(list(K), dtype=np.float64)
    # mode n's Gram has size L[n] (mode n still has length L[n] when it is taken)
    ev = np.empty(sum(L), dtype=np.float64)
    Tc, tp, is_f = _tensor_arg(T)
    if order is None:
        rc = lib.orc_sthosvd(len(L), _i64(L), _i64(K), tp, is_f, _fptrs(Fout), _dptr(G), _dptr(ev))
    else:
        if len(order) != len(L):
            raise ValueError("order must list every mode once")
        perm = (ctypes.c_int * len(L))(*[int(m) for m in order])
        rc = lib.orc_sthosvd_order(len(L), _i64(L), _i64(K), tp, is_f, perm, _fptrs(Fout), _dptr(G),
                                   _dptr(ev))
        if rc == -2:
            raise ValueError("order must be a permutation of the modes")
    if rc < 0:
        raise RuntimeError("oracle Jacobi eigensolver did not converge")
    if return_evals:
        out, off = [], 0
        for n in range(len(L)):
            out.append(ev[off:off + L[n]].copy())
            off += L[n]
        return Fout, G, out
    return Fout, G


def norm2(X: np.ndarray) -> float:
    lib = _load()
    Xc, xp, is_f = _tensor_arg(X)
    if is_f:
        return lib.orc_norm2_f(Xc.size, xp)
    return lib.orc_norm2_d(Xc.size, Xc.ctypes.data_as(_dp))


def fit(normT2: float, normG2: float) -> float:
    """Sec. 2.2 error as fit = 1 - ||T - G x F|| / ||T||, via ||T||^2 - ||G||^2."""
    return _load().orc_fit(float(normT2), float(normG2))


def reconstruct(G: np.ndarray, Fs: Sequence[np.ndarray]) -> np.ndarray:
    lib = _load()
    G = np.ascontiguousarray(G, dtype=np.float64)
    K = list(G.shape)
    L = [F.shape[0] for F in Fs]
    Fin = [np.ascontiguousarray(F, dtype=np.float64) for F in Fs]
    out = np.empty(L, dtype=np.float64)
    lib.orc_reconstruct(len(L), _i64(L), _i64(K), _dptr(G), _fptrs(Fin), _dptr(out))
    return out


def residual(T: np.ndarray, G: np.ndarray, Fs: Sequence[np.ndarray]) -> float:
    """Direct ||T - G x_1 F_1 ... x_N F_N||_F."""
    lib = _load()
    L = list(T.shape)
    G = np.ascontiguousarray(G, dtype=np.float64)
    K = list(G.shape)
    Fin = [np.ascontiguousarray(F, dtype=np.float64) for F in Fs]
    Tc, tp, is_f = _tensor_arg(T)
    return lib.orc_residual(len(L), _i64(L), _i64(K), tp, is_f, _dptr(G), _fptrs(Fin))


# --------------------------------------------------------------------------
# Sec. 3 planner oracle
# --------------------------------------------------------------------------
def tree_bruteforce(L: Sequence[int], K: Sequence[int], elems: bool = False):
    """Enumerate every TTM-tree: (count, min cost, max cost) in MACs, or in
    elements moved (|In| + |Out| per internal node) with elems=True."""
    lib = _load()
    c, mn, mx = _u64(), _u64(), _u64()
    rc = lib.orc_tree_bruteforce_model(len(L), _i64(L), _i64(K), 1 if elems else 0, ctypes.byref(c),
                                       ctypes.byref(mn), ctypes.byref(mx))
    if rc != 0:
        raise ValueError("brute force supports 2 <= N <= 6")
    return c.value, mn.value, mx.value


def tree_dp(L: Sequence[int], K: Sequence[int], greedy: bool = False) -> int:
    """Optimal TTM-tree cost by the Sec. 3.3 recurrence (top-down, memoised)."""
    return int(_load().orc_tree_dp(len(L), _i64(L), _i64(K), 1 if greedy else 0))


def chain_cost(L: Sequence[int], K: Sequence[int], order: Sequence[int] | None = None) -> int:
    order = list(range(len(L))) if order is None else list(order)
    arr = (ctypes.c_int * len(order))(*order)
    return int(_load().orc_chain_cost(len(L), _i64(L), _i64(K), arr))


def k_order(L: Sequence[int], K: Sequence[int]):
    """Sec. 3.2 K-ordering: increasing K_n (stable)."""
    return sorted(range(len(L)), key=lambda n: K[n])


def h_order(L: Sequence[int], K: Sequence[int]):
    """Sec. 3.2 h-ordering: increasing h_n = K_n / L_n (stable; exact rational compare)."""
    from fractions import Fraction
    return sorted(range(len(L)), key=lambda n: Fraction(K[n], L[n]))


def balanced_cost(L: Sequence[int], K: Sequence[int], order: Sequence[int] | None = None) -> int:
    order = list(range(len(L))) if order is None else list(order)
    arr = (ctypes.c_int * len(order))(*order)
    return int(_load().orc_balanced_cost(len(L), _i64(L), _i64(K), arr))


def tree_cost(L: Sequence[int], K: Sequence[int], labels: Sequence[int], parents: Sequence[int],
              elems: bool = False):
    """Validate a tree (Sec. 3.1 properties i-iv) and return its cost (MACs, or
    elements moved with elems=True), or None."""
    n = len(labels)
    la = (ctypes.c_int * n)(*labels)
    pa = (ctypes.c_int * n)(*parents)
    r = int(_load().orc_tree_cost_model(len(L), _i64(L), _i64(K), n, la, pa, 1 if elems else 0))
    return None if r == ORC_INF else r


# --------------------------------------------------------------------------
def core_chain_cost(L: Sequence[int], K: Sequence[int], order: Sequence[int]) -> int:
    """Multiply-adds of the new-core chain (Fig. 2) with the modes in `order`."""
    arr = (ctypes.c_int * len(L))(*[int(m) for m in order])
    return int(_load().orc_core_chain_cost(len(L), _i64(L), _i64(K), arr))


def core_chain_bruteforce(L: Sequence[int], K: Sequence[int]) -> int:
    """Least new-core chain cost over all N! mode orders."""
    return int(_load().orc_core_chain_bruteforce(len(L), _i64(L), _i64(K)))


def sthosvd_order_cost(L: Sequence[int], K: Sequence[int], order: Sequence[int], elems: bool = False) -> int:
    """Cost of STHOSVD with the modes in `order`: multiply-adds (Gram L_m |Y| +
    TTM K_m |Y| per step) or elements moved (2 |Y| + |Y| K_m / L_m per step)."""
    arr = (ctypes.c_int * len(L))(*[int(m) for m in order])
    return int(_load().orc_sthosvd_order_cost(len(L), _i64(L), _i64(K), arr, 1 if elems else 0))


def sthosvd_order_bruteforce(L: Sequence[int], K: Sequence[int], elems: bool = False):
    """(least cost, the lexicographically first order reaching it, natural order's cost)
    over all N! mode orders of STHOSVD."""
    N = len(L)
    best = (ctypes.c_int * N)()
    bc, nc = _u64(), _u64()
    rc = _load().orc_sthosvd_order_bruteforce(N, _i64(L), _i64(K), 1 if elems else 0, best,
                                              ctypes.byref(bc), ctypes.byref(nc))
    if rc:
        raise ValueError("N out of range")
    return int(bc.value), list(best), int(nc.value)


# FP8 E4M3 storage with one FP32 scale per 64 consecutive elements
# --------------------------------------------------------------------------
def e4m3_decode(code: int) -> float:
    """Value of an E4M3 code (format definition; NaN for 0x7F / 0xFF)."""
    return _load().orc_e4m3_decode(int(code))


def e4m3_encode(v: float) -> int:
    """E4M3 code of v: round to nearest, ties to the even code, saturate at 448."""
    return _load().orc_e4m3_encode(float(v))


def fp8_quantize(x: np.ndarray):
    """Codes (uint8, same length) and scales (float32, one per 64 elements) of
    the flattened float32 array x: s = amax / 448 per slab, q = E4M3(x / s)."""
    lib = _load()
    xf = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    n = xf.size
    q = np.empty(n, dtype=np.uint8)
    s = np.empty((n + 63) // 64, dtype=np.float32)
    lib.orc_fp8_quantize(n, xf.ctypes.data, q.ctypes.data, s.ctypes.data)
    return q, s


def fp8_dequantize(q: np.ndarray, s: np.ndarray) -> np.ndarray:
    """s[i // 64] * decode(q[i]) in float64."""
    lib = _load()
    qc = np.ascontiguousarray(q, dtype=np.uint8).reshape(-1)
    sc = np.ascontiguousarray(s, dtype=np.float32).reshape(-1)
    out = np.empty(qc.size, dtype=np.float64)
    lib.orc_fp8_dequantize(qc.size, qc.ctypes.data, sc.ctypes.data, out.ctypes.data_as(_dp))
    return out
