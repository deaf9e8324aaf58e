"""Python binding of the GB300 dense Tucker / HOOI library (include/tucker.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libtucker_gb300.so.  There is no CPU fallback; if the library is
not built the import of any entry point raises.

Tensors are torch tensors on the current CUDA device, contiguous; factor
matrices are (L_n, K_n) row-major with the factor dtype (float64 for FP64
tensors, float32 otherwise); bf16 tensors are passed as torch.bfloat16.
Every call is asynchronous on torch's current stream (or `stream=`).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
# TUCKER_LIB_VARIANT=debug loads the debug build (index-checked kernels, see
# build.build(debug=True) and tucker_debug_check)
DEBUG_VARIANT = os.environ.get("TUCKER_LIB_VARIANT", "") == "debug"
LIB_PATH = os.path.join(_HERE, "libtucker_gb300_debug.so" if DEBUG_VARIANT else "libtucker_gb300.so")

TUCKER_F32, TUCKER_F64, TUCKER_BF16, TUCKER_FP8_E4M3, TUCKER_BF16_SPLIT = 0, 1, 2, 3, 4
TREE_OPTIMAL, TREE_CHAIN, TREE_CHAIN_K, TREE_CHAIN_H, TREE_BALANCED = 0, 1, 2, 3, 4
COST_MACS, COST_ELEMS = 0, 1
PLAN_NO_FUSED_ROOT = 1
PLAN_STHOSVD_ORDER = 2
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "WORKSPACE", -4: "CUDA", -5: "TIMEOUT",
          -6: "NONFINITE", -7: "INCOMPLETE"}
TUCKER_ERR_INCOMPLETE = -7

_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vpp = ctypes.POINTER(ctypes.c_void_p)


class TuckerError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class PlanOpts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("tree", ctypes.c_int32),
                ("cost_model", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("ws_cap", ctypes.c_uint64)]


class Node(ctypes.Structure):
    _fields_ = [("label", ctypes.c_int32), ("parent", ctypes.c_int32),
                ("in_elems", ctypes.c_uint64), ("out_elems", ctypes.c_uint64),
                ("macs", ctypes.c_uint64), ("ws_offset", ctypes.c_uint64)]


class ProfRec(ctypes.Structure):
    _fields_ = [("node", ctypes.c_int32), ("label", ctypes.c_int32), ("ms", ctypes.c_float)]


def lib():
    """Load libtucker_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1707_05594_gb300.build.build("
                          f"{'debug=True' if DEBUG_VARIANT else ''})")
    L = ctypes.CDLL(LIB_PATH)
    L.tucker_plan.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.POINTER(PlanOpts),
                              ctypes.POINTER(ctypes.c_void_p)]
    L.tucker_plan_cost.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p,
                                   ctypes.POINTER(ctypes.c_size_t)]
    L.tucker_plan_fused_root.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]
    L.tucker_plan_sthosvd.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), _u64p]
    L.tucker_plan_nodes.argtypes = [ctypes.c_void_p, ctypes.POINTER(Node), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
    L.tucker_plan_destroy.argtypes = [ctypes.c_void_p]
    L.tucker_plan_destroy.restype = None
    L.tucker_sthosvd.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _vpp, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.tucker_hooi_sweep.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _vpp, _vpp,
                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.tucker_core.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _vpp, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.tucker_hooi_sweep_core.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _vpp, _vpp,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]
    L.tucker_hooi_sweep_gs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _vpp, _vpp, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.tucker_norm2.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.tucker_fit.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p]
    L.tucker_ttm.argtypes = [ctypes.c_int, _i64p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L.tucker_ttm_pair.argtypes = [ctypes.c_int, _i64p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_void_p]
    L.tucker_gram.argtypes = [ctypes.c_int, _i64p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_void_p]
    L.tucker_eig_topk.argtypes = [ctypes.c_int, _i64p, _i64p, _vpp, _vpp, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.tucker_convert_bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p]
    L.tucker_set_kernel_policy.argtypes = [ctypes.c_int]
    L.tucker_fp8_bytes.argtypes = [ctypes.c_int64]
    L.tucker_fp8_bytes.restype = ctypes.c_size_t
    L.tucker_convert_fp8.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p]
    L.tucker_bf16_split_bytes.argtypes = [ctypes.c_int64]
    L.tucker_bf16_split_bytes.restype = ctypes.c_size_t
    L.tucker_bf16_split_lo_offset.argtypes = [ctypes.c_int64]
    L.tucker_bf16_split_lo_offset.restype = ctypes.c_size_t
    L.tucker_device_status.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.tucker_debug_build.argtypes = []
    L.tucker_debug_check.argtypes = [_i64p, _i64p, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p,
                                     ctypes.c_int, ctypes.c_int]
    L.tucker_selftest_wait_timeout.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    L.tucker_check_finite.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    L.tucker_eig_topk_noalloc.argtypes = [ctypes.c_int, _i64p, _i64p, _vpp, _vpp, ctypes.c_int,
                                          ctypes.c_void_p]
    L.tucker_eig_ws_bytes.argtypes = [ctypes.c_int, _i64p, _i64p]
    L.tucker_eig_ws_bytes.restype = ctypes.c_size_t
    L.tucker_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.tucker_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(ProfRec), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]
    L.tucker_launch_count.restype = ctypes.c_uint64
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    L.tucker_batch_plan.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, _i64p, ctypes.POINTER(vp)]
    L.tucker_batch_info.argtypes = [vp, ctypes.POINTER(sz), _i64p, _i64p, _i64p]
    L.tucker_batch_offsets.argtypes = [vp, _i64p, _i64p, _i64p]
    L.tucker_batch_destroy.argtypes = [vp]
    L.tucker_batch_destroy.restype = None
    L.tucker_batch_prepare.argtypes = [vp, vp, sz, vp]
    L.tucker_batch_sthosvd.argtypes = [vp, vp, vp, vp, vp, sz, vp]
    L.tucker_batch_sweep.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
    L.tucker_batch_norm2.argtypes = [vp, vp, vp, vp, sz, vp]
    L.tucker_batch_fit.argtypes = [vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.tucker_batch_sweep_fused.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.tucker_batch_set_fused.argtypes = [vp, ctypes.c_int]
    L.tucker_batch_queue_offset.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.tucker_batch_graph_create.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, sz, ctypes.POINTER(vp)]
    L.tucker_batch_graph_launch.argtypes = [vp, vp, vp]
    L.tucker_batch_graph_destroy.argtypes = [vp]
    L.tucker_batch_graph_destroy.restype = None
    L.tucker_batch_autotune.argtypes = [vp, vp, vp, vp, vp, sz, ctypes.c_int, vp]
    L.tucker_batch_tuning.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    L.tucker_batch_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.tucker_last_error.restype = ctypes.c_char_p
    L.tucker_version.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != 0:
        msg = lib().tucker_last_error().decode(errors="replace")
        raise TuckerError(rc, where, msg)


def _i64(a: Sequence[int]):
    return (ctypes.c_int64 * len(a))(*[int(x) for x in a])


def _ptrs(ts):
    for t in ts:
        _req(t, "tensor")
    return (ctypes.c_void_p * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


def _dp(t, name):
    """Device pointer of a contiguous CUDA tensor (the ABI takes dense row-major
    buffers; a strided view would be read as if it were dense)."""
    _req(t, name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if isinstance(t, Fp8Tensor):
        return TUCKER_FP8_E4M3
    if isinstance(t, Bf16SplitTensor):
        return TUCKER_BF16_SPLIT
    if t.dtype == torch.float32:
        return TUCKER_F32
    if t.dtype == torch.float64:
        return TUCKER_F64
    if t.dtype == torch.bfloat16:
        return TUCKER_BF16
    raise TypeError(f"unsupported tensor dtype {t.dtype}")


def factor_torch_dtype(code: int):
    import torch
    return torch.float64 if code == TUCKER_F64 else torch.float32


def _req(t, name):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


@dataclass
class Plan:
    """Owns a tucker_plan_t (library-owned TTM-tree + workspace layout)."""
    handle: ctypes.c_void_p
    L: tuple
    K: tuple
    dtype: int
    tree: int

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.tucker_plan_destroy(self.handle)
            self.handle = None

    @property
    def N(self):
        return len(self.L)

    @property
    def factor_dtype(self):
        return factor_torch_dtype(self.dtype)


def tucker_plan(L: Sequence[int], K: Sequence[int], dtype: int = TUCKER_F32,
                tree: int = TREE_OPTIMAL, cost_model: int = COST_MACS,
                fuse_root: bool = True, sthosvd_order: bool = False, ws_cap: int = 0) -> Plan:
    """ws_cap: workspace cap in bytes (0: none); the plan gives up the fused
    root, then the STHOSVD order, to meet it (see include/tucker.h)."""
    h = ctypes.c_void_p()
    flags = (0 if fuse_root else PLAN_NO_FUSED_ROOT) | (PLAN_STHOSVD_ORDER if sthosvd_order else 0)
    opts = PlanOpts(dtype, tree, cost_model, flags, int(ws_cap))
    _check(lib().tucker_plan(len(L), _i64(L), _i64(K), ctypes.byref(opts), ctypes.byref(h)),
           "tucker_plan")
    return Plan(h, tuple(int(x) for x in L), tuple(int(x) for x in K), dtype, tree)


def tucker_plan_fused_root(plan: Plan):
    """(first, second) node indices of the fused root children, or None."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().tucker_plan_fused_root(plan.handle, ctypes.byref(a), ctypes.byref(b)),
           "tucker_plan_fused_root")
    return None if a.value < 0 else (a.value, b.value)


def tucker_plan_sthosvd(plan: Plan):
    """(mode order of tucker_sthosvd, its cost under the plan's cost model)."""
    order = (ctypes.c_int * plan.N)()
    cost = ctypes.c_uint64()
    _check(lib().tucker_plan_sthosvd(plan.handle, order, ctypes.byref(cost)), "tucker_plan_sthosvd")
    return list(order), cost.value


def tucker_plan_cost(plan: Plan):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    w = ctypes.c_size_t()
    _check(lib().tucker_plan_cost(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                  ctypes.byref(w)), "tucker_plan_cost")
    return {"tree_macs": a.value, "tree_elems": b.value, "core_macs": c.value,
            "ws_bytes": w.value}


def tucker_plan_nodes(plan: Plan) -> List[dict]:
    n = ctypes.c_int()
    _check(lib().tucker_plan_nodes(plan.handle, None, 0, ctypes.byref(n)), "tucker_plan_nodes")
    arr = (Node * n.value)()
    _check(lib().tucker_plan_nodes(plan.handle, arr, n.value, ctypes.byref(n)),
           "tucker_plan_nodes")
    return [{"label": x.label, "parent": x.parent, "in_elems": x.in_elems,
             "out_elems": x.out_elems, "macs": x.macs, "ws_offset": x.ws_offset} for x in arr]


def workspace(plan: Plan, device=None):
    """Allocates a workspace of the plan's size (a torch uint8 buffer)."""
    import torch
    nb = tucker_plan_cost(plan)["ws_bytes"]
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device or "cuda")


def tucker_sthosvd(plan: Plan, T, F: Sequence, G, ws, stream=None):
    _req(T, "T")
    _check(lib().tucker_sthosvd(plan.handle, _dp(T, "T"), _ptrs(F),
                                _dp(G, "G"), _dp(ws, "ws"),
                                ws.numel(), _stream(stream)), "tucker_sthosvd")


def tucker_hooi_sweep(plan: Plan, T, F_in: Sequence, F_out: Sequence, ws, stream=None):
    _req(T, "T")
    _check(lib().tucker_hooi_sweep(plan.handle, _dp(T, "T"), _ptrs(F_in),
                                   _ptrs(F_out), _dp(ws, "ws"), ws.numel(),
                                   _stream(stream)), "tucker_hooi_sweep")


def tucker_hooi_sweep_gs(plan: Plan, T, F_in: Sequence, F_out: Sequence, G_out, ws, stream=None):
    """HOOI sweep in the Gauss-Seidel form (each mode uses the factors already
    updated in this sweep); G_out (or None) receives the core of F_out."""
    _req(T, "T")
    _check(lib().tucker_hooi_sweep_gs(plan.handle, _dp(T, "T"), _ptrs(F_in), _ptrs(F_out),
                                      _dp(G_out, "G_out") if G_out is not None else None,
                                      _dp(ws, "ws"), ws.numel(), _stream(stream)),
           "tucker_hooi_sweep_gs")


def tucker_hooi_sweep_core(plan: Plan, T, F_in: Sequence, F_out: Sequence, G_in, ws, stream=None):
    """HOOI sweep that also returns the core of its INPUT factors (from the tree)."""
    _req(T, "T")
    _check(lib().tucker_hooi_sweep_core(plan.handle, _dp(T, "T"), _ptrs(F_in),
                                        _ptrs(F_out),
                                        _dp(G_in, "G_in") if G_in is not None else None,
                                        _dp(ws, "ws"), ws.numel(), _stream(stream)),
           "tucker_hooi_sweep_core")


def tucker_core(plan: Plan, T, F: Sequence, G, ws, stream=None):
    _check(lib().tucker_core(plan.handle, _dp(T, "T"), _ptrs(F),
                             _dp(G, "G"), _dp(ws, "ws"),
                             ws.numel(), _stream(stream)), "tucker_core")


def tucker_norm2(plan: Plan, T, out, stream=None):
    _check(lib().tucker_norm2(plan.handle, _dp(T, "T"),
                              _dp(out, "out"), _stream(stream)), "tucker_norm2")


def tucker_fit(plan: Plan, G, normT2, out, stream=None):
    _check(lib().tucker_fit(plan.handle, _dp(G, "G"),
                            _dp(normT2, "normT2"), _dp(out, "out"),
                            _stream(stream)), "tucker_fit")


def tucker_ttm(X, n: int, F, Y, stream=None):
    _req(X, "X")
    _check(lib().tucker_ttm(X.dim(), _i64(X.shape), _dp(X, "X"),
                            _dtype_code(X), n, _dp(F, "F"), F.shape[1],
                            _dp(Y, "Y"), _stream(stream)), "tucker_ttm")


def tucker_ttm_pair(X, a: int, Fa, Ya, b: int, Fb, Yb, stream=None):
    """Ya = X x_a Fa^T and Yb = X x_b Fb^T (a < b) from one read of X (the
    fused root kernel); Ya / Yb FP32, or BF16 for a BF16 X."""
    _req(X, "X")
    _check(lib().tucker_ttm_pair(X.dim(), _i64(X.shape), _dp(X, "X"), _dtype_code(X), a,
                                 _dp(Fa, "Fa"), Fa.shape[1], b, _dp(Fb, "Fb"), Fb.shape[1],
                                 _dp(Ya, "Ya"), _dp(Yb, "Yb"), _dtype_code(Ya), _stream(stream)),
           "tucker_ttm_pair")


def tucker_gram(Z, n: int, W, stream=None):
    _req(Z, "Z")
    _check(lib().tucker_gram(Z.dim(), _i64(Z.shape), _dp(Z, "Z"),
                             _dtype_code(Z), n, _dp(W, "W"), _stream(stream)),
           "tucker_gram")


def tucker_eig_ws_bytes(Ls: Sequence[int], Ks: Sequence[int]) -> int:
    return int(lib().tucker_eig_ws_bytes(len(Ls), _i64(Ls), _i64(Ks)))


def _eig_args(Ws: Sequence, Fs: Sequence):
    """(L list, K list, factor dtype code) of an eigensolver call, after the
    checks the C entry points cannot make on raw pointers: one output per
    matrix, every W a float64 (L, L) matrix, every F an (L, K) matrix and all
    F of one type, float32 or float64."""
    import torch
    if len(Ws) == 0 or len(Ws) != len(Fs):
        raise ValueError("need one output factor per matrix")
    fdt = Fs[0].dtype
    if fdt not in (torch.float32, torch.float64):
        raise TypeError(f"factors must be float32 or float64, not {fdt}")
    Ls, Ks = [], []
    for W, F in zip(Ws, Fs):
        if W.dtype != torch.float64 or W.dim() != 2 or W.shape[0] != W.shape[1]:
            raise TypeError("every W must be a square float64 matrix")
        if F.dtype != fdt:
            raise TypeError("all factors must have the same dtype")
        if F.dim() != 2 or F.shape[0] != W.shape[0]:
            raise ValueError("every F must be an (L, K) matrix with L = W.shape[0]")
        Ls.append(int(W.shape[0]))
        Ks.append(int(F.shape[1]))
    return Ls, Ks, (TUCKER_F64 if fdt == torch.float64 else TUCKER_F32)


def tucker_eig_topk(Ws: Sequence, Fs: Sequence, ws, stream=None):
    Ls, Ks, fcode = _eig_args(Ws, Fs)
    _check(lib().tucker_eig_topk(len(Ws), _i64(Ls), _i64(Ks), _ptrs(Ws), _ptrs(Fs),
                                 fcode, _dp(ws, "ws"), ws.numel(),
                                 _stream(stream)), "tucker_eig_topk")


def tucker_eig_topk_noalloc(Ws: Sequence, Fs: Sequence, stream=None):
    """Leading eigenvectors without any device allocation or workspace: for
    callers that must not allocate (see include/tucker.h).  Uses a fixed
    scratch array inside the library shared by all calls."""
    Ls, Ks, fcode = _eig_args(Ws, Fs)
    _check(lib().tucker_eig_topk_noalloc(len(Ws), _i64(Ls), _i64(Ks), _ptrs(Ws), _ptrs(Fs),
                                         fcode, _stream(stream)),
           "tucker_eig_topk_noalloc")


def tucker_convert_bf16(x, hi, lo=None, stream=None):
    """hi = bf16(x) (round to nearest even), lo = bf16(x - hi) when given."""
    _req(x, "x")
    _check(lib().tucker_convert_bf16(ctypes.c_void_p(x.data_ptr()), _dp(hi, "hi"),
                                     _dp(lo, "lo") if lo is not None else None,
                                     x.numel(), _stream(stream)), "tucker_convert_bf16")


class Fp8Tensor:
    """A tensor stored as FP8 E4M3 codes with one float scale per 64 elements
    (the layout of tucker_fp8_bytes) in a uint8 CUDA buffer.  Passed wherever
    a plan of type TUCKER_FP8_E4M3 takes T."""

    def __init__(self, buf, shape):
        self.buf = buf
        self.shape = tuple(int(x) for x in shape)
        self.is_cuda = buf.is_cuda
        self.device = buf.device

    def data_ptr(self):
        return self.buf.data_ptr()

    def is_contiguous(self):
        return True

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for x in self.shape:
            n *= x
        return n

    def codes(self):
        return self.buf[:self.numel()]

    def scales(self):
        import torch
        n = self.numel()
        off = (n + 255) // 256 * 256
        return self.buf[off:off + 4 * ((n + 63) // 64)].view(torch.float32)


def tucker_fp8_bytes(n: int) -> int:
    return int(lib().tucker_fp8_bytes(int(n)))


def tucker_convert_fp8(x, stream=None) -> Fp8Tensor:
    """FP8 E4M3 copy of the float32 CUDA tensor x with per-64 scales."""
    import torch
    _req(x, "x")
    if x.dtype != torch.float32:
        raise TypeError("tucker_convert_fp8 takes a float32 tensor")
    buf = torch.empty(max(256, tucker_fp8_bytes(x.numel())), dtype=torch.uint8, device=x.device)
    _check(lib().tucker_convert_fp8(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                    x.numel(), _stream(stream)), "tucker_convert_fp8")
    return Fp8Tensor(buf, x.shape)


class Bf16SplitTensor:
    """An FP32 tensor held as two BF16 tensors hi = bf16(x), lo = bf16(x - hi)
    in one uint8 CUDA buffer (the layout of tucker_bf16_split_bytes: hi, then
    lo from tucker_bf16_split_lo_offset).  Passed wherever a plan of type
    TUCKER_BF16_SPLIT takes T."""

    def __init__(self, buf, shape):
        self.buf = buf
        self.shape = tuple(int(x) for x in shape)
        self.is_cuda = buf.is_cuda
        self.device = buf.device

    def data_ptr(self):
        return self.buf.data_ptr()

    def is_contiguous(self):
        return True

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for x in self.shape:
            n *= x
        return n

    def hi(self):
        import torch
        return self.buf[:2 * self.numel()].view(torch.bfloat16).view(self.shape)

    def lo(self):
        import torch
        off = int(lib().tucker_bf16_split_lo_offset(self.numel()))
        return self.buf[off:off + 2 * self.numel()].view(torch.bfloat16).view(self.shape)


def tucker_bf16_split(x, stream=None) -> Bf16SplitTensor:
    """Split BF16 copy (hi + lo) of the float32 CUDA tensor x."""
    import torch
    _req(x, "x")
    if x.dtype != torch.float32:
        raise TypeError("tucker_bf16_split takes a float32 tensor")
    n = x.numel()
    buf = torch.empty(max(256, int(lib().tucker_bf16_split_bytes(n))), dtype=torch.uint8, device=x.device)
    off = int(lib().tucker_bf16_split_lo_offset(n))
    _check(lib().tucker_convert_bf16(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                     ctypes.c_void_p(buf.data_ptr() + off), n, _stream(stream)),
           "tucker_bf16_split")
    return Bf16SplitTensor(buf, x.shape)


def tucker_set_kernel_policy(policy: int) -> None:
    _check(lib().tucker_set_kernel_policy(int(policy)), "tucker_set_kernel_policy")


def tucker_device_status(reset: bool = True) -> int:
    st = ctypes.c_int(0)
    _check(lib().tucker_device_status(ctypes.byref(st), 1 if reset else 0), "tucker_device_status")
    return st.value


def tucker_debug_build() -> bool:
    """True when the loaded library is the index-checked debug build."""
    return bool(lib().tucker_debug_build())


def tucker_debug_check(reset: bool = True) -> dict:
    """Out-of-range index ranges recorded by the debug build's kernels since
    the last reset: {"count", "index", "bound", "line", "file"} (count 0 in
    the normal build).  Synchronous."""
    idx, bnd = ctypes.c_int64(0), ctypes.c_int64(0)
    line = ctypes.c_int(0)
    buf = ctypes.create_string_buffer(256)
    n = lib().tucker_debug_check(ctypes.byref(idx), ctypes.byref(bnd), ctypes.byref(line), buf, 256,
                                 1 if reset else 0)
    if n < 0:
        _check(n, "tucker_debug_check")
    return {"count": n, "index": idx.value, "bound": bnd.value, "line": line.value,
            "file": os.path.basename(buf.value.decode())}


def tucker_check_finite(X, stream=None) -> None:
    """Raises TuckerError (NONFINITE) when X holds a NaN or an Inf."""
    _check(lib().tucker_check_finite(_dp(X, "X"), _dtype_code(X), X.numel(), _stream(stream)),
           "tucker_check_finite")


def tucker_selftest_wait_timeout(stream=None) -> int:
    """Runs the bounded-wait self-test (a wait that nothing completes gives up
    after its limit); returns 2 when the wait gave up, 1 if it completed."""
    out = ctypes.c_int(0)
    _check(lib().tucker_selftest_wait_timeout(ctypes.byref(out), _stream(stream)),
           "tucker_selftest_wait_timeout")
    return out.value


def tucker_profile_enable(plan: Plan, capacity: int) -> None:
    _check(lib().tucker_profile_enable(plan.handle, int(capacity)), "tucker_profile_enable")


def tucker_profile_read(plan: Plan, capacity: int) -> List[tuple]:
    """[(node, label, ms), ...] in recording order (at most `capacity`);
    waits for the events and empties the ring."""
    arr = (ProfRec * max(1, capacity))()
    n = ctypes.c_int()
    _check(lib().tucker_profile_read(plan.handle, arr, capacity, ctypes.byref(n)),
           "tucker_profile_read")
    return [(arr[i].node, arr[i].label, arr[i].ms) for i in range(min(n.value, capacity))]


def tucker_launch_count() -> int:
    return int(lib().tucker_launch_count())


def tucker_last_error() -> str:
    return lib().tucker_last_error().decode(errors="replace")


def tucker_version() -> int:
    return lib().tucker_version()


# ---------------------------------------------------------------- helpers ---
class Decomposition:
    """Convenience driver over the C ABI: holds T, the plan, workspace, factors,
    core and the cached ||T||^2 on one device.  Every step calls the library."""

    def __init__(self, T, K: Sequence[int], tree: int = TREE_OPTIMAL,
                 cost_model: int = COST_MACS, sthosvd_order: bool = False):
        import torch
        self.T = T
        self.code = _dtype_code(T)
        self.plan = tucker_plan(T.shape, K, self.code, tree, cost_model, sthosvd_order=sthosvd_order)
        self.ws = workspace(self.plan, T.device)
        fdt = self.plan.factor_dtype
        L = T.shape
        self.F = [torch.empty(L[n], K[n], dtype=fdt, device=T.device) for n in range(len(L))]
        self.F_next = [torch.empty_like(f) for f in self.F]
        self.G = torch.empty(*K, dtype=fdt, device=T.device)
        self.normT2 = torch.empty(1, dtype=torch.float64, device=T.device)
        self.fit_out = torch.empty(2, dtype=torch.float64, device=T.device)
        tucker_norm2(self.plan, T, self.normT2)

    def sthosvd(self):
        tucker_sthosvd(self.plan, self.T, self.F, self.G, self.ws)
        tucker_fit(self.plan, self.G, self.normT2, self.fit_out)

    def sweep(self, with_core: bool = True):
        """One HOOI sweep; then the new core of the new factors and the fit."""
        tucker_hooi_sweep(self.plan, self.T, self.F, self.F_next, self.ws)
        self.F, self.F_next = self.F_next, self.F
        if with_core:
            tucker_core(self.plan, self.T, self.F, self.G, self.ws)
            tucker_fit(self.plan, self.G, self.normT2, self.fit_out)

    def sweep_fused(self):
        """One HOOI sweep whose tree also yields the core (and fit) of the
        factors it starts from: after this call G and fit() describe the
        previous factors, F holds the new ones."""
        tucker_hooi_sweep_core(self.plan, self.T, self.F, self.F_next, self.G, self.ws)
        tucker_fit(self.plan, self.G, self.normT2, self.fit_out)
        self.F, self.F_next = self.F_next, self.F

    def fit(self) -> float:
        return float(self.fit_out[0].item())

    def state_dict(self) -> dict:
        """Checkpoint: the HOOI state is the factors (and the core of the last
        step); copied to host memory."""
        return {"L": tuple(self.T.shape), "K": tuple(self.G.shape),
                "F": [f.detach().cpu().clone() for f in self.F],
                "G": self.G.detach().cpu().clone()}

    def load_state_dict(self, sd: dict) -> None:
        """Resume from state_dict(): same lengths and ranks required."""
        if tuple(sd["L"]) != tuple(self.T.shape) or tuple(sd["K"]) != tuple(self.G.shape):
            raise ValueError("checkpoint of a different shape")
        for f, s in zip(self.F, sd["F"]):
            f.copy_(s)
        self.G.copy_(sd["G"])


# ---------------------------------------------------------- batched form ---
def _vp(t):
    return _dp(t, "tensor") if t is not None else None


class BatchPlan:
    """Owns a tucker_batch_t: `count` FP32 tensors of order N with their own
    lengths dims[i][n] and core lengths ranks[i][n], packed back to back."""

    def __init__(self, dims: Sequence[Sequence[int]], ranks: Sequence[Sequence[int]]):
        self.count = len(dims)
        self.N = len(dims[0]) if self.count else 0
        flat_d = [int(x) for d in dims for x in d]
        flat_r = [int(x) for r in ranks for x in r]
        if len(flat_d) != self.count * self.N or len(flat_r) != self.count * self.N:
            raise ValueError("dims and ranks need count x N entries")
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.ranks = [tuple(int(x) for x in r) for r in ranks]
        h = ctypes.c_void_p()
        _check(lib().tucker_batch_plan(self.count, self.N, _i64(flat_d), _i64(flat_r),
                                       ctypes.byref(h)), "tucker_batch_plan")
        self.handle = h
        ws = ctypes.c_size_t()
        te, fe, ge = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tucker_batch_info(h, ctypes.byref(ws), ctypes.byref(te), ctypes.byref(fe),
                                       ctypes.byref(ge)), "tucker_batch_info")
        self.ws_bytes, self.t_elems, self.f_elems, self.g_elems = ws.value, te.value, fe.value, ge.value
        t_off = (ctypes.c_int64 * self.count)()
        f_off = (ctypes.c_int64 * (self.count * self.N))()
        g_off = (ctypes.c_int64 * self.count)()
        _check(lib().tucker_batch_offsets(h, t_off, f_off, g_off), "tucker_batch_offsets")
        self.t_off, self.f_off, self.g_off = list(t_off), list(f_off), list(g_off)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tucker_batch_destroy(self.handle)

    # views of the packed buffers
    def tensor(self, T, i: int):
        n = 1
        for x in self.dims[i]:
            n *= x
        return T[self.t_off[i]:self.t_off[i] + n].view(*self.dims[i])

    def factor(self, F, i: int, n: int):
        o = self.f_off[i * self.N + n]
        L, K = self.dims[i][n], self.ranks[i][n]
        return F[o:o + L * K].view(L, K)

    def core(self, G, i: int):
        n = 1
        for x in self.ranks[i]:
            n *= x
        return G[self.g_off[i]:self.g_off[i] + n].view(*self.ranks[i])


def tucker_batch_prepare(b: BatchPlan, ws, stream=None):
    _check(lib().tucker_batch_prepare(b.handle, _vp(ws), ws.numel() * ws.element_size(),
                                      _stream(stream)), "tucker_batch_prepare")


def tucker_batch_sthosvd(b: BatchPlan, T, F, G, ws, stream=None):
    _check(lib().tucker_batch_sthosvd(b.handle, _vp(T), _vp(F), _vp(G), _vp(ws),
                                      ws.numel() * ws.element_size(), _stream(stream)),
           "tucker_batch_sthosvd")


def tucker_batch_sweep(b: BatchPlan, T, F_in, F_out, G_in, ws, stream=None):
    _check(lib().tucker_batch_sweep(b.handle, _vp(T), _vp(F_in), _vp(F_out), _vp(G_in), _vp(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)),
           "tucker_batch_sweep")


def tucker_batch_sweep_fused(b: BatchPlan, T, F_in, F_out, G_in, normT2, fit, ws, stream=None):
    """tucker_batch_sweep + tucker_batch_fit of (F_in, G_in) as one
    persistent launch (plus the gated full eigensolver path)."""
    _check(lib().tucker_batch_sweep_fused(b.handle, _vp(T), _vp(F_in), _vp(F_out), _vp(G_in), _vp(normT2),
                                          _vp(fit), _vp(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "tucker_batch_sweep_fused")


def tucker_batch_queue_offset(b: BatchPlan) -> int:
    off = ctypes.c_size_t(0)
    _check(lib().tucker_batch_queue_offset(b.handle, ctypes.byref(off)), "tucker_batch_queue_offset")
    return off.value


def tucker_batch_set_fused(b: BatchPlan, on: bool):
    _check(lib().tucker_batch_set_fused(b.handle, 1 if on else 0), "tucker_batch_set_fused")


def tucker_batch_norm2(b: BatchPlan, T, normT2, ws, stream=None):
    _check(lib().tucker_batch_norm2(b.handle, _vp(T), _vp(normT2), _vp(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)),
           "tucker_batch_norm2")


def tucker_batch_fit(b: BatchPlan, T, F, G, normT2, fit, ws, stream=None):
    """fit[i] = 1 - ||T_i - G_i x F_i|| / ||T_i|| from the residual itself."""
    _check(lib().tucker_batch_fit(b.handle, _vp(T), _vp(F), _vp(G), _vp(normT2), _vp(fit),
                                  _vp(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "tucker_batch_fit")


def tucker_batch_autotune(b: BatchPlan, T, F, G, ws, reps: int = 5, stream=None):
    """Times every candidate launch configuration of each sweep site on these
    buffers and keeps the fastest (synchronous; overwrites G with the core of
    F).  Graphs recorded earlier must be created again."""
    _check(lib().tucker_batch_autotune(b.handle, _vp(T), _vp(F), _vp(G), _vp(ws),
                                       ws.numel() * ws.element_size(), int(reps), _stream(stream)),
           "tucker_batch_autotune")


_SITE_KIND = {0: "level", 1: "core", 2: "fit"}


def tucker_batch_tuning(b: BatchPlan):
    """The launch configuration of every sweep site: a list of dicts with the
    site (kind, index), its positions per thread, staging row length and node
    order, and the default's and the chosen configuration's ms per launch from
    the last autotune (-1 before one)."""
    n = ctypes.c_int()
    _check(lib().tucker_batch_tuning(b.handle, 0, ctypes.byref(n), None, None), "tucker_batch_tuning")
    cfg = (ctypes.c_int * (6 * n.value))()
    ms = (ctypes.c_float * (2 * n.value))()
    _check(lib().tucker_batch_tuning(b.handle, n.value, ctypes.byref(n), cfg, ms), "tucker_batch_tuning")
    out = []
    for i in range(n.value):
        c = cfg[6 * i:6 * i + 6]
        out.append({"site": _SITE_KIND[c[0]], "index": c[1], "ppt": c[2], "stage_c": c[3],
                    "order": c[4], "async": c[5], "ms_default": ms[2 * i], "ms_tuned": ms[2 * i + 1]})
    return out


def tucker_batch_set_tuning(b: BatchPlan, sites):
    """Sets every site's configuration from tucker_batch_tuning's list (the
    dicts' site, index, ppt, stage_c, order, async); prepare the batch again after."""
    kind = {v: k for k, v in _SITE_KIND.items()}
    flat = []
    for s in sites:
        flat += [kind[s["site"]], s["index"], s["ppt"], s["stage_c"], s["order"], s.get("async", 0)]
    arr = (ctypes.c_int * len(flat))(*flat)
    _check(lib().tucker_batch_set_tuning(b.handle, len(sites), arr), "tucker_batch_set_tuning")


class BatchGraph:
    """An executable CUDA graph of one batched sweep (tucker_batch_graph_*)."""

    def __init__(self, b: BatchPlan, T, F_in, F_out, G_in, normT2, fit, ws):
        self.b = b
        self._keep = (T, F_in, F_out, G_in, normT2, fit, ws)
        h = ctypes.c_void_p()
        _check(lib().tucker_batch_graph_create(b.handle, _vp(T), _vp(F_in), _vp(F_out), _vp(G_in),
                                               _vp(normT2), _vp(fit), _vp(ws),
                                               ws.numel() * ws.element_size(), ctypes.byref(h)),
               "tucker_batch_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().tucker_batch_graph_launch(self.b.handle, self.handle, _stream(stream)),
               "tucker_batch_graph_launch")

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tucker_batch_graph_destroy(self.handle)


class BatchDecomposition:
    """Batched driver: STHOSVD, then sweeps that alternate between two factor
    buffers (through two recorded graphs, A -> B and B -> A, or direct calls).
    After each sweep G and fit describe the factors the sweep started from;
    factors() is the newest factor buffer."""

    # Below this many tensors per SM the per-site launches are taken before
    # autotune() times both forms: the fused sweep's CTAs need several tensors
    # each to hide their latency (measured on GB300: per-site faster with 1024
    # tensors, fused faster with 4096).
    FUSED_MIN_TENSORS_PER_SM = 16

    def __init__(self, T, dims, ranks, fused=None):
        import torch
        self.T = T
        self.b = BatchPlan(dims, ranks)
        # fused: each sweep (and its fit) is one persistent launch
        # (tucker_batch_sweep_fused); else the per-site launches; None: by
        # the batch's size until autotune() times both
        if fused is None:
            sms = torch.cuda.get_device_properties(T.device).multi_processor_count
            fused = self.b.count >= self.FUSED_MIN_TENSORS_PER_SM * sms
        self.fused = bool(fused)
        tucker_batch_set_fused(self.b, self.fused)
        self.form_ms = None  # ms per sweep of each form, from the last autotune()
        if T.numel() != self.b.t_elems or T.dtype != torch.float32:
            raise ValueError("T must hold the packed FP32 tensors of the batch")
        dev = T.device
        self.ws = torch.empty(self.b.ws_bytes, dtype=torch.uint8, device=dev)
        tucker_batch_prepare(self.b, self.ws)
        self.Fbuf = [torch.empty(self.b.f_elems, dtype=torch.float32, device=dev) for _ in range(2)]
        self.cur = 0
        self.G = torch.empty(self.b.g_elems, dtype=torch.float32, device=dev)
        self.normT2 = torch.empty(self.b.count, dtype=torch.float64, device=dev)
        self.fit_out = torch.empty(self.b.count, dtype=torch.float64, device=dev)
        tucker_batch_norm2(self.b, T, self.normT2, self.ws)
        self._graphs = None

    def sthosvd(self):
        tucker_batch_sthosvd(self.b, self.T, self.Fbuf[self.cur], self.G, self.ws)
        tucker_batch_fit(self.b, self.T, self.Fbuf[self.cur], self.G, self.normT2, self.fit_out,
                         self.ws)

    def set_fused(self, on: bool):
        """Sweeps by the fused persistent launch (True) or the per-site
        launches (False); recorded graphs are dropped."""
        self.fused = bool(on)
        tucker_batch_set_fused(self.b, self.fused)
        self._graphs = None

    def autotune(self, reps: int = 5):
        """Tunes the batch's launch configurations on the current factors
        (tucker_batch_autotune), then times `reps` graph sweeps of each form
        (per-site with the tuned configurations, and fused) from the current
        factors and keeps the faster (form_ms holds both times).  The factors
        are restored afterwards; G and fit are overwritten.  Both forms give
        the same factors and cores."""
        import torch
        self._graphs = None
        tucker_batch_autotune(self.b, self.T, self.Fbuf[self.cur], self.G, self.ws, reps)
        F0, cur0 = self.Fbuf[self.cur].clone(), self.cur
        ms = {}
        for on in (False, True):
            self.set_fused(on)
            self.sweep(graph=True)  # records the graphs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(max(1, reps)):
                self.sweep(graph=True)
            e1.record()
            torch.cuda.synchronize()
            ms["fused" if on else "per_site"] = e0.elapsed_time(e1) / max(1, reps)
            self.cur = cur0
            self.Fbuf[cur0].copy_(F0)
        self.form_ms = ms
        self.set_fused(ms["fused"] < ms["per_site"])
        return tucker_batch_tuning(self.b)

    def sweep(self, graph: bool = True):
        src, dst = self.Fbuf[self.cur], self.Fbuf[1 - self.cur]
        if graph:
            if self._graphs is None:
                A, B = self.Fbuf
                self._graphs = (
                    BatchGraph(self.b, self.T, A, B, self.G, self.normT2, self.fit_out, self.ws),
                    BatchGraph(self.b, self.T, B, A, self.G, self.normT2, self.fit_out, self.ws))
            self._graphs[self.cur].launch()
        elif self.fused:
            tucker_batch_sweep_fused(self.b, self.T, src, dst, self.G, self.normT2, self.fit_out, self.ws)
        else:
            tucker_batch_sweep(self.b, self.T, src, dst, self.G, self.ws)
            tucker_batch_fit(self.b, self.T, src, self.G, self.normT2, self.fit_out, self.ws)
        self.cur ^= 1

    def factors(self):
        return self.Fbuf[self.cur]
