"""Tiled QR factorization on NVIDIA GB300 (sm_103a) - Python binding of libtqr.

The method is the tiled QR of Bouwmeester's thesis (Chapter 3): a p x q tile matrix is
factored by the task graph of an elimination list (FlatTree, PlasmaTree(BS), BinaryTree,
Fibonacci, Greedy, GrASAP, ASAP) of GEQRT/TTQRT panel kernels and UNMQR/TTMQR updates,
run by one persistent CUDA kernel.  Every computation happens in libtqr (include/tqr.h);
this module only marshals arguments.  PyTorch provides device memory and streams.

Matrices are column-major: pass torch tensors of shape (m, n) whose stride is (1, ld)
(``colmajor(x)`` makes one).  There is no CPU fallback: the functions raise when the
CUDA library is not built or no GPU is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtqr.so")

FLAT, PLASMA, BINARY, FIBONACCI, GREEDY, GRASAP, ASAP = range(7)
TS = 16  # flag: the TS form of a tree (TSQRT/TSMQR for rows that never pivot)
TREES = {"flat": FLAT, "plasma": PLASMA, "binary": BINARY, "fibonacci": FIBONACCI,
         "greedy": GREEDY, "grasap": GRASAP, "asap": ASAP}
TREES.update({name + "-ts": v | TS for name, v in list(TREES.items())})
FP64, BF16, FP16, BF16X3, FP32, BF16X6, Z64 = 0, 1, 2, 3, 4, 5, 6
PRECS = {"fp64": FP64, "bf16": BF16, "fp16": FP16, "bf16x3": BF16X3, "fp32": FP32, "bf16x6": BF16X6, "z64": Z64}
TQR_ETIMEOUT = 3
TQR_EUNSUPPORTED = 5

_lib = None


class TqrError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str):
        super().__init__(f"{fn} failed with status {status}: {detail}")
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded libtqr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1303_3182_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        c_i64p = ctypes.POINTER(ctypes.c_int64)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "tqr_elimlist": (i32, [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_int32), c_i64p, c_i64p]),
            "tqr_schedule": (i32, [i32, i32, i32, i32, i32, c_i64p, c_i64p, c_i64p, c_i64p]),
            "tqr_set_claim_order": (i32, [i32, c_i64p]),
            "tqr_set_claim_order_ts": (i32, [i32, c_i64p]),
            "tqr_set_column_parts": (i32, [i32]),
            "tqr_set_claim_order_tc": (i32, [i32, c_i64p]),
            "tqr_schedule_ts": (i32, [i32, i32, i32, i32, i32, c_i64p, c_i64p, c_i64p, c_i64p]),
            "tqr_debug_claim_order": (i32, [i32, i32, i32, i32, i32, i32, c_i64p, ctypes.POINTER(ctypes.c_int32),
                                             c_i64p]),
            "tqr_workspace_size": (i32, [i64, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_size_t)]),
            "tqr_factor": (i32, [i64, i64, i32, i32, i32, i32, i32, vp, i64, vp, vp]),
            "tqr_apply_qt": (i32, [i64, i64, i32, i32, i32, i32, i32, i32, vp, i64, vp, vp, i64, i64, vp]),
            "tqr_trsm": (i32, [i64, i32, vp, i64, vp, i64, i64, vp]),
            "tqr_trsm_static": (i32, [i64, i32, vp, i64, vp, i64, i64, vp]),
            "tqr_lstsq": (i32, [i64, i64, i64, i32, i32, i32, i32, i32, vp, i64, vp, i64, vp, i64,
                                dbl, i32, ctypes.POINTER(ctypes.c_int), vp, ctypes.c_size_t, vp]),
            "tqr_lstsq_workspace_size": (i32, [i64, i64, i64, i32, i32, i32,
                                               ctypes.POINTER(ctypes.c_size_t)]),
            "tqr_nominal_flops": (dbl, [i64, i64]),
            "tqr_fp64_peak": (i32, [ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]),
            "tqr_set_wait_limit_ns": (i64, [i64]),
            "tqr_set_sync": (i32, [i32]),
            "tqr_sync_status": (i32, [vp]),
            "tqr_strerror": (ctypes.c_char_p, [i32]),
            "tqr_last_error": (ctypes.c_char_p, []),
            "tqr_finalize": (None, []),
            "tqr_plan_stats": (i32, [i64, i64, i32, i32, i32, c_i64p]),
            "tqr_plan_counts": (i32, [i64, i64, i32, i32, i32, c_i64p]),
            "tqr_debug_drop_edge": (None, [i64]),
            "tqr_set_timing": (i32, [i32]),
            "tqr_set_trace": (i32, [i32]),
            "tqr_launch_count": (i64, [i32]),
            "tqr_trace_fetch": (i64, [c_i64p, i64]),
            "tqr_kernel_time": (i32, [i32, ctypes.POINTER(ctypes.c_double), c_i64p, i32]),
            "tqr_batch_params": (i32, [i32, c_i64p, c_i64p, i32, c_i64p, i32,
                                       ctypes.POINTER(ctypes.c_int)]),
            "tqr_batch_workspace_size": (i32, [i32, c_i64p, c_i64p, i32, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_size_t)]),
            "tqr_batch_plan_create": (i32, [i32, c_i64p, c_i64p, ctypes.POINTER(vp), c_i64p,
                                            ctypes.POINTER(ctypes.c_int), i32, ctypes.POINTER(vp),
                                            ctypes.POINTER(vp)]),
            "tqr_batch_order": (i32, [i32, c_i64p, c_i64p, i32, ctypes.POINTER(ctypes.c_int), i32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), c_i64p]),
            "tqr_batch_plan_run": (i32, [vp, i32, vp]),
            "tqr_batch_plan_status": (i32, [vp, vp]),
            "tqr_batch_plan_info": (i32, [vp, c_i64p]),
            "tqr_batch_plan_destroy": (None, [vp]),
            "tqr_batch_autotune": (i32, [i32, c_i64p, c_i64p, i32, c_i64p, i32, ctypes.POINTER(ctypes.c_int), vp]),
            "tqr_factor_batched": (i32, [i32, c_i64p, c_i64p, ctypes.POINTER(vp), c_i64p,
                                         ctypes.POINTER(ctypes.c_int), i32, ctypes.POINTER(vp), vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn: str, status: int) -> None:
    if status != 0:
        L = lib()
        detail = L.tqr_strerror(status).decode()
        extra = L.tqr_last_error().decode()
        raise TqrError(fn, status, detail + (f" ({extra})" if extra else ""))


def _tree(tree) -> int:
    return TREES[tree] if isinstance(tree, str) else int(tree)


def _prec(prec) -> int:
    return PRECS[prec] if isinstance(prec, str) else int(prec)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ld(x, rows: int) -> int:
    """Leading dimension of a column-major (m, n) tensor view."""
    if x.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if x.shape[1] > 1 and x.stride(0) != 1:
        raise ValueError("tensor must be column-major: stride (1, ld)")
    if x.shape[1] == 1 and x.stride(0) != 1:
        raise ValueError("tensor must be column-major: stride (1, ld)")
    ld = x.stride(1) if x.shape[1] > 1 else max(rows, 1)
    return max(ld, rows)


def colmajor(x):
    """A column-major copy (stride (1, m)) of a 2-D tensor."""
    return x.t().contiguous().t()


# ---------------------------------------------------------------------------------
# Host-only entry points
# ---------------------------------------------------------------------------------

def elimlist(p: int, q: int, tree="greedy", bs: int = 1):
    """Elimination list (E x 3 int32 array of (k, i, piv), 0-based) and the critical
    path in units of nb^3/3."""
    L = lib()
    n = ctypes.c_int64(0)
    cp = ctypes.c_int64(0)
    _check("tqr_elimlist", L.tqr_elimlist(p, q, _tree(tree), bs, None, ctypes.byref(n), None))
    arr = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check("tqr_elimlist", L.tqr_elimlist(p, q, _tree(tree), bs,
                                          arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          ctypes.byref(n), ctypes.byref(cp)))
    return arr[:n.value], cp.value


def _weights4(weights):
    if weights is None:
        return None
    w = (ctypes.c_int64 * len(weights))(*[int(x) for x in weights])
    return ctypes.cast(w, ctypes.POINTER(ctypes.c_int64))


def schedule(p: int, q: int, tree="greedy", bs: int = 1, nproc: int = 1, weights=None):
    """Bounded-processor schedule of the factorization task graph on nproc processors:
    (CP-method makespan, ALAP Derived bound, lost area); weights are four kernel weights
    (GEQRT, TTQRT, UNMQR, TTMQR; None = 4, 2, 6, 6; TS kernels 3 x TTQRT, 2 x TTMQR), six
    (..., TSQRT, TSMQR), seven (..., operand-image preparation: the tensor-core graph) or
    nine (..., TTQRT block, TSQRT block: the tensor-core graph with split panels)."""
    ms, bound, la = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    if weights is not None and len(weights) in (6, 7, 9):
        weights = list(weights) + [0] * (9 - len(weights))
        fn, name = lib().tqr_schedule_ts, "tqr_schedule_ts"
    else:
        fn, name = lib().tqr_schedule, "tqr_schedule"
    _check(name, fn(p, q, _tree(tree), bs, nproc, _weights4(weights), ctypes.byref(ms), ctypes.byref(bound),
                    ctypes.byref(la)))
    return ms.value, bound.value, la.value


def set_claim_order(mode: int, weights=None) -> None:
    """Executor claim order of later factorization plans: 0 = earliest start on unbounded
    processors, 1 = start order of the bounded-processor CP-method schedule with the given
    kernel weights (GEQRT, TTQRT, UNMQR, TTMQR[, TSQRT, TSMQR[, preparation, TTQRT block,
    TSQRT block]]), 2 = the default (1 with
    built-in GB300 weights for the tensor-core precisions and fp64, 0 for fp32)."""
    if weights is not None and len(weights) == 9:
        _check("tqr_set_claim_order_tc", lib().tqr_set_claim_order_tc(mode, _weights4(weights)))
    elif weights is not None and len(weights) == 6:
        _check("tqr_set_claim_order_ts", lib().tqr_set_claim_order_ts(mode, _weights4(weights)))
    else:
        _check("tqr_set_claim_order", lib().tqr_set_claim_order(mode, _weights4(weights)))


def set_column_parts(mode: int) -> None:
    """Column parts of later fp64 / fp32 factorization plans (tqr_set_column_parts): 0 =
    never, 1 = automatic (small graphs bound by their critical path), 2 = always."""
    _check("tqr_set_column_parts", lib().tqr_set_column_parts(mode))


def claim_order(p: int, q: int, tree="greedy", bs: int = 1, mode: int = 0, nproc: int = 1, weights=None):
    """The executor's claim order of a p x q factorization task graph (test hook): an
    (ntask, 5) int32 array of (kind, i, piv, k, j) rows in claim order."""
    L = lib()
    n = ctypes.c_int64(0)
    _check("tqr_debug_claim_order", L.tqr_debug_claim_order(p, q, _tree(tree), bs, mode, nproc, _weights4(weights),
                                                            None, ctypes.byref(n)))
    arr = np.zeros((max(n.value, 1), 5), dtype=np.int32)
    _check("tqr_debug_claim_order", L.tqr_debug_claim_order(p, q, _tree(tree), bs, mode, nproc, _weights4(weights),
                                                            arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                            ctypes.byref(n)))
    return arr[:n.value]


def plan_stats(m: int, n: int, nb: int, tree="greedy", bs: int = 1):
    out = (ctypes.c_int64 * 6)()
    _check("tqr_plan_stats", lib().tqr_plan_stats(m, n, nb, _tree(tree), bs, out))
    return {"GEQRT": out[0], "TTQRT": out[1], "UNMQR": out[2], "TTMQR": out[3],
            "edges": out[4], "cp": out[5]}


def plan_counts(m: int, n: int, nb: int, tree="greedy", bs: int = 1):
    """Task counts of a factorization graph including the TS kernels (tree may be a TS
    form, e.g. "plasma-ts")."""
    out = (ctypes.c_int64 * 8)()
    _check("tqr_plan_counts", lib().tqr_plan_counts(m, n, nb, _tree(tree), bs, out))
    return {"GEQRT": out[0], "TTQRT": out[1], "UNMQR": out[2], "TTMQR": out[3],
            "TSQRT": out[4], "TSMQR": out[5], "edges": out[6], "cp": out[7]}


def workspace_size(m: int, n: int, nb: int, ib: int, prec="fp64") -> int:
    out = ctypes.c_size_t(0)
    _check("tqr_workspace_size", lib().tqr_workspace_size(m, n, nb, ib, _prec(prec), ctypes.byref(out)))
    return out.value


def nominal_flops(m: int, n: int) -> float:
    return lib().tqr_nominal_flops(m, n)


def fp64_peak(stream=None):
    """Measured FP64 TFLOP/s of the current GPU: {"dfma": ..., "dmma": ...}."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check("tqr_fp64_peak", lib().tqr_fp64_peak(ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return {"dfma": a.value, "dmma": b.value}


def set_wait_limit_ns(ns: int) -> int:
    return lib().tqr_set_wait_limit_ns(ns)


def set_sync(on: bool) -> bool:
    """Synchronize and check the device status inside every call (default on)."""
    return bool(lib().tqr_set_sync(1 if on else 0))


def set_timing(on: bool) -> bool:
    """Bracket every library kernel launch with CUDA events (see tqr_set_timing)."""
    return bool(lib().tqr_set_timing(1 if on else 0))


KERNEL_KINDS = {"factor": 0, "apply_q": 1, "trsm": 2, "refine": 3}


def kernel_time(kind, reset: bool = True):
    """(total device ms, launches) accumulated for one kernel kind since the last reset."""
    ms = ctypes.c_double(0)
    n = ctypes.c_int64(0)
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check("tqr_kernel_time", lib().tqr_kernel_time(k, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
    return ms.value, n.value


def launch_count(reset: bool = False) -> int:
    """Kernels launched by the library so far (tqr_launch_count)."""
    return int(lib().tqr_launch_count(1 if reset else 0))


def set_trace(on: bool) -> bool:
    """Record per-task globaltimer stamps in every executor launch (tqr_set_trace)."""
    return bool(lib().tqr_set_trace(1 if on else 0))


def trace_fetch():
    """The last traced launch as an (ntask, 12) int64 array: kind, i, piv, k | j << 16,
    claim, start, end (ns), sm, and four phase durations (ns)."""
    L = lib()
    n = L.tqr_trace_fetch(None, 0)
    out = np.zeros((max(n, 1), 12), dtype=np.int64)
    got = L.tqr_trace_fetch(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n)
    if got < 0:
        raise TqrError("tqr_trace_fetch", int(-got), "no trace")
    return out[:got]


def debug_drop_edge(e: int) -> None:
    lib().tqr_debug_drop_edge(e)


def finalize() -> None:
    lib().tqr_finalize()


# ---------------------------------------------------------------------------------
# Device entry points (torch tensors on a CUDA device)
# ---------------------------------------------------------------------------------

def _dtype_of(prec):
    import torch
    p = _prec(prec)
    return torch.complex128 if p == Z64 else (torch.float64 if p == FP64 else torch.float32)


def factor(A, nb: int, ib: int, tree="greedy", bs: int = 1, prec="fp64", T=None, stream=None):
    """Tiled QR of A in place (column-major CUDA tensor: float64 for fp64, complex128 for
    z64, float32 otherwise).  Returns the T workspace tensor (bytes)."""
    import torch
    m, n = A.shape
    if A.dtype != _dtype_of(prec) or not A.is_cuda:
        raise ValueError("A must be a CUDA tensor of the precision's storage type")
    lda = _ld(A, m)
    if T is None:
        T = torch.empty(workspace_size(m, n, nb, ib, prec), dtype=torch.uint8, device=A.device)
    _check("tqr_factor", lib().tqr_factor(m, n, nb, ib, _tree(tree), bs, _prec(prec),
                                          ctypes.c_void_p(A.data_ptr()), lda,
                                          ctypes.c_void_p(T.data_ptr()), _stream(stream)))
    return T


def apply_qt(A, T, B, nb: int, ib: int, tree="greedy", bs: int = 1, prec="fp64",
             trans: int = 0, stream=None):
    """B <- Q^T B (trans=0; Q^H for z64) or Q B (trans=1) in place; B is a float64
    (complex128 for z64) column-major tensor with A's row count."""
    import torch
    m, n = A.shape
    want = torch.complex128 if _prec(prec) == Z64 else torch.float64
    if B.dtype != want or B.shape[0] != m:
        raise ValueError("B must be float64 (complex128 for z64) with m rows")
    _check("tqr_apply_qt", lib().tqr_apply_qt(m, n, nb, ib, _tree(tree), bs, _prec(prec), trans,
                                              ctypes.c_void_p(A.data_ptr()), _ld(A, m),
                                              ctypes.c_void_p(T.data_ptr()),
                                              ctypes.c_void_p(B.data_ptr()), _ld(B, m),
                                              B.shape[1], _stream(stream)))
    return B


def trsm(A, B, n: int, prec="fp64", stream=None):
    """Solve R X = B in place (R: the n x n upper triangle of factored A)."""
    _check("tqr_trsm", lib().tqr_trsm(n, _prec(prec), ctypes.c_void_p(A.data_ptr()), _ld(A, A.shape[0]),
                                      ctypes.c_void_p(B.data_ptr()), _ld(B, B.shape[0]), B.shape[1],
                                      _stream(stream)))
    return B


def trsm_static(A, B, n: int, prec="fp64", stream=None):
    """tqr_trsm_static: the same solve as trsm() without any device allocation (scratch in
    a fixed array inside the library; n <= 262144; calls must not overlap on the GPU)."""
    _check("tqr_trsm_static", lib().tqr_trsm_static(n, _prec(prec), ctypes.c_void_p(A.data_ptr()),
                                                    _ld(A, A.shape[0]), ctypes.c_void_p(B.data_ptr()),
                                                    _ld(B, B.shape[0]), B.shape[1], _stream(stream)))
    return B


def lstsq_workspace_size(m, n, nrhs, nb, ib, prec="fp64") -> int:
    out = ctypes.c_size_t(0)
    _check("tqr_lstsq_workspace_size",
           lib().tqr_lstsq_workspace_size(m, n, nrhs, nb, ib, _prec(prec), ctypes.byref(out)))
    return out.value


def lstsq(A, B, nb: int, ib: int, tree="greedy", bs: int = 1, prec="fp64", tol: float = 1e-14,
          max_iter: int = 100, X=None, workspace=None, stream=None, return_iters: bool = False):
    """Least-squares solution X of min ||A X - B|| (float64 column-major CUDA tensors;
    complex128 for z64)."""
    import torch
    m, n = A.shape
    nrhs = B.shape[1]
    if X is None:
        dt = torch.complex128 if _prec(prec) == Z64 else torch.float64
        X = colmajor(torch.empty((n, nrhs), dtype=dt, device=A.device))
    if workspace is None:
        workspace = torch.empty(lstsq_workspace_size(m, n, nrhs, nb, ib, prec), dtype=torch.uint8,
                                device=A.device)
    iters = ctypes.c_int(0)
    _check("tqr_lstsq", lib().tqr_lstsq(m, n, nrhs, nb, ib, _tree(tree), bs, _prec(prec),
                                        ctypes.c_void_p(A.data_ptr()), _ld(A, m),
                                        ctypes.c_void_p(B.data_ptr()), _ld(B, m),
                                        ctypes.c_void_p(X.data_ptr()), _ld(X, n), tol, max_iter,
                                        ctypes.byref(iters), ctypes.c_void_p(workspace.data_ptr()),
                                        workspace.numel(), _stream(stream)))
    return (X, iters.value) if return_iters else X


# ---------------------------------------------------------------------------------
# Batched factorization (many independent matrices, one persistent launch)
# ---------------------------------------------------------------------------------

def _i64(a):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def batch_autotune(ms, ns, prec="fp32", stream=None):
    """tqr_batch_autotune: the library's per-size-class tuning table of a batch, an
    (nclasses, 8) int64 array of rows (m_lo, m_hi, n_lo, n_hi, nb, ib, tree, bs), tuned by
    device timing on first use and cached in the library."""
    m, mp = _i64(ms)
    n, np_ = _i64(ns)
    rows = ctypes.c_int(0)
    L = lib()
    _check("tqr_batch_autotune", L.tqr_batch_autotune(len(m), mp, np_, _prec(prec), None, 0, ctypes.byref(rows),
                                                      _stream(stream)))
    table = np.zeros((max(rows.value, 1), 8), dtype=np.int64)
    _check("tqr_batch_autotune", L.tqr_batch_autotune(len(m), mp, np_, _prec(prec),
                                                      table.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                      rows.value, ctypes.byref(rows), _stream(stream)))
    return table[:rows.value]


def batch_params(ms, ns, prec="fp32", table=None):
    """(nbatch, 4) int32 array of per-matrix (nb, ib, tree, bs): the first row of
    ``table`` (rows m_lo, m_hi, n_lo, n_hi, nb, ib, tree, bs) covering each matrix, else
    the library's built-in size classes; table="auto" takes batch_autotune's table."""
    if isinstance(table, str) and table == "auto":
        table = batch_autotune(ms, ns, prec)
    m, mp = _i64(ms)
    n, np_ = _i64(ns)
    out = np.zeros((len(m), 4), dtype=np.int32)
    if table is not None and len(table):
        t, tp = _i64(np.asarray(table, dtype=np.int64).reshape(-1, 8))
        nrows = t.shape[0]
    else:
        t, tp, nrows = None, None, 0
    _check("tqr_batch_params", lib().tqr_batch_params(len(m), mp, np_, _prec(prec), tp, nrows,
                                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return out


def batch_workspace_offsets(ms, ns, prec="fp32", params=None):
    """Byte offsets (nbatch + 1) of the per-matrix T workspaces in one buffer."""
    m, mp = _i64(ms)
    n, np_ = _i64(ns)
    off = np.zeros(len(m) + 1, dtype=np.uint64)
    pp = None
    if params is not None:
        params = np.ascontiguousarray(np.asarray(params, dtype=np.int32))
        pp = params.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check("tqr_batch_workspace_size",
           lib().tqr_batch_workspace_size(len(m), mp, np_, _prec(prec), pp,
                                          off.ctypes.data_as(ctypes.POINTER(ctypes.c_size_t))))
    return off.astype(np.int64)


def batch_order(ms, ns, prec="fp32", params=None, slots: int = 152):
    """Merged claim order of a batch (host only): arrays (matrix, local task index)."""
    m, mp = _i64(ms)
    n, np_ = _i64(ns)
    pp = None
    if params is not None:
        params = np.ascontiguousarray(np.asarray(params, dtype=np.int32))
        pp = params.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cnt = ctypes.c_int64(0)
    L = lib()
    _check("tqr_batch_order", L.tqr_batch_order(len(m), mp, np_, _prec(prec), pp, slots, None, None,
                                                ctypes.byref(cnt)))
    mat = np.zeros(max(cnt.value, 1), dtype=np.int32)
    loc = np.zeros(max(cnt.value, 1), dtype=np.int32)
    _check("tqr_batch_order", L.tqr_batch_order(len(m), mp, np_, _prec(prec), pp, slots,
                                                mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                loc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                ctypes.byref(cnt)))
    return mat[:cnt.value], loc[:cnt.value]


class BatchPlan:
    """tqr_batch_plan: the merged task graph of a batch, bound to its A and T buffers.
    ``As`` is a list of column-major CUDA tensors; ``T`` one uint8 CUDA buffer carved at
    ``batch_workspace_offsets``.  Keep both alive while the plan is used."""

    def __init__(self, As, prec="fp32", params=None, T=None):
        import torch
        self.prec = _prec(prec)
        dt = _dtype_of(prec)
        ms = [int(a.shape[0]) for a in As]
        ns = [int(a.shape[1]) for a in As]
        for a in As:
            if a.dtype != dt or not a.is_cuda:
                raise ValueError("every matrix must be a CUDA tensor of the precision's storage type")
        self.params = batch_params(ms, ns, prec) if params is None else \
            np.ascontiguousarray(np.asarray(params, dtype=np.int32).reshape(-1, 4))
        off = batch_workspace_offsets(ms, ns, prec, self.params)
        if T is None:
            T = torch.empty(int(off[-1]), dtype=torch.uint8, device=As[0].device)
        self.T, self.As = T, list(As)
        base = T.data_ptr()
        self._m, mp = _i64(ms)
        self._n, np_ = _i64(ns)
        self._lda, lp = _i64([_ld(a, r) for a, r in zip(As, ms)])
        VP = ctypes.c_void_p * len(As)
        self._A = VP(*[a.data_ptr() for a in As])
        self._T = VP(*[base + int(o) for o in off[:-1]])
        h = ctypes.c_void_p(0)
        _check("tqr_batch_plan_create",
               lib().tqr_batch_plan_create(len(As), mp, np_, self._A, lp,
                                           self.params.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                           self.prec, self._T, ctypes.byref(h)))
        self._h = h

    def run(self, use_graph: bool = False, stream=None):
        _check("tqr_batch_plan_run", lib().tqr_batch_plan_run(self._h, 1 if use_graph else 0, _stream(stream)))

    def status(self, stream=None):
        """Wait for the stream; raise if the last run's device status is an error."""
        _check("tqr_batch_plan_status", lib().tqr_batch_plan_status(self._h, _stream(stream)))

    def info(self):
        out = (ctypes.c_int64 * 6)()
        _check("tqr_batch_plan_info", lib().tqr_batch_plan_info(self._h, out))
        return {"tasks": out[0], "edges": out[1], "matrices": out[2], "slots": out[3],
                "graph": bool(out[4]), "flops": float(out[5])}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tqr_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor_batched(As, prec="fp32", params=None, T=None, stream=None):
    """One-shot batched factorization (tqr_factor_batched) of a list of column-major CUDA
    tensors in place.  params None: the library's autotuned settings (NULL through the
    C ABI; T is sized from the same cached tuning table).  Returns (T buffer, byte
    offsets, params)."""
    import torch
    ms = [int(a.shape[0]) for a in As]
    ns = [int(a.shape[1]) for a in As]
    auto = params is None
    params = batch_params(ms, ns, prec, "auto") if auto else \
        np.ascontiguousarray(np.asarray(params, dtype=np.int32).reshape(-1, 4))
    off = batch_workspace_offsets(ms, ns, prec, params)
    if T is None:
        T = torch.empty(int(off[-1]), dtype=torch.uint8, device=As[0].device)
    m, mp = _i64(ms)
    n, np_ = _i64(ns)
    lda, lp = _i64([_ld(a, r) for a, r in zip(As, ms)])
    VP = ctypes.c_void_p * len(As)
    Ap = VP(*[a.data_ptr() for a in As])
    Tp = VP(*[T.data_ptr() + int(o) for o in off[:-1]])
    _check("tqr_factor_batched",
           lib().tqr_factor_batched(len(As), mp, np_, Ap, lp,
                                    None if auto else params.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    _prec(prec), Tp, _stream(stream)))
    return T, off, params
