"""Python binding of libcw.so, the sm_103a sparse-embedding (CountSketch) library.

Argument marshalling only: every step of every call runs in the library's CUDA
kernels.  Tensors must already live on the current CUDA device; the current
torch stream is passed to the library.  The functions keep the C names of
``include/cw.h`` (cw_sketch_csr, cw_solve_sketch, ...), raise ``CWError`` on a
non-zero status, and fail loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

__all__ = [
    "CWError", "lib", "load", "status_string", "device_status", "cw_csr_check",
    "cw_hash", "cw_sketch_csr", "cw_sketch_csr_rows", "cw_sketch_csr_general", "cw_sketch_dense", "cw_sketch_vec",
    "cw_gram", "cw_qr", "cw_solve_sketch", "cw_solve_sketch_dense", "cw_lsqr_precond", "cw_lsqr_precond_host", "cw_leverage",
    "cw_sketch_csr_values", "cw_sketch_dense_values", "cw_sketch_values_backward_csr",
    "cw_sketch_values_backward_dense", "SketchValues", "Batch", "EXPORTS", "HEADER",
    "cw_solve_sketched", "cw_solve_sketched_backward", "cw_normal_solve", "cw_excess_residual", "cw_scale_rows",
    "cw_scale_rows_backward", "SketchedSolve", "ScaleRows",
]

HEADER = os.path.join(_build.ROOT, "include", "cw.h")
EXPORTS = (
    "cw_status_string", "cw_version", "cw_device_status", "cw_selftest_barrier_timeout", "cw_csr_check", "cw_hash", "cw_sketch_csr",
    "cw_sketch_csr_rows", "cw_sketch_csr_general", "cw_sketch_csr_noalloc", "cw_noalloc_status", "cw_sketch_dense",
    "cw_sketch_vec", "cw_gram", "cw_qr", "cw_solve_sketch", "cw_batch_create", "cw_batch_run", "cw_batch_finish", "cw_batch_info",
    "cw_batch_phases", "cw_batch_destroy", "cw_sketch_csr_values", "cw_sketch_dense_values",
    "cw_sketch_values_backward_csr", "cw_sketch_values_backward_dense", "cw_solve_sketch_dense", "cw_lsqr_precond",
    "cw_lsqr_precond_host", "cw_leverage", "cw_launch_count", "cw_profile_enable", "cw_profile_get", "cw_profile_reset",
    "cw_solve_sketched", "cw_solve_sketched_backward", "cw_normal_solve", "cw_excess_residual", "cw_scale_rows",
    "cw_scale_rows_backward", "cw_probe_gather64",
)


class CWError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__("%s: %s" % (where, status_string(status)))


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _BatchProblem(ctypes.Structure):
    _fields_ = [("A", _CSR), ("b", ctypes.c_void_p), ("m", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("x", ctypes.c_void_p), ("SA", ctypes.c_void_p), ("Sb", ctypes.c_void_p)]


BATCH_AUTOTUNE = 1
BATCH_EAGER = 2


_lock = threading.Lock()
_lib = None
_i64, _u64, _i32, _f64, _p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
_SIGS = {
    "cw_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "cw_version": ([], ctypes.c_int),
    "cw_device_status": ([_p], ctypes.c_int),
    "cw_selftest_barrier_timeout": ([_i32, _i64, _p], ctypes.c_int),
    "cw_csr_check": ([ctypes.POINTER(_CSR), _p], ctypes.c_int),
    "cw_hash": ([_u64, _i64, _i64, _i64, _p, _p, _p], ctypes.c_int),
    "cw_sketch_csr": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_sketch_csr_rows": ([ctypes.POINTER(_CSR), _i64, _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_sketch_csr_noalloc": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_noalloc_status": ([_p], ctypes.c_int),
    "cw_sketch_csr_values": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _p, _p, _p, _p], ctypes.c_int),
    "cw_sketch_dense_values": ([_p, _i64, _i64, _i64, _p, _i64, _u64, _p, _p, _p, _p], ctypes.c_int),
    "cw_sketch_values_backward_csr": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _p, _p, _p, _p], ctypes.c_int),
    "cw_sketch_values_backward_dense": ([_p, _i64, _i64, _i64, _p, _i64, _u64, _p, _p, _p, _p], ctypes.c_int),
    "cw_batch_create": ([_p, _i32, _i32, _p, _p], ctypes.c_int),
    "cw_batch_run": ([_p, _p], ctypes.c_int),
    "cw_batch_finish": ([_p, _p, _p, _p], ctypes.c_int),
    "cw_batch_info": ([_p, _p], ctypes.c_int),
    "cw_batch_phases": ([_p, _p, _p, _i32], ctypes.c_int),
    "cw_batch_destroy": ([_p], ctypes.c_int),
    "cw_sketch_csr_general": ([ctypes.POINTER(_CSR), _p, _i64, _i64, _i32, _u64, _p, _p, _p], ctypes.c_int),
    "cw_sketch_dense": ([_p, _i64, _i64, _i64, _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_sketch_vec": ([_p, _i64, _i64, _u64, _p, _p], ctypes.c_int),
    "cw_qr": ([_p, _i64, _i64, _p, _p, _p, _p], ctypes.c_int),
    "cw_solve_sketch": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_solve_sketch_dense": ([_p, _i64, _i64, _i64, _p, _i64, _u64, _p, _p, _p], ctypes.c_int),
    "cw_lsqr_precond": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _f64, _i32, _p,
                         ctypes.POINTER(_i32), ctypes.POINTER(_f64), _p], ctypes.c_int),
    "cw_lsqr_precond_host": ([ctypes.POINTER(_CSR), _p, _i64, _u64, _f64, _i32, _p,
                              ctypes.POINTER(_i32), ctypes.POINTER(_f64), _p], ctypes.c_int),
    "cw_leverage": ([_p, _i64, _i64, _i64, _i64, _u64, _i32, _p, _p, _p], ctypes.c_int),
    "cw_gram": ([_p, _i64, _i64, _p, _p, _p], ctypes.c_int),
    "cw_solve_sketched": ([_p, _p, _i64, _i64, _p, _p, _p], ctypes.c_int),
    "cw_solve_sketched_backward": ([_p, _p, _i64, _i64, _p, _p, _p, _p, _p, _p], ctypes.c_int),
    "cw_normal_solve": ([_p, _i64, _p, _p, _p, _p], ctypes.c_int),
    "cw_excess_residual": ([_p, _i64, _p, _p, _p, _p, _p, _p], ctypes.c_int),
    "cw_scale_rows": ([_p, _p, _i64, _i64, _i64, _p, _p, _p, _p], ctypes.c_int),
    "cw_scale_rows_backward": ([_p, _p, _i64, _i64, _p, _p, _p, _p], ctypes.c_int),
    "cw_launch_count": ([], ctypes.c_longlong),
    "cw_profile_enable": ([ctypes.c_int], ctypes.c_int),
    "cw_profile_get": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_f64)], ctypes.c_int),
    "cw_profile_reset": ([], ctypes.c_int),
    "cw_probe_gather64": ([_p, _i64, _i64, ctypes.c_int, ctypes.c_int, _p, _p], ctypes.c_int),
}


def load(path=None):
    """Load libcw.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = _build.LIB
            if not _build.up_to_date():
                _build.build()
        if not os.path.exists(path):
            raise ImportError("libcw.so not found at %s; run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name, None)
            if f is None:
                continue  # reported by tests/test_abi.py
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def lib():
    return load()


def status_string(status):
    try:
        return load().cw_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - library missing
        return "status %d" % status


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _ptr_rows(A, name="A"):
    """Row-major float32 CUDA matrix, possibly a column slice (leading dimension = stride(0))."""
    if not isinstance(A, torch.Tensor) or A.dtype != torch.float32 or not A.is_cuda:
        raise TypeError("%s must be a float32 CUDA tensor" % name)
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("%s must be row-major (unit column stride)" % name)
    return ctypes.c_void_p(A.data_ptr())


def _check(st, where):
    if st != 0:
        raise CWError(st, where)


def _csr(A):
    """A: object with n, d, row_ptr, col, val (e.g. workloads.CSR on a CUDA device)."""
    c = _CSR()
    c.n, c.d = int(A.n), int(A.d)
    c.nnz = int(A.col.numel())
    c.row_ptr = _ptr(A.row_ptr, torch.int32, "row_ptr")
    c.col = _ptr(A.col, torch.int32, "col") if c.nnz else None
    c.val = _ptr(A.val, torch.float32, "val") if c.nnz else None
    return c


def device_status():
    """Synchronises the current stream; raises if a kernel flagged invalid input."""
    _check(load().cw_device_status(_stream()), "cw_device_status")


# ---------------------------------------------------------------- entry points

def cw_csr_check(A):
    """Raises CWError unless A is a valid CSR (monotone row_ptr, columns in range, distinct per row)."""
    c = _csr(A)
    _check(load().cw_csr_check(ctypes.byref(c), _stream()), "cw_csr_check")


def cw_hash(seed, m, i0, count, device=None):
    """(bucket int32, sign int8) for rows i0 .. i0+count-1."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    bucket = torch.empty(count, dtype=torch.int32, device=dev)
    sign = torch.empty(count, dtype=torch.int8, device=dev)
    _check(load().cw_hash(seed, m, i0, count, _ptr(bucket), _ptr(sign), _stream()), "cw_hash")
    return bucket, sign


def cw_sketch_csr(A, b, m, seed, SA=None, Sb=None):
    dev = A.val.device
    SA = torch.empty(m, A.d, dtype=torch.float32, device=dev) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(m, dtype=torch.float32, device=dev)
    c = _csr(A)
    _check(load().cw_sketch_csr(ctypes.byref(c), _ptr(b, torch.float32, "b"), m, seed,
                                _ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"), _stream()),
           "cw_sketch_csr")
    return SA, Sb


def cw_sketch_csr_rows(A, i0, b, m, seed, SA=None, Sb=None):
    dev = A.val.device
    SA = torch.empty(m, A.d, dtype=torch.float32, device=dev) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(m, dtype=torch.float32, device=dev)
    c = _csr(A)
    _check(load().cw_sketch_csr_rows(ctypes.byref(c), i0, _ptr(b, torch.float32, "b"), m, seed,
                                     _ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"), _stream()),
           "cw_sketch_csr_rows")
    return SA, Sb


def cw_sketch_csr_general(A, b, q, v, kappa, seed, SA=None, Sb=None):
    dev = A.val.device
    t = q * v * kappa
    SA = torch.empty(t, A.d, dtype=torch.float32, device=dev) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(t, dtype=torch.float32, device=dev)
    c = _csr(A)
    _check(load().cw_sketch_csr_general(ctypes.byref(c), _ptr(b, torch.float32, "b"), q, v, kappa, seed,
                                        _ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"),
                                        _stream()), "cw_sketch_csr_general")
    return SA, Sb


def cw_sketch_dense(A, b, m, seed, SA=None, Sb=None, lda=None):
    n, d = A.shape
    lda = A.stride(0) if lda is None else lda
    if A.stride(1) != 1:
        raise ValueError("A must be row-major")
    SA = torch.empty(m, d, dtype=torch.float32, device=A.device) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(m, dtype=torch.float32, device=A.device)
    if A.dtype != torch.float32 or not A.is_cuda:
        raise TypeError("A must be a float32 CUDA tensor")
    _check(load().cw_sketch_dense(ctypes.c_void_p(A.data_ptr()), n, d, lda, _ptr(b, torch.float32, "b"), m,
                                  seed, _ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"),
                                  _stream()), "cw_sketch_dense")
    return SA, Sb


def cw_sketch_vec(x, m, seed, Sx=None):
    Sx = torch.empty(m, dtype=torch.float32, device=x.device) if Sx is None else Sx
    _check(load().cw_sketch_vec(_ptr(x, torch.float32, "x"), x.numel(), m, seed,
                                _ptr(Sx, torch.float32, "Sx"), _stream()), "cw_sketch_vec")
    return Sx


def cw_gram(SA, Sb=None):
    """[SA | Sb]^T [SA | Sb] (float64, (d+1) x (d+1); d x d without Sb)."""
    m, d = SA.shape
    nc = d + (1 if Sb is not None else 0)
    G = torch.empty(nc, nc, dtype=torch.float64, device=SA.device)
    _check(load().cw_gram(_ptr(SA, torch.float32, "SA"), m, d, _ptr(Sb, torch.float32, "Sb"),
                          _ptr(G, torch.float64, "G"), _stream()), "cw_gram")
    return G


def cw_qr(SA, Sb=None):
    """(R float64 d x d, c float64 d or None) from the float64 Householder QR of SA."""
    m, d = SA.shape
    R = torch.empty(d, d, dtype=torch.float64, device=SA.device)
    c = torch.empty(d, dtype=torch.float64, device=SA.device) if Sb is not None else None
    _check(load().cw_qr(_ptr(SA, torch.float32, "SA"), m, d, _ptr(Sb, torch.float32, "Sb"),
                        _ptr(R, torch.float64, "R"), _ptr(c, torch.float64, "c"), _stream()), "cw_qr")
    return R, c


def cw_solve_sketch(A, b, m, seed, want_R=False):
    dev = A.val.device
    x = torch.empty(A.d, dtype=torch.float64, device=dev)
    R = torch.empty(A.d, A.d, dtype=torch.float64, device=dev) if want_R else None
    c = _csr(A)
    _check(load().cw_solve_sketch(ctypes.byref(c), _ptr(b, torch.float32, "b"), m, seed,
                                  _ptr(x, torch.float64, "x"), _ptr(R, torch.float64, "R"), _stream()),
           "cw_solve_sketch")
    return (x, R) if want_R else x


def cw_sketch_csr_values(A, b, m, seed, v, SA=None, Sb=None):
    dev = A.val.device
    SA = torch.empty(m, A.d, dtype=torch.float32, device=dev) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(m, dtype=torch.float32, device=dev)
    c = _csr(A)
    _check(load().cw_sketch_csr_values(ctypes.byref(c), _ptr(b, torch.float32, "b"), m, seed,
                                       _ptr(v, torch.float32, "v"), _ptr(SA, torch.float32, "SA"),
                                       _ptr(Sb, torch.float32, "Sb"), _stream()), "cw_sketch_csr_values")
    return SA, Sb


def cw_sketch_dense_values(A, b, m, seed, v, SA=None, Sb=None):
    n, d = A.shape
    if A.stride(1) != 1:
        raise ValueError("A must be row-major")
    SA = torch.empty(m, d, dtype=torch.float32, device=A.device) if SA is None else SA
    if b is not None and Sb is None:
        Sb = torch.empty(m, dtype=torch.float32, device=A.device)
    _check(load().cw_sketch_dense_values(_ptr_rows(A), n, d, A.stride(0),
                                         _ptr(b, torch.float32, "b"), m, seed, _ptr(v, torch.float32, "v"),
                                         _ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"),
                                         _stream()), "cw_sketch_dense_values")
    return SA, Sb


def cw_sketch_values_backward_csr(A, b, m, seed, gSA, gSb=None, gv=None):
    gv = torch.empty(A.n, dtype=torch.float32, device=A.val.device) if gv is None else gv
    c = _csr(A)
    _check(load().cw_sketch_values_backward_csr(ctypes.byref(c), _ptr(b, torch.float32, "b"), m, seed,
                                                _ptr(gSA.contiguous(), torch.float32, "gSA"),
                                                _ptr(None if gSb is None else gSb.contiguous(), torch.float32,
                                                     "gSb"),
                                                _ptr(gv, torch.float32, "gv"), _stream()),
           "cw_sketch_values_backward_csr")
    return gv


def cw_sketch_values_backward_dense(A, b, m, seed, gSA, gSb=None, gv=None):
    n, d = A.shape
    gv = torch.empty(n, dtype=torch.float32, device=A.device) if gv is None else gv
    _check(load().cw_sketch_values_backward_dense(_ptr_rows(A), n, d, A.stride(0),
                                                  _ptr(b, torch.float32, "b"), m, seed,
                                                  _ptr(gSA.contiguous(), torch.float32, "gSA"),
                                                  _ptr(None if gSb is None else gSb.contiguous(), torch.float32,
                                                       "gSb"),
                                                  _ptr(gv, torch.float32, "gv"), _stream()),
           "cw_sketch_values_backward_dense")
    return gv


class SketchValues(torch.autograd.Function):
    """(SA, Sb) = (S(v) A, S(v) b) as a differentiable function of the values v.

    ``apply(v, A, b, m, seed)``: v (n,) float32 CUDA tensor; A a CUDA CSR (n,
    d, row_ptr, col, val) or a row-major float32 CUDA tensor; b (n,) or None.
    The forward and backward are the library's kernels (cw_sketch_*_values,
    cw_sketch_values_backward_*); only v receives a gradient.
    """

    @staticmethod
    def forward(ctx, v, A, b, m, seed):
        dense = isinstance(A, torch.Tensor)
        vv = v.detach().contiguous()
        if dense:
            SA, Sb = cw_sketch_dense_values(A, b, m, seed, vv)
        else:
            SA, Sb = cw_sketch_csr_values(A, b, m, seed, vv)
        ctx.A, ctx.b, ctx.m, ctx.seed, ctx.dense = A, b, m, seed, dense
        if Sb is None:
            return SA
        return SA, Sb

    @staticmethod
    def backward(ctx, gSA, gSb=None):
        fn = cw_sketch_values_backward_dense if ctx.dense else cw_sketch_values_backward_csr
        gv = fn(ctx.A, ctx.b, ctx.m, ctx.seed, gSA.float(), None if gSb is None else gSb.float())
        return gv, None, None, None, None


def cw_solve_sketched(SA, Sb):
    """(x' float64 d, R float64 d x d): argmin ||SA x - Sb|| by the float64 Householder QR of SA."""
    m, d = SA.shape
    x = torch.empty(d, dtype=torch.float64, device=SA.device)
    R = torch.empty(d, d, dtype=torch.float64, device=SA.device)
    _check(load().cw_solve_sketched(_ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"), m, d,
                                    _ptr(x, torch.float64, "x"), _ptr(R, torch.float64, "R"), _stream()),
           "cw_solve_sketched")
    return x, R


def cw_solve_sketched_backward(SA, Sb, R, x, gx):
    """(gSA, gSb) float32: the gradients of L(x') given gx = dL/dx' (float64)."""
    m, d = SA.shape
    gSA = torch.empty(m, d, dtype=torch.float32, device=SA.device)
    gSb = torch.empty(m, dtype=torch.float32, device=SA.device)
    _check(load().cw_solve_sketched_backward(_ptr(SA, torch.float32, "SA"), _ptr(Sb, torch.float32, "Sb"), m, d,
                                             _ptr(R, torch.float64, "R"), _ptr(x, torch.float64, "x"),
                                             _ptr(gx, torch.float64, "gx"), _ptr(gSA, torch.float32, "gSA"),
                                             _ptr(gSb, torch.float32, "gSb"), _stream()),
           "cw_solve_sketched_backward")
    return gSA, gSb


def cw_normal_solve(G, want_R=False):
    """(x* float64 d, r2 float64 0-dim[, R float64 d x d]) from the bordered
    Gram [A b]^T [A b] ((d+1) x (d+1))."""
    d = G.shape[0] - 1
    x = torch.empty(d, dtype=torch.float64, device=G.device)
    r2 = torch.empty((), dtype=torch.float64, device=G.device)
    R = torch.empty(d, d, dtype=torch.float64, device=G.device) if want_R else None
    _check(load().cw_normal_solve(_ptr(G, torch.float64, "G"), d, _ptr(x, torch.float64, "x"),
                                  _ptr(r2, torch.float64, "r2"), _ptr(R, torch.float64, "R"), _stream()),
           "cw_normal_solve")
    return (x, r2, R) if want_R else (x, r2)


def cw_excess_residual(G, xstar, r2, x, want_grad=True):
    """(rho^2 - 1 float64 0-dim, its gradient in x float64 d or None)."""
    d = G.shape[0] - 1
    loss = torch.empty((), dtype=torch.float64, device=G.device)
    gx = torch.empty(d, dtype=torch.float64, device=G.device) if want_grad else None
    _check(load().cw_excess_residual(_ptr(G, torch.float64, "G"), d, _ptr(xstar, torch.float64, "xstar"),
                                     _ptr(r2, torch.float64, "r2"), _ptr(x, torch.float64, "x"),
                                     _ptr(loss, torch.float64, "loss"), _ptr(gx, torch.float64, "gx"), _stream()),
           "cw_excess_residual")
    return loss, gx


def cw_scale_rows(P, Pb, ms, w, M=None, y=None):
    """(M, y): the first ms rows of P (and Pb) scaled by w, the rest copied."""
    m, d = P.shape
    M = torch.empty_like(P) if M is None else M
    if Pb is not None and y is None:
        y = torch.empty_like(Pb)
    _check(load().cw_scale_rows(_ptr(P, torch.float32, "P"), _ptr(Pb, torch.float32, "Pb"), m, d, ms,
                                _ptr(w, torch.float32, "w"), _ptr(M, torch.float32, "M"),
                                _ptr(y, torch.float32, "y"), _stream()), "cw_scale_rows")
    return M, y


def cw_scale_rows_backward(P, Pb, ms, gM, gy):
    """gw (ms float32): gw_k = <gM_k, P_k> + gy_k Pb_k."""
    d = P.shape[1]
    gw = torch.empty(ms, dtype=torch.float32, device=P.device)
    _check(load().cw_scale_rows_backward(_ptr(P, torch.float32, "P"), _ptr(Pb, torch.float32, "Pb"), ms, d,
                                         _ptr(gM, torch.float32, "gM"), _ptr(gy, torch.float32, "gy"),
                                         _ptr(gw, torch.float32, "gw"), _stream()), "cw_scale_rows_backward")
    return gw


class SketchedSolve(torch.autograd.Function):
    """x' = argmin ||SA x - Sb|| (float64) as a differentiable function of the
    sketched system: forward cw_solve_sketched (method "qr", the Householder
    QR) or cw_gram + cw_normal_solve (method "normal", the Cholesky factor of
    [SA Sb]^T [SA Sb]: the same R and x' up to rounding, without the QR's grid
    barriers), backward cw_solve_sketched_backward (the hand-derived gradients
    of the normal equations)."""

    @staticmethod
    def forward(ctx, SA, Sb, method="qr"):
        SA, Sb = SA.detach().contiguous(), Sb.detach().contiguous()
        if method == "qr":
            x, R = cw_solve_sketched(SA, Sb)
        elif method == "normal":
            x, _, R = cw_normal_solve(cw_gram(SA, Sb), want_R=True)
        else:
            raise ValueError("method must be 'qr' or 'normal'")
        ctx.save_for_backward(SA, Sb, R, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        SA, Sb, R, x = ctx.saved_tensors
        gSA, gSb = cw_solve_sketched_backward(SA, Sb, R, x, gx.contiguous().double())
        return gSA, gSb, None


class ScaleRows(torch.autograd.Function):
    """(M, y) = the first ms rows of (P, Pb) scaled by w (values tied per
    bucket: diag(w) S A); only w receives a gradient (cw_scale_rows_backward)."""

    @staticmethod
    def forward(ctx, w, P, Pb, ms):
        M, y = cw_scale_rows(P, Pb, ms, w.detach().contiguous())
        ctx.P, ctx.Pb, ctx.ms = P, Pb, ms
        return M, y

    @staticmethod
    def backward(ctx, gM, gy):
        if gM is None:
            gM = torch.zeros_like(ctx.P)
        if gy is None and ctx.Pb is not None:
            gy = torch.zeros_like(ctx.Pb)
        gw = cw_scale_rows_backward(ctx.P, ctx.Pb, ctx.ms, gM.contiguous().float(),
                                    None if gy is None else gy.contiguous().float())
        return gw, None, None, None


class Batch:
    """A plan for many independent sketch-and-solve problems (cw_batch_*).

    problems: list of (A, b, m, seed) with A a CUDA CSR (n, d, row_ptr, col,
    val) and b a CUDA float32 vector; the tensors must stay alive and in place
    while the plan exists.  ``keep_sketch`` gives each problem its own SA / Sb
    tensors (``self.SA[p]``, ``self.Sb[p]``).  ``run()`` launches the batch;
    ``finish()`` waits and returns the per-problem status list.  ``x[p]`` is
    problem p's float64 solution.
    """

    def __init__(self, problems, autotune=False, eager=False, keep_sketch=False):
        lib = load()
        self._lib = lib
        self._plan = ctypes.c_void_p(None)
        self._keep = []
        self.x, self.SA, self.Sb = [], [], []
        arr = (_BatchProblem * len(problems))()
        for i, (A, b, m, seed) in enumerate(problems):
            dev = A.val.device
            x = torch.zeros(A.d, dtype=torch.float64, device=dev)
            self.x.append(x)
            SA = torch.empty(m, A.d, dtype=torch.float32, device=dev) if keep_sketch else None
            Sb = torch.empty(m, dtype=torch.float32, device=dev) if keep_sketch else None
            self.SA.append(SA)
            self.Sb.append(Sb)
            arr[i].A = _csr(A)
            arr[i].b = _ptr(b, torch.float32, "b")
            arr[i].m = int(m)
            arr[i].seed = int(seed)
            arr[i].x = _ptr(x, torch.float64, "x")
            arr[i].SA = _ptr(SA, torch.float32, "SA")
            arr[i].Sb = _ptr(Sb, torch.float32, "Sb")
            self._keep.append((A, b))
        flags = (BATCH_AUTOTUNE if autotune else 0) | (BATCH_EAGER if eager else 0)
        _check(lib.cw_batch_create(arr, len(problems), flags, _stream(), ctypes.byref(self._plan)),
               "cw_batch_create")
        self.count = len(problems)

    def run(self):
        _check(self._lib.cw_batch_run(self._plan, _stream()), "cw_batch_run")

    def finish(self):
        st = (ctypes.c_int32 * self.count)()
        fb = ctypes.c_int32(0)
        _check(self._lib.cw_batch_finish(self._plan, _stream(), st, ctypes.byref(fb)), "cw_batch_finish")
        return list(st)

    def info(self):
        v = (ctypes.c_int64 * 9)()
        _check(self._lib.cw_batch_info(self._plan, v), "cw_batch_info")
        keys = ("slab", "ctas_per_sm", "grid", "graph", "units", "tuned", "device_bytes", "steps", "lanes_per_row")
        return dict(zip(keys, [int(t) for t in v]))

    def phases(self):
        """Phase durations (ms) of the last completed run of the solve kernel."""
        v = (ctypes.c_double * 32)()
        k = self._lib.cw_batch_phases(self._plan, _stream(), v, 32)
        if k < 0:
            _check(k, "cw_batch_phases")
        names = ["gram", "cholesky"]
        for s in range((k - 2) // 2):
            names += ["residual_%d" % s, "correction_%d" % s]
        return dict(zip(names, [float(v[i]) for i in range(k)]))

    def close(self):
        if self._plan:
            self._lib.cw_batch_destroy(self._plan)
            self._plan = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cw_solve_sketch_dense(A, b, m, seed, want_R=False):
    n, d = A.shape
    x = torch.empty(d, dtype=torch.float64, device=A.device)
    R = torch.empty(d, d, dtype=torch.float64, device=A.device) if want_R else None
    _check(load().cw_solve_sketch_dense(_ptr(A, torch.float32, "A"), n, d, A.stride(0),
                                        _ptr(b, torch.float32, "b"), m, seed, _ptr(x, torch.float64, "x"),
                                        _ptr(R, torch.float64, "R"), _stream()), "cw_solve_sketch_dense")
    return (x, R) if want_R else x


def cw_lsqr_precond(A, b, m, seed, rtol=1e-6, max_iter=100, allow_noconv=False):
    """Returns (x float64 d, iterations, final test value)."""
    dev = A.val.device
    x = torch.empty(A.d, dtype=torch.float64, device=dev)
    it = ctypes.c_int32(0)
    ft = ctypes.c_double(0.0)
    c = _csr(A)
    st = load().cw_lsqr_precond(ctypes.byref(c), _ptr(b, torch.float32, "b"), m, seed, float(rtol), int(max_iter),
                                _ptr(x, torch.float64, "x"), ctypes.byref(it), ctypes.byref(ft), _stream())
    if not (allow_noconv and st == -6):
        _check(st, "cw_lsqr_precond")
    return x, it.value, ft.value


def _host_ptr(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) torch.Tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def cw_lsqr_precond_host(A, b, m, seed, rtol=1e-6, max_iter=100, allow_noconv=False, x=None):
    """cw_lsqr_precond for A (CSR) and b in host memory (page-locked tensors copy
    asynchronously); returns (x float64 d on the host, iterations, final test)."""
    c = _CSR()
    c.n, c.d = int(A.n), int(A.d)
    c.nnz = int(A.col.numel())
    c.row_ptr = _host_ptr(A.row_ptr, torch.int32, "row_ptr")
    c.col = _host_ptr(A.col, torch.int32, "col") if c.nnz else None
    c.val = _host_ptr(A.val, torch.float32, "val") if c.nnz else None
    if x is None:
        x = torch.empty(A.d, dtype=torch.float64)
    it = ctypes.c_int32(0)
    ft = ctypes.c_double(0.0)
    st = load().cw_lsqr_precond_host(ctypes.byref(c), _host_ptr(b, torch.float32, "b"), m, seed, float(rtol),
                                     int(max_iter), _host_ptr(x, torch.float64, "x"), ctypes.byref(it),
                                     ctypes.byref(ft), _stream())
    if not (allow_noconv and st == -6):
        _check(st, "cw_lsqr_precond_host")
    return x, it.value, ft.value


def cw_leverage(A, m, seed, G):
    """lev[i] = ||(A R^-1 G)_i||^2 / k for dense float32 A (n x d) and float64 G (d x k)."""
    n, d = A.shape
    k = G.shape[1]
    lev = torch.empty(n, dtype=torch.float32, device=A.device)
    _check(load().cw_leverage(_ptr(A, torch.float32, "A"), n, d, A.stride(0), m, seed, k,
                              _ptr(G, torch.float64, "G"), _ptr(lev, torch.float32, "lev"), _stream()),
           "cw_leverage")
    return lev


# ---------------------------------------------------------------- measurement hooks

def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(load().cw_launch_count())


def profile_enable(on=True):
    load().cw_profile_enable(1 if on else 0)


def profile_reset():
    load().cw_profile_reset()


def profile_get(kernel):
    """(launches, total milliseconds) of a named library kernel since the last reset."""
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(load().cw_profile_get(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)), "cw_profile_get")
    return int(n.value), float(ms.value)


def probe_gather64(a, nseg, sequential=False, ctas_per_sm=4, out=None):
    """One launch of the 64-byte segment read probe over the float32 device
    tensor ``a`` (a power-of-two multiple of 16 elements) on the current
    stream; time it with events on that stream (nseg * 64 bytes per launch)."""
    if a.dtype != torch.float32 or not a.is_cuda or not a.is_contiguous() or a.numel() % 16:
        raise ValueError("a: a contiguous float32 CUDA tensor of 16 * 2^k elements")
    out = torch.zeros(1, dtype=torch.float32, device=a.device) if out is None else out
    _check(load().cw_probe_gather64(_ptr(a, torch.float32, "a"), a.numel() // 16, int(nseg),
                                    1 if sequential else 0, int(ctas_per_sm), _ptr(out, torch.float32, "out"),
                                    _stream()), "cw_probe_gather64")
    return out
