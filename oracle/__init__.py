"""CPU oracle for the CountSketch hot path of Clarkson & Woodruff (arXiv 1207.6365).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
float64 restatement of what the GPU library computes.  Only the tests, the
smoke check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the GPU path (its own C core, its own
loader, its own hash implementation).

Contents, each following the paper passage named in its docstring:

* ``hash`` / ``coeffs`` / ``poly_values``: the seeded map (h, sigma) that
  defines S = Phi D (Section 2).  C core with 128-bit arithmetic; a second,
  arbitrary-precision version lives in ``oracle.hash_bigint``.
* ``sketch_csr`` / ``sketch_dense`` / ``sketch_vec``: SA and Sb by the plain
  loop over rows in ascending order, float64 sums (Section 2; Theorem "lin reg"
  sketches A and b with the same S).
* ``sketch_csr_general`` / ``dense_S_general`` / ``general_seeds``: the
  generalized sparse embedding (Section "Generalized Sparse Embedding
  Matrices": blockdiag(B^(1..q)) P with kappa stacked sketches per block), as a
  row loop in C and as the explicit matrix built block by block.
* ``sketch_*_values`` / ``sketch_values_backward_*`` / ``dense_S_values``:
  the sketch with values v_i at the hash positions (S(v)[h(i), i] = v_i) and
  the gradient of a loss with respect to v, gv_i = <dL/dSA[h(i)], A_i> +
  dL/dSb[h(i)] b_i (SA and Sb are linear in v).
* ``qr_r`` / ``solve_sketch``: Householder QR of SA (LAPACK through numpy), R
  normalised to a positive diagonal, then x' = R^-1 Q^T Sb (proof of Theorem
  "renRegAlg": "a QR factorization of SA and then computing R^-1 Q^T SB").
* ``lsqr_precond``: LSQR (Paige and Saunders, 1982) on y -> A R^-1 y, the
  CG-like method preconditioned by R of Section 7.6 ("Iterative Methods for
  Regression").
* ``leverage_same``: u'_i = ||(A R^-1 G)_i||^2 / k (Theorem "icml", Section 6,
  with Pi_2 = G / sqrt(k)); ``leverage_exact``: ||Q_i||^2 of a float64 QR of A.
* ``lstsq_exact_*`` / ``residual_ratio``: exact least squares by Householder
  QR of [A | b] (row-block streaming) and ||Ax'-b|| / ||Ax*-b||.

Numerical pins for all of these are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.linalg as sla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "libcw_oracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def build(force=False):
    """Compile the C core with gcc into oracle/_build (host code only)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIBPATH)
             or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIBPATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-fopenmp", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_coeffs.argtypes = [_u64, _p]
            lib.orc_poly_values.argtypes = [_u64, _i64, _i64, _p, _p]
            lib.orc_hash.argtypes = [_u64, _i64, _i64, _i64, _p, _p]
            lib.orc_sketch_csr.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _u64, _i64, _p, _p]
            lib.orc_sketch_csr_parallel.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _u64, _i64, ctypes.c_int,
                                                    _p, _p]
            lib.orc_sketch_dense.argtypes = [_i64, _i64, _i64, _p, _p, _i64, _u64, _i64, _p, _p]
            lib.orc_seeds_after_coeffs.argtypes = [_u64, _i64, _p]
            lib.orc_sketch_csr_values.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _u64, _p, _p, _p]
            lib.orc_sketch_values_backward_csr.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _u64, _p, _p, _p]
            lib.orc_sketch_csr_general.argtypes = [_i64, _i64, _p, _p, _p, _p, _i64, _i64, _i64, _u64, _p, _p]
            lib.orc_csr_matvec.argtypes = [_i64, _p, _p, _p, _p, _p]
            lib.orc_csr_rmatvec.argtypes = [_i64, _i64, _p, _p, _p, _p, _p]
            for f in (lib.orc_coeffs, lib.orc_poly_values, lib.orc_hash, lib.orc_sketch_csr,
                      lib.orc_seeds_after_coeffs, lib.orc_sketch_csr_general, lib.orc_sketch_csr_values,
                      lib.orc_sketch_values_backward_csr,
                      lib.orc_sketch_dense, lib.orc_csr_matvec, lib.orc_csr_rmatvec):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _np(a, dtype):
    """Host numpy array (accepts numpy arrays and CPU/GPU torch tensors)."""
    if a is None:
        return None
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- the map h, sigma

def coeffs(seed):
    """The 8 polynomial coefficients (bucket c0..c3, sign c0..c3) for ``seed``."""
    out = np.zeros(8, dtype=np.uint64)
    _load().orc_coeffs(_u64(seed), _ptr(out))
    return [int(v) for v in out]


def poly_values(seed, i0, count):
    """Raw g_bucket(i), g_sign(i) (mod 2^61-1) for i in [i0, i0+count)."""
    gb = np.zeros(count, dtype=np.uint64)
    gs = np.zeros(count, dtype=np.uint64)
    _load().orc_poly_values(_u64(seed), _i64(i0), _i64(count), _ptr(gb), _ptr(gs))
    return gb, gs


def hash(seed, m, i0, count):  # noqa: A001 - the paper's h
    """(bucket int32, sign int8) for rows i0 .. i0+count-1 (Section 2 map h, D)."""
    bucket = np.zeros(count, dtype=np.int32)
    sign = np.zeros(count, dtype=np.int8)
    _load().orc_hash(_u64(seed), _i64(m), _i64(i0), _i64(count), _ptr(bucket), _ptr(sign))
    return bucket, sign


def dense_S(seed, m, n, i0=0):
    """The explicit m x n matrix S = Phi D (only for tiny n): S[h(i), i] = sigma(i)."""
    h, s = hash(seed, m, i0, n)
    S = np.zeros((m, n))
    S[h, np.arange(n)] = s
    return S


# ---------------------------------------------------------------- SA, Sb

def sketch_csr(row_ptr, col, val, d, b, m, seed, i0=0):
    """(SA float64 m x d, Sb float64 m or None) by the plain row loop (Section 2)."""
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    n = row_ptr.shape[0] - 1
    SA = np.zeros((m, d))
    Sb = np.zeros(m) if b is not None else None
    _load().orc_sketch_csr(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b),
                           _i64(m), _u64(seed), _i64(i0), _ptr(SA), _ptr(Sb))
    return SA, Sb


def sketch_csr_parallel(row_ptr, col, val, d, b, m, seed, i0=0, threads=0):
    """The same (SA, Sb) as sketch_csr on all host cores (threads <= 0: all):
    rows sorted by bucket, buckets summed in parallel in ascending row order,
    so the sums and their order equal the plain loop's (bitwise identical)."""
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    n = row_ptr.shape[0] - 1
    SA = np.zeros((m, d))
    Sb = np.zeros(m) if b is not None else None
    _load().orc_sketch_csr_parallel(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _i64(m),
                                    _u64(seed), _i64(i0), ctypes.c_int(int(threads)), _ptr(SA), _ptr(Sb))
    return SA, Sb


def sketch_dense(A, b, m, seed, i0=0):
    """(SA, Sb) for dense row-major float32 A (Section 2)."""
    A = _np(A, np.float32)
    b = _np(b, np.float32)
    n, d = A.shape
    SA = np.zeros((m, d))
    Sb = np.zeros(m) if b is not None else None
    _load().orc_sketch_dense(_i64(n), _i64(d), _i64(d), _ptr(A), _ptr(b), _i64(m), _u64(seed),
                             _i64(i0), _ptr(SA), _ptr(Sb))
    return SA, Sb


def sketch_vec(x, m, seed, i0=0):
    """Sx for a float32 vector x (the d = 1 case)."""
    x = _np(x, np.float32)
    SA, _ = sketch_dense(x.reshape(-1, 1), None, m, seed, i0)
    return SA[:, 0]


# ---------------------------------------------------------------- sketch values and their gradient

def dense_S_values(seed, m, n, v):
    """The explicit m x n matrix S(v): S[h(i), i] = v_i (tiny n only)."""
    h, _ = hash(seed, m, 0, n)
    S = np.zeros((m, n))
    S[h, np.arange(n)] = _np(v, np.float64)
    return S


def sketch_csr_values(row_ptr, col, val, d, b, m, seed, v):
    """(SA(v), Sb(v)) in float64: SA[h(i)] += v_i A_i (row loop, C core)."""
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    v = _np(v, np.float32)
    n = row_ptr.shape[0] - 1
    SA = np.zeros((m, d))
    Sb = np.zeros(m) if b is not None else None
    _load().orc_sketch_csr_values(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _i64(m),
                                  _u64(seed), _ptr(v), _ptr(SA), _ptr(Sb))
    return SA, Sb


def sketch_values_backward_csr(row_ptr, col, val, d, b, m, seed, gSA, gSb=None):
    """gv_i = <gSA[h(i)], A_i> + gSb[h(i)] b_i in float64 (C core)."""
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    gSA = np.ascontiguousarray(gSA, dtype=np.float64)
    gSb = None if gSb is None else np.ascontiguousarray(gSb, dtype=np.float64)
    n = row_ptr.shape[0] - 1
    gv = np.zeros(n)
    _load().orc_sketch_values_backward_csr(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b),
                                           _i64(m), _u64(seed), _ptr(gSA), _ptr(gSb), _ptr(gv))
    return gv


def sketch_dense_values(A, b, m, seed, v):
    """(SA(v), Sb(v)) for dense A in float64 (scatter-add by bucket, numpy)."""
    A = _np(A, np.float32).astype(np.float64)
    v = _np(v, np.float32).astype(np.float64)
    h, _ = hash(seed, m, 0, A.shape[0])
    SA = np.zeros((m, A.shape[1]))
    np.add.at(SA, h, v[:, None] * A)
    Sb = None
    if b is not None:
        Sb = np.zeros(m)
        np.add.at(Sb, h, v * _np(b, np.float32).astype(np.float64))
    return SA, Sb


def sketch_values_backward_dense(A, b, m, seed, gSA, gSb=None):
    """gv_i = <gSA[h(i)], A_i> + gSb[h(i)] b_i for dense A in float64 (numpy)."""
    A = _np(A, np.float32).astype(np.float64)
    h, _ = hash(seed, m, 0, A.shape[0])
    gv = (np.asarray(gSA, dtype=np.float64)[h] * A).sum(axis=1)
    if gSb is not None and b is not None:
        gv += np.asarray(gSb, dtype=np.float64)[h] * _np(b, np.float32).astype(np.float64)
    return gv


# ---------------------------------------------------------------- generalized sparse embedding

def general_seeds(seed, kappa):
    """Seeds of the kappa inner sketches: the raw SplitMix64 outputs that follow
    the eight accepted coefficient draws of ``seed``."""
    out = np.zeros(kappa, dtype=np.uint64)
    _load().orc_seeds_after_coeffs(_u64(seed), _i64(kappa), _ptr(out))
    return [int(x) for x in out]


def dense_S_general(seed, q, v, kappa, n):
    """The explicit t x n generalized sparse embedding (t = q v kappa), built as
    the paper writes it (Section "Generalized Sparse Embedding Matrices", "The
    construction"): a permutation P that lists the rows of block 1, then block
    2, ... (h = the bucket map of ``seed`` over q buckets, rows in ascending
    order within a block), times the block-diagonal matrix of B^(1..q), where
    B^(i) stacks kappa sparse embeddings (Section 2) Phi_b D_b / sqrt(kappa) of
    v rows each.  Inner sketch b hashes a row by its index in A.  Tiny n only.
    """
    h, _ = hash(seed, q, 0, n)
    seeds = general_seeds(seed, kappa)
    order = np.argsort(h, kind="stable")
    P = np.zeros((n, n))
    P[np.arange(n), order] = 1.0
    blocks = []
    for i in range(q):
        rows_i = order[h[order] == i]          # rows of A in h^-1(i), ascending
        Bi = np.zeros((v * kappa, len(rows_i)))
        for bidx in range(kappa):
            hb, sb = hash(seeds[bidx], v, 0, n)
            for c, r in enumerate(rows_i):
                Bi[bidx * v + hb[r], c] = sb[r] / np.sqrt(kappa)
        blocks.append(Bi)
    return sla.block_diag(*blocks) @ P if n > 0 else np.zeros((q * v * kappa, 0))


def sketch_csr_general(row_ptr, col, val, d, b, q, v, kappa, seed):
    """(SA, Sb) of the generalized sparse embedding by the plain row loop (C core)."""
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    n = row_ptr.shape[0] - 1
    t = q * v * kappa
    SA = np.zeros((t, d))
    Sb = np.zeros(t) if b is not None else None
    _load().orc_sketch_csr_general(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _i64(q),
                                   _i64(v), _i64(kappa), _u64(seed), _ptr(SA), _ptr(Sb))
    return SA, Sb


def csr_matvec(row_ptr, col, val, x):
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    x = _np(x, np.float64)
    n = row_ptr.shape[0] - 1
    y = np.zeros(n)
    _load().orc_csr_matvec(_i64(n), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def csr_rmatvec(row_ptr, col, val, d, z):
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    z = _np(z, np.float64)
    n = row_ptr.shape[0] - 1
    g = np.zeros(d)
    _load().orc_csr_rmatvec(_i64(n), _i64(d), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(z), _ptr(g))
    return g


# ---------------------------------------------------------------- QR and sketch-and-solve

def qr_r(SA, Sb=None):
    """Householder QR of SA (float64): R with a positive diagonal, and c = Q^T Sb.

    The sign convention (diag R > 0) is this build's reading; the paper leaves it
    open.  Returns (R, c) with c None when Sb is None.
    """
    SA = np.asarray(SA, dtype=np.float64)
    Q, R = np.linalg.qr(SA, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    R = s[:, None] * R
    c = None
    if Sb is not None:
        c = s * (Q.T @ np.asarray(Sb, dtype=np.float64))
    return R, c


def gram(SA, Sb=None):
    """[SA | Sb]^T [SA | Sb] in float64 (d x d without Sb).

    Section 7.6 preconditions with any R for which SA R^-1 has orthonormal
    columns up to scale; the Cholesky factor of this Gram matrix is such an R
    (R^T R = (SA)^T SA).
    """
    X = np.asarray(SA, dtype=np.float64)
    if Sb is not None:
        X = np.concatenate([X, np.asarray(Sb, dtype=np.float64)[:, None]], axis=1)
    return X.T @ X


def solve_sketch(SA, Sb):
    """x' = argmin ||SA x - Sb|| = R^-1 Q^T Sb (proof of Theorem "renRegAlg")."""
    R, c = qr_r(SA, Sb)
    x = sla.solve_triangular(R, c, lower=False)
    return x, R


def residual_norm_csr(row_ptr, col, val, b, x):
    y = csr_matvec(row_ptr, col, val, x)
    return float(np.linalg.norm(y - _np(b, np.float32).astype(np.float64)))


def lstsq_exact_dense(A, b):
    """x* = argmin ||Ax - b|| by Householder QR of [A | b] in float64.

    Returns (x*, ||Ax* - b||).
    """
    A = np.asarray(_np(A, np.float32), dtype=np.float64)
    b = np.asarray(_np(b, np.float32), dtype=np.float64)
    d = A.shape[1]
    R = np.linalg.qr(np.column_stack([A, b]), mode="r")
    x = sla.solve_triangular(R[:d, :d], R[:d, d], lower=False)
    return x, abs(float(R[d, d]))


def lstsq_exact_csr(row_ptr, col, val, d, b, block=1 << 15):
    """x* for CSR A by streaming Householder QR of [A | b] over row blocks (float64).

    The running (d+1) x (d+1) triangle is stacked on each dense row block and
    re-factored, so memory stays O(block * d).  Returns (x*, ||Ax* - b||).
    """
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32)
    n = row_ptr.shape[0] - 1
    Rr = np.zeros((0, d + 1))
    for s in range(0, n, block):
        e = min(n, s + block)
        blk = np.zeros((e - s, d + 1))
        lo, hi = int(row_ptr[s]), int(row_ptr[e])
        rows = np.repeat(np.arange(e - s), np.diff(row_ptr[s:e + 1]))
        np.add.at(blk, (rows, col[lo:hi]), val[lo:hi].astype(np.float64))
        blk[:, d] = b[s:e]
        Rr = np.linalg.qr(np.vstack([Rr, blk]), mode="r")
    x = sla.solve_triangular(Rr[:d, :d], Rr[:d, d], lower=False)
    return x, abs(float(Rr[d, d]))


def residual_ratio_csr(row_ptr, col, val, b, x, rstar_norm):
    """rho = ||A x - b|| / ||A x* - b|| in float64."""
    return residual_norm_csr(row_ptr, col, val, b, x) / rstar_norm


# ---------------------------------------------------------------- preconditioned LSQR

def lsqr_precond(matvec, rmatvec, b, R, x0, rtol, max_iter):
    """LSQR on min ||A R^-1 y - b||, started at y0 = R x0, returning x = R^-1 y.

    Section 7.6 of the paper runs a CG-like method on the well-conditioned
    A R with R from a subspace embedding; this is Paige and Saunders' LSQR
    (Golub-Kahan bidiagonalisation plus Givens QR) on that operator.  Stopping
    rule (this build's reading of "relative residual 1e-6"): stop when
    ||(AR^-1)^T r|| / (||AR^-1||_F ||r||) <= rtol, or when
    ||r|| <= rtol (||b|| + ||AR^-1||_F ||y||), all norms being the LSQR
    recurrence estimates except ||b|| and ||y||, which are computed.
    ``max_iter`` iterations without meeting either test is a non-convergence.

    Returns (x, iterations, test2, converged, history) where history holds the
    per-iteration (rnorm estimate, arnorm estimate).
    """
    b = np.asarray(b, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    y0 = R @ x0

    def abar(v):  # A R^-1 v
        return matvec(sla.solve_triangular(R, v, lower=False))

    def abar_t(u):  # R^-T A^T u
        return sla.solve_triangular(R, rmatvec(u), lower=False, trans="T")

    r0 = b - matvec(x0)
    beta = float(np.linalg.norm(r0))
    d = R.shape[0]
    dy = np.zeros(d)
    history = []
    if beta == 0.0:
        return x0.copy(), 0, 0.0, True, history
    u = r0 / beta
    g = abar_t(u)
    alpha = float(np.linalg.norm(g))
    if alpha == 0.0:
        return x0.copy(), 0, 0.0, True, history
    v = g / alpha
    w = v.copy()
    phibar = beta
    rhobar = alpha
    anorm2 = 0.0
    test2 = np.inf
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        z = abar(v) - alpha * u
        beta = float(np.linalg.norm(z))
        anorm2 += alpha * alpha + beta * beta
        if beta > 0.0:
            u = z / beta
            g = abar_t(u) - beta * v
        else:
            g = -beta * v
        alpha = float(np.linalg.norm(g))
        if alpha > 0.0:
            v = g / alpha
        rho = float(np.hypot(rhobar, beta))
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        dy = dy + (phi / rho) * w
        w = v - (theta / rho) * w
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        anorm = np.sqrt(anorm2)
        ynorm = float(np.linalg.norm(y0 + dy))
        history.append((rnorm, arnorm))
        test2 = arnorm / (anorm * rnorm) if rnorm > 0 else 0.0
        if test2 <= rtol or rnorm <= rtol * (bnorm + anorm * ynorm):
            converged = True
            break
    x = x0 + sla.solve_triangular(R, dy, lower=False)
    return x, it, float(test2), converged, history


def lsqr_precond_csr(row_ptr, col, val, d, b, R, x0, rtol, max_iter):
    row_ptr = _np(row_ptr, np.int32)
    col = _np(col, np.int32)
    val = _np(val, np.float32)
    b = _np(b, np.float32).astype(np.float64)
    return lsqr_precond(lambda x: csr_matvec(row_ptr, col, val, x),
                        lambda z: csr_rmatvec(row_ptr, col, val, d, z),
                        b, R, x0, rtol, max_iter)


# ---------------------------------------------------------------- leverage scores

def leverage_same(A, R, G, rows=None, chunk=1 << 16):
    """u'_i = ||(A R^-1 G)_i||^2 / k in float64 (Theorem "icml", Pi_2 = G/sqrt(k)).

    ``rows`` optionally restricts the output to those row indices.
    """
    A = _np(A, np.float32)
    R = np.asarray(R, dtype=np.float64)
    G = np.asarray(_np(G, np.float64), dtype=np.float64)
    k = G.shape[1]
    M = sla.solve_triangular(R, G, lower=False)
    if rows is not None:
        rows = np.asarray(rows)
        Y = A[rows].astype(np.float64) @ M
        return (Y * Y).sum(axis=1) / k
    n = A.shape[0]
    out = np.empty(n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        Y = A[s:e].astype(np.float64) @ M
        out[s:e] = (Y * Y).sum(axis=1) / k
    return out


def leverage_exact(A):
    """u_i = ||Q_i||^2 with Q from a float64 Householder QR of the stored A."""
    A = np.asarray(_np(A, np.float32), dtype=np.float64)
    Q = np.linalg.qr(A, mode="reduced")[0]
    return (Q * Q).sum(axis=1)


def distortion(SA, A_R):
    """Singular values of SA R_A^-1 (= S Q for A = Q R_A): the embedding distortion.

    Report-only quantity (the paper's bounds on it carry unspecified constants).
    """
    M = sla.solve_triangular(np.asarray(A_R, dtype=np.float64), np.eye(A_R.shape[0]), lower=False)
    return np.linalg.svd(np.asarray(SA, dtype=np.float64) @ M, compute_uv=False)
