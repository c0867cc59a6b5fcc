"""Seeded synthetic inputs shaped like the paper's regression and leverage workloads.

This module is shared by the tests, the CPU oracle and the benchmark.  It holds
no arithmetic of the sketching method (no hashing, no bucketing, no sketch):
only random sparse / dense matrices, right-hand sides and Gaussian matrices.
Everything is drawn with torch generators seeded from the documented integer
seeds, on the device the caller names (``"cpu"`` for the CPU test suite,
``"cuda"`` for the full-size workloads, which would take minutes on the host).
A given (function, arguments, device) always returns the same arrays.

Recipes (the tall regression setting of Section 7 and the leverage setting of
Section 6 of the paper):

* ``csr_fixed_k``: every row has exactly ``k`` distinct columns, sampled without
  replacement with probabilities ``p`` over the ``d`` columns (uniform, or
  Zipf(s): p_c proportional to c^-s for c = 1..d).  Sampling without
  replacement uses exponential keys (Efraimidis and Spirakis, 2006): column c
  gets E_c / p_c with E_c ~ Exp(1) and the k smallest keys win, which has the
  same law as drawing columns one at a time and rejecting repeats.  Columns are
  stored ascending within a row.  Values are N(0,1) drawn in float64 and
  stored as float32.
* ``csr_random_lengths``: row lengths uniform in [kmin, kmax] (optionally a
  fraction of empty rows), uniform distinct columns.
* ``dense_lowrank``: A = U diag(sigma) V^T with U (n x d) and V (d x d) the
  sign-fixed Q factors of Gaussian matrices (Haar distributed), float32.
* ``rhs``: b = A x0 + noise * N(0,1), x0 ~ N(0,1)^d, float32.
* ``gaussian``: G ~ N(0,1)^{d x k}, float64.
* ``family_basis`` / ``family_matrix``: the learned-sketch workload, a family of
  matrices A = U diag(sigma) V^T + 1e-3 N(0,1) (n x d) with V (d x d) Haar and
  fixed for the family (seed 7), U (n x d) Haar per matrix (sign-fixed Q of a
  float32 Gaussian's QR), sigma_j = j^-1.5, b = A x0 + 0.05 N(0,1); matrix k of
  the family is drawn from seed 1000003 + k.
* ``batch_shapes`` / ``batch_problem``: the batched regression workload, many
  independent problems with n log-uniform in [2^lo, 2^hi] (n = floor(2^U),
  U uniform), d drawn uniformly from a set, row lengths uniform in
  [kmin, kmax] (at most d) with uniform distinct columns, N(0,1) values,
  b = A x0 + 0.1 N(0,1), sketch rows m = 4 d^2, seed of problem p = p + 1.
"""
from __future__ import annotations

import math

import numpy as np
import torch

__all__ = [
    "CSR",
    "csr_fixed_k",
    "csr_uniform",
    "csr_zipf",
    "csr_random_lengths",
    "rhs",
    "dense_lowrank",
    "dense_gaussian",
    "gaussian",
    "geometric_sigma",
    "zipf_probs",
    "batch_shapes",
    "batch_problem",
    "family_basis",
    "family_matrix",
]

_CHUNK = 1 << 18


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


class CSR:
    """CSR matrix with int32 row_ptr / col and float32 val torch tensors, shape (n, d)."""

    def __init__(self, n, d, row_ptr, col, val):
        self.n = int(n)
        self.d = int(d)
        self.row_ptr = row_ptr.to(torch.int32).contiguous()
        self.col = col.to(torch.int32).contiguous()
        self.val = val.to(torch.float32).contiguous()

    @property
    def nnz(self):
        return int(self.col.numel())

    @property
    def device(self):
        return self.val.device

    def to(self, device):
        return CSR(self.n, self.d, self.row_ptr.to(device), self.col.to(device), self.val.to(device))

    def numpy(self):
        """(row_ptr, col, val) as host numpy arrays."""
        return (self.row_ptr.cpu().numpy(), self.col.cpu().numpy(), self.val.cpu().numpy())

    def rows(self, r0, r1):
        """The sub-matrix of rows [r0, r1) as a new CSR (row_ptr rebased to 0)."""
        rp = self.row_ptr[r0:r1 + 1].to(torch.int64)
        s, e = int(rp[0]), int(rp[-1])
        return CSR(r1 - r0, self.d, (rp - s).to(torch.int32), self.col[s:e], self.val[s:e])

    def to_dense(self, dtype=torch.float64):
        out = torch.zeros(self.n, self.d, dtype=dtype, device=self.device)
        lens = (self.row_ptr[1:] - self.row_ptr[:-1]).to(torch.int64)
        rows = torch.repeat_interleave(torch.arange(self.n, device=self.device), lens)
        out.index_put_((rows, self.col.to(torch.int64)), self.val.to(dtype), accumulate=True)
        return out

    def matvec(self, x):
        """y = A x in float64 (x of length d)."""
        x = torch.as_tensor(x, dtype=torch.float64, device=self.device)
        lens = (self.row_ptr[1:] - self.row_ptr[:-1]).to(torch.int64)
        rows = torch.repeat_interleave(torch.arange(self.n, device=self.device), lens)
        prod = self.val.to(torch.float64) * x[self.col.to(torch.int64)]
        y = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        y.index_add_(0, rows, prod)
        return y


def zipf_probs(d, s):
    c = torch.arange(1, d + 1, dtype=torch.float64)
    p = c ** (-float(s))
    return p / p.sum()


def csr_fixed_k(n, d, k, p, seed, device="cpu"):
    """n x d CSR with exactly k distinct columns per row drawn without replacement from p."""
    if not 0 <= k <= d:
        raise ValueError("need 0 <= k <= d")
    g = _gen(seed, device)
    inv_p = (1.0 / torch.as_tensor(p, dtype=torch.float64)).to(torch.float32).to(device)
    col = torch.empty(n * k, dtype=torch.int32, device=device)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        keys = torch.empty(e - s, d, dtype=torch.float32, device=device).exponential_(generator=g)
        keys *= inv_p
        idx = keys.topk(k, dim=1, largest=False).indices.sort(dim=1).values
        col[s * k:e * k] = idx.reshape(-1).to(torch.int32)
    val = torch.randn(n * k, dtype=torch.float64, device=device, generator=g).to(torch.float32)
    row_ptr = torch.arange(n + 1, dtype=torch.int64, device=device) * k
    return CSR(n, d, row_ptr.to(torch.int32), col, val)


def csr_uniform(n, d, k, seed, device="cpu"):
    """Exactly k distinct uniformly chosen columns per row, N(0,1) values."""
    return csr_fixed_k(n, d, k, torch.full((d,), 1.0 / d, dtype=torch.float64), seed, device)


def csr_zipf(n, d, k, s, seed, device="cpu"):
    """Exactly k distinct columns per row from Zipf(s) over d columns, N(0,1) values."""
    return csr_fixed_k(n, d, k, zipf_probs(d, s), seed, device)


def csr_random_lengths(n, d, kmin, kmax, seed, empty_frac=0.0, device="cpu"):
    """Row lengths uniform in [kmin, kmax], a fraction ``empty_frac`` of rows empty."""
    g = _gen(seed, device)
    lens = torch.randint(kmin, kmax + 1, (n,), generator=g, device=device)
    if empty_frac > 0:
        lens = torch.where(torch.rand(n, generator=g, device=device) < empty_frac,
                           torch.zeros_like(lens), lens)
    lens = lens.clamp(max=d)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(lens, 0)
    nnz = int(row_ptr[-1])
    # per row: the first len_i columns of a uniformly random key order (distinct, uniform)
    col = torch.empty(nnz, dtype=torch.int32, device=device)
    kmax_eff = int(lens.max()) if n else 0
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        if kmax_eff == 0:
            break
        keys = torch.rand(e - s, d, generator=g, device=device)
        idx = keys.topk(kmax_eff, dim=1, largest=False).indices
        L = lens[s:e]
        take = torch.arange(kmax_eff, device=device)[None, :] < L[:, None]
        big = torch.where(take, idx, torch.full_like(idx, d))
        big = big.sort(dim=1).values
        col[int(row_ptr[s]):int(row_ptr[e])] = big[take].to(torch.int32)
    val = torch.randn(nnz, dtype=torch.float64, device=device, generator=g).to(torch.float32)
    return CSR(n, d, row_ptr.to(torch.int32), col, val)


def rhs(A, noise, seed):
    """b = A x0 + noise * N(0,1) with x0 ~ N(0,1)^d.  Returns (b float32, x0 float64).

    ``A`` is a CSR or a dense float32 tensor; b lives on A's device.
    """
    dev = A.device
    g = _gen(seed, dev)
    if isinstance(A, CSR):
        d = A.d
        x0 = torch.randn(d, dtype=torch.float64, device=dev, generator=g)
        y = A.matvec(x0)
        n = A.n
    else:
        n, d = A.shape
        x0 = torch.randn(d, dtype=torch.float64, device=dev, generator=g)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        for s in range(0, n, _CHUNK):
            e = min(n, s + _CHUNK)
            y[s:e] = A[s:e].to(torch.float64) @ x0
    b = y + noise * torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    return b.to(torch.float32), x0


def _haar(rows, cols, g, device):
    q, r = torch.linalg.qr(torch.randn(rows, cols, dtype=torch.float64, device=device, generator=g))
    s = torch.sign(torch.diagonal(r))
    s[s == 0] = 1.0
    return q * s


def geometric_sigma(d, lo):
    """sigma_j = lo^((j-1)/(d-1)), j = 1..d: geometric from 1 down to lo (float64)."""
    if d == 1:
        return torch.ones(1, dtype=torch.float64)
    return torch.tensor(float(lo), dtype=torch.float64) ** (torch.arange(d, dtype=torch.float64) / (d - 1))


def dense_lowrank(n, d, sigma, seed, device="cpu"):
    """A = U diag(sigma) V^T with U (n x d) and V (d x d) Haar; float32 (n, d) row-major."""
    g = _gen(seed, device)
    V = _haar(d, d, g, device)
    U = _haar(n, d, g, device)
    A = (U * torch.as_tensor(sigma, dtype=torch.float64, device=device)) @ V.T
    return A.to(torch.float32).contiguous()


def dense_gaussian(n, d, seed, device="cpu"):
    g = _gen(seed, device)
    return torch.randn(n, d, dtype=torch.float64, device=device, generator=g).to(torch.float32)


def gaussian(d, k, seed, device="cpu"):
    """G ~ N(0,1)^{d x k}, float64 (the Johnson-Lindenstrauss matrix of Section 6)."""
    g = _gen(seed, device)
    return torch.randn(d, k, dtype=torch.float64, device=device, generator=g)


def batch_shapes(count, seed, log2n=(12, 18), dset=(16, 32, 64, 128), krange=(4, 32)):
    """Per problem a dict(n, d, m, kmin, kmax, seed) of the batched workload."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, dtype=torch.float64, generator=g) * (log2n[1] - log2n[0]) + log2n[0]
    di = torch.randint(0, len(dset), (count,), generator=g)
    out = []
    for p in range(count):
        d = int(dset[int(di[p])])
        out.append(dict(n=int(math.floor(2.0 ** float(u[p]))), d=d, m=4 * d * d, kmin=min(krange[0], d),
                        kmax=min(krange[1], d), seed=p + 1))
    return out


def batch_problem(shape, device="cpu"):
    """(A, b) of one problem of ``batch_shapes``."""
    s = shape
    A = csr_random_lengths(s["n"], s["d"], s["kmin"], s["kmax"], seed=100003 + s["seed"], device=device)
    b, _ = rhs(A, 0.1, seed=200003 + s["seed"])
    return A, b


def family_basis(d=128, seed=7, device="cpu"):
    """(V, sigma) of the matrix family: V (d x d) Haar float64, sigma_j = j^-1.5."""
    g = _gen(seed, device)
    V = _haar(d, d, g, device)
    sigma = torch.arange(1, d + 1, dtype=torch.float64, device=device) ** -1.5
    return V, sigma


def haar_rinv(Z):
    """R^-1 (float64, d x d) for the Cholesky factor R of Z^T Z: Z R^-1 is the Q
    factor of Z's QR with R's diagonal positive (the two are the same matrix),
    Haar-distributed for a Gaussian Z."""
    d = Z.shape[1]
    R = torch.linalg.cholesky((Z.T @ Z).double()).T
    return torch.linalg.solve_triangular(R, torch.eye(d, dtype=torch.float64, device=Z.device), upper=True)


def family_matrix(k, n, V, sigma, device="cpu"):
    """(A float32 (n, d) row-major, b float32 (n,)) of member k of the family:
    A = U diag(sigma) V^T + 1e-3 N(0, 1), b = A x0 + 0.05 N(0, 1).

    U is the Q factor, with R's diagonal made positive, of an n x d Gaussian
    Z: that Q is Haar-distributed, and it equals Z R^-1 for the Cholesky
    factor R of Z^T Z (the positive-diagonal QR factor is unique), so A is
    formed as Z (R^-1 diag(sigma) V^T) by one matrix product."""
    d = V.shape[0]
    g = _gen(1000003 + k, device)
    Z = torch.randn(n, d, dtype=torch.float32, device=device, generator=g)
    Rinv = haar_rinv(Z)
    mix = (Rinv * sigma.to(device=device, dtype=torch.float64)) @ V.to(device=device, dtype=torch.float64).T
    A = Z @ mix.to(torch.float32)
    del Z
    A += 1e-3 * torch.randn(n, d, dtype=torch.float32, device=device, generator=g)
    x0 = torch.randn(d, dtype=torch.float64, device=device, generator=g)
    y = (A.double() @ x0) if n * d <= (1 << 24) else torch.cat(
        [A[s:s + _CHUNK].double() @ x0 for s in range(0, n, _CHUNK)])
    b = y + 0.05 * torch.randn(n, dtype=torch.float64, device=device, generator=g)
    return A.contiguous(), b.to(torch.float32)

