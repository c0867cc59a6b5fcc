"""Learned + random sketch for sketch-and-solve on a matrix family.

The sketch stacks two halves of m/2 rows each: S = [S_L(v); S_R].
* S_R is the sparse embedding of Section 2 (seed_R): one random sign per
  column, so every column of S keeps a random entry and the worst-case
  guarantee of the random half survives.
* S_L(v) has the hash positions of Section 2 (seed_L) with trainable values v_i
  (initialised to the signs): SA_L(v) = S_L(v) A through the library's
  kernels (``SketchValues``: cw_sketch_dense_values forward, the gather
  backward cw_sketch_values_backward_dense).
x'(v) = argmin ||S A x - S b|| is solved by a float64 Householder QR of the
m x d sketch (torch on the device, differentiable), and the training loss is
the exact excess squared residual ratio
    rho^2 - 1 = ||A (x' - x*)||^2 / ||A x* - b||^2
(b - A x* is orthogonal to the range of A), computed from the d x d Gram
matrix of A and x*, which are fixed per matrix.  Adam updates v.

The comparison is against the plain sparse embedding with the same m (one
sign per column, seed_P), and the trained sketch is used only if it beats the
plain one on held-out matrices (otherwise the plain sketch is kept).
"""
from __future__ import annotations

import math

import torch

from . import SketchValues, cw_hash, cw_sketch_dense, cw_solve_sketch_dense


class MatrixStats:
    """Per-matrix constants of the loss: G = A^T A, x*, ||A x* - b||^2 (float64)."""

    def __init__(self, A, b, chunk=1 << 18):
        d = A.shape[1]
        G = torch.zeros(d, d, dtype=torch.float64, device=A.device)
        c = torch.zeros(d, dtype=torch.float64, device=A.device)
        for s in range(0, A.shape[0], chunk):
            Ab = A[s:s + chunk].double()
            G += Ab.T @ Ab
            c += Ab.T @ b[s:s + chunk].double()
        L = torch.linalg.cholesky(G)
        xs = torch.cholesky_solve(c[:, None], L)[:, 0]
        r2 = 0.0
        for s in range(0, A.shape[0], chunk):
            r = A[s:s + chunk].double() @ xs - b[s:s + chunk].double()
            r2 += float((r * r).sum())
        self.G, self.xstar, self.rstar2 = G, xs, r2

    def excess(self, x):
        """rho^2 - 1 for the solution x (differentiable in x)."""
        e = x - self.xstar
        return (e @ (self.G @ e)) / self.rstar2

    def ratio(self, x):
        return math.sqrt(1.0 + float(self.excess(x)))


def qr_solve(SA, Sb):
    """argmin ||SA x - Sb|| by a float64 Householder QR (differentiable)."""
    Q, R = torch.linalg.qr(SA.double())
    return torch.linalg.solve_triangular(R, (Q.T @ Sb.double())[:, None], upper=True)[:, 0]


class LearnedSketch:
    """S = [S_L(v); S_R] with m/2 rows each; v trainable (float32, length n)."""

    def __init__(self, n, m, seed_L=11, seed_R=12, device="cuda"):
        if m % 2:
            raise ValueError("m must be even")
        self.n, self.m, self.mh = n, m, m // 2
        self.seed_L, self.seed_R = seed_L, seed_R
        _, sign = cw_hash(seed_L, self.mh, 0, n)
        self.v = sign.to(torch.float32).clone().requires_grad_(True)

    def random_half(self, A, b):
        return cw_sketch_dense(A, b, self.mh, self.seed_R)

    def solve(self, A, b, rand_half=None):
        SA_R, Sb_R = rand_half if rand_half is not None else self.random_half(A, b)
        SA_L, Sb_L = SketchValues.apply(self.v, A, b, self.mh, self.seed_L)
        return qr_solve(torch.cat([SA_L, SA_R]), torch.cat([Sb_L, Sb_R]))


def plain_ratio(A, b, stats, m, seed_P):
    """Residual ratio of the plain sparse embedding with m rows (cw_solve_sketch_dense)."""
    return stats.ratio(cw_solve_sketch_dense(A, b, m, seed_P))


def train(sketch, train_set, epochs, lr=1e-3, seed=0, log=None):
    """Adam on v over (A, b, stats, random half) tuples; returns mean loss per epoch."""
    opt = torch.optim.Adam([sketch.v], lr=lr)
    g = torch.Generator().manual_seed(seed)
    hist = []
    for ep in range(epochs):
        order = torch.randperm(len(train_set), generator=g).tolist()
        tot = 0.0
        for i in order:
            A, b, st, rh = train_set[i]
            opt.zero_grad(set_to_none=True)
            loss = st.excess(sketch.solve(A, b, rh))
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        hist.append(tot / len(train_set))
        if log:
            log(ep, hist[-1])
    return hist


def evaluate(sketch, test_set, m, seed_P):
    """Mean residual ratios on test matrices: plain sketch, learned + random."""
    plain, learned = [], []
    with torch.no_grad():
        for A, b, st, rh in test_set:
            plain.append(plain_ratio(A, b, st, m, seed_P))
            learned.append(st.ratio(sketch.solve(A, b, rh)))
    return sum(plain) / len(plain), sum(learned) / len(learned)
