"""Learned + random sketches for sketch-and-solve on a matrix family.

The sketch stacks two halves of m/2 rows each: S = [S_L; S_R].
* S_R is the sparse embedding of Section 2 (seed_R): one random sign per
  column, so every column of S keeps a random entry and the worst-case
  guarantee of the random half survives.
* S_L has the hash positions of Section 2 (seed_L) with trainable values.
  Two parameterisations:
  - ``LearnedSketch``: one value v_i per column of S (n free values,
    initialised to the signs); SA_L = S_L(v) A through the library's values
    sketch and its gather backward (``SketchValues``).
  - ``TiedSketch``: one value w_k per row of S_L (m/2 free values, initialised
    to 1), i.e. v_i = w_{h(i)} sigma(i), so S_L(v) = diag(w) S_L and
    SA_L = diag(w) (S_L A).  The loss then depends on A only through the two
    plain sketches and the Gram matrix of [A b], which are kept per matrix
    (``TiedMember``) instead of A itself.
x'(S) = argmin ||S A x - S b|| is the library's float64 Householder solve of
the sketched system (``SketchedSolve``: cw_solve_sketched forward, the
hand-derived cw_solve_sketched_backward; ``method="normal"`` trains through
the Cholesky factor of the sketched system's Gram matrix instead, the same R
and x' up to rounding at a fraction of the QR's latency; ratios are always
judged through the QR), and the loss is the excess squared residual ratio
    rho^2 - 1 = ||A (x' - x*)||^2 / ||A x* - b||^2
(b - A x* is orthogonal to the range of A), computed by the library from the
bordered Gram matrix of [A b] (``MatrixStats``: cw_gram, cw_normal_solve,
cw_excess_residual).  Adam updates the values.

The comparison is against the plain sparse embedding with the same m (one
sign per column, seed_P).  ``select_or_fallback`` keeps the trained sketch
only if it beats the plain one on a selection set of held-out matrices; the
ratios reported afterwards come from a separate report set.
"""
from __future__ import annotations

import math

import torch

from . import (ScaleRows, SketchedSolve, SketchValues, cw_excess_residual, cw_gram, cw_hash, cw_normal_solve,
               cw_sketch_dense, cw_solve_sketch_dense)


class _Excess(torch.autograd.Function):
    """rho^2 - 1 as a differentiable function of x (cw_excess_residual)."""

    @staticmethod
    def forward(ctx, x, G, xstar, r2):
        loss, gx = cw_excess_residual(G, xstar, r2, x.detach().contiguous())
        ctx.save_for_backward(gx)
        return loss

    @staticmethod
    def backward(ctx, g):
        (gx,) = ctx.saved_tensors
        return gx * g, None, None, None


class MatrixStats:
    """Per-matrix constants of the loss: the bordered Gram matrix
    G = [A b]^T [A b] (cw_gram), x* and ||A x* - b||^2 (cw_normal_solve)."""

    def __init__(self, A, b):
        self.G = cw_gram(A, b)
        self.xstar, self.rstar2 = cw_normal_solve(self.G)

    def excess(self, x):
        """rho^2 - 1 for the solution x (differentiable in x)."""
        return _Excess.apply(x, self.G, self.xstar, self.rstar2)

    def ratio(self, x):
        loss, _ = cw_excess_residual(self.G, self.xstar, self.rstar2, x.detach().contiguous(), want_grad=False)
        return math.sqrt(1.0 + float(loss))


def plain_ratio(A, b, stats, m, seed_P):
    """Residual ratio of the plain sparse embedding with m rows (cw_solve_sketch_dense)."""
    return stats.ratio(cw_solve_sketch_dense(A, b, m, seed_P))


class FullMember:
    """One matrix for ``LearnedSketch``: A, b, the loss constants, the random
    half's sketch and the plain sketch's residual ratio."""

    def __init__(self, A, b, stats, rand_half, plain):
        self.A, self.b, self.stats, self.rand_half, self.plain = A, b, stats, rand_half, plain


class LearnedSketch:
    """S = [S_L(v); S_R] with m/2 rows each; v trainable (float32, one value per column)."""

    def __init__(self, n, m, seed_L=11, seed_R=12, device="cuda", method="qr"):
        if m % 2:
            raise ValueError("m must be even")
        self.method = method
        self.n, self.m, self.mh = n, m, m // 2
        self.seed_L, self.seed_R = seed_L, seed_R
        _, sign = cw_hash(seed_L, self.mh, 0, n)
        self.v = sign.to(torch.float32).clone().requires_grad_(True)

    def parameters(self):
        return [self.v]

    def random_half(self, A, b):
        return cw_sketch_dense(A, b, self.mh, self.seed_R)

    def solve(self, A, b, rand_half=None, method="qr"):
        SA_R, Sb_R = rand_half if rand_half is not None else self.random_half(A, b)
        SA_L, Sb_L = SketchValues.apply(self.v, A, b, self.mh, self.seed_L)
        return SketchedSolve.apply(torch.cat([SA_L, SA_R]), torch.cat([Sb_L, Sb_R]), method)

    def member(self, A, b, m_plain=None, seed_P=13):
        """The FullMember of (A, b); A is kept (the values sketch reads it every step)."""
        st = MatrixStats(A, b)
        plain = plain_ratio(A, b, st, m_plain or self.m, seed_P)
        return FullMember(A, b, st, self.random_half(A, b), plain)

    def loss(self, member):
        return member.stats.excess(self.solve(member.A, member.b, member.rand_half, self.method))

    def ratio(self, member):
        with torch.no_grad():
            return member.stats.ratio(self.solve(member.A, member.b, member.rand_half))


class TiedMember:
    """What the tied sketch needs of one matrix: P = [S_L A; S_R A] and
    Pb = [S_L b; S_R b] (plain sketches, m x d and m), the loss constants, and
    the plain sketch's residual ratio (m rows, seed_P)."""

    def __init__(self, P, Pb, stats, plain):
        self.P, self.Pb, self.stats, self.plain = P, Pb, stats, plain


class TiedSketch:
    """S = [diag(w) S_L; S_R] with m/2 rows each; w trainable (float32, one value
    per row of S_L, i.e. per learned bucket)."""

    def __init__(self, m, seed_L=11, seed_R=12, device="cuda", method="qr"):
        if m % 2:
            raise ValueError("m must be even")
        self.method = method
        self.m, self.mh = m, m // 2
        self.seed_L, self.seed_R = seed_L, seed_R
        self.w = torch.ones(self.mh, dtype=torch.float32, device=device, requires_grad=True)

    def parameters(self):
        return [self.w]

    def values(self, n):
        """The per-column values v_i = w_{h(i)} sigma(i) of S_L (float32, n)."""
        bucket, sign = cw_hash(self.seed_L, self.mh, 0, n)
        return self.w.detach()[bucket.long()] * sign.to(torch.float32)

    def sketch_pair(self, A, b):
        SA_L, Sb_L = cw_sketch_dense(A, b, self.mh, self.seed_L)
        SA_R, Sb_R = cw_sketch_dense(A, b, self.mh, self.seed_R)
        return torch.cat([SA_L, SA_R]), torch.cat([Sb_L, Sb_R])

    def solve_sketched(self, P, Pb, method="qr"):
        M, y = ScaleRows.apply(self.w, P, Pb, self.mh)
        return SketchedSolve.apply(M, y, method)

    def solve(self, A, b):
        return self.solve_sketched(*self.sketch_pair(A, b))

    def member(self, A, b, m_plain=None, seed_P=13):
        """The TiedMember of (A, b); A itself is not kept."""
        st = MatrixStats(A, b)
        P, Pb = self.sketch_pair(A, b)
        plain = plain_ratio(A, b, st, m_plain or self.m, seed_P)
        return TiedMember(P, Pb, st, plain)

    def loss(self, member):
        return member.stats.excess(self.solve_sketched(member.P, member.Pb, self.method))

    def ratio(self, member):
        with torch.no_grad():
            return member.stats.ratio(self.solve_sketched(member.P, member.Pb))


def train(sketch, members, epochs, lr=1e-3, seed=0, log=None):
    """Adam (one matrix per step, in a seeded random order each epoch) on the
    sketch's values; returns the mean loss per epoch.  ``members`` are
    ``sketch.member`` results."""
    opt = torch.optim.Adam(sketch.parameters(), lr=lr)
    g = torch.Generator().manual_seed(seed)
    hist = []
    for ep in range(epochs):
        order = torch.randperm(len(members), generator=g).tolist()
        tot = torch.zeros((), dtype=torch.float64, device=sketch.parameters()[0].device)
        for i in order:
            opt.zero_grad(set_to_none=True)
            loss = sketch.loss(members[i])
            loss.backward()
            opt.step()
            tot += loss.detach()
        hist.append(float(tot) / len(members))
        if log:
            log(ep, hist[-1])
    return hist


def evaluate(sketch, members):
    """Per-matrix residual ratios (plain, learned + random) on held-out members
    (each member carries its plain ratio)."""
    plain = [mem.plain for mem in members]
    learned = [sketch.ratio(mem) for mem in members]
    return plain, learned


class Selection:
    """The outcome of ``select_or_fallback``: the sketch to use for new matrices
    of the family."""

    def __init__(self, sketch, use_learned, m, seed_P, mean_plain, mean_learned):
        self.sketch, self.use_learned = sketch, use_learned
        self.m, self.seed_P = m, seed_P
        self.mean_plain, self.mean_learned = mean_plain, mean_learned

    @property
    def name(self):
        return "learned" if self.use_learned else "plain"

    def solve(self, A, b):
        """x' for a new matrix: the trained sketch if it won the selection,
        else the plain sparse embedding with the same m."""
        if self.use_learned:
            with torch.no_grad():
                return self.sketch.solve(A, b)
        return cw_solve_sketch_dense(A, b, self.m, self.seed_P)


def select_or_fallback(sketch, selection_members, m, seed_P):
    """Keep the trained sketch only if its mean residual ratio on the selection
    members is below the plain sketch's; otherwise fall back to plain."""
    if not selection_members:
        raise ValueError("select_or_fallback needs at least one selection member")
    plain, learned = evaluate(sketch, selection_members)
    mp, ml = sum(plain) / len(plain), sum(learned) / len(learned)
    return Selection(sketch, ml < mp, m, seed_P, mp, ml)


def gaussian_sketch_ratio(m, d):
    """sqrt(1 + d / (m - d - 1)): the expected residual ratio of sketch-and-solve
    with an m-row Gaussian sketch when the noise is Gaussian, the level an
    oblivious sketch reaches on a family whose rows are exchangeable."""
    return math.sqrt(1.0 + d / (m - d - 1.0))
