"""Host logic of the learned sketch (no GPU): the selection between the trained
and the plain sketch, and the Gaussian-sketch reference ratio."""
import math

import numpy as np
import pytest

from paper_1207_6365_gb300 import learned as L


class _Member:
    def __init__(self, plain, learned):
        self.plain, self.learned = plain, learned


class _Sketch:
    """Stands in for a trained sketch: its ratio on a member is stored."""

    def ratio(self, member):
        return member.learned


def test_select_keeps_learned_only_when_it_wins_on_the_selection_set():
    sk = _Sketch()
    wins = [_Member(1.04, 1.02), _Member(1.03, 1.03), _Member(1.05, 1.04)]
    sel = L.select_or_fallback(sk, wins, m=2048, seed_P=13)
    assert sel.use_learned and sel.name == "learned"
    assert sel.mean_plain == pytest.approx(sum(m.plain for m in wins) / 3)
    assert sel.mean_learned == pytest.approx(sum(m.learned for m in wins) / 3)
    loses = [_Member(1.02, 1.03), _Member(1.03, 1.03)]
    sel = L.select_or_fallback(sk, loses, m=2048, seed_P=13)
    assert not sel.use_learned and sel.name == "plain"
    ties = [_Member(1.03, 1.03)]
    assert not L.select_or_fallback(sk, ties, m=2048, seed_P=13).use_learned   # a tie keeps plain
    with pytest.raises(ValueError):
        L.select_or_fallback(sk, [], m=2048, seed_P=13)


def test_evaluate_reports_both_ratios_per_member():
    members = [_Member(1.1, 1.2), _Member(1.3, 1.0)]
    plain, learned = L.evaluate(_Sketch(), members)
    assert plain == [1.1, 1.3] and learned == [1.2, 1.0]


def test_gaussian_sketch_ratio():
    # E[rho^2] - 1 = d / (m - d - 1) for an m-row Gaussian sketch
    assert L.gaussian_sketch_ratio(2048, 128) == pytest.approx(math.sqrt(1 + 128 / 1919))
    assert L.gaussian_sketch_ratio(10 ** 9, 1) == pytest.approx(1.0, abs=1e-8)


def test_gaussian_sketch_ratio_matches_simulation():
    # For a Gaussian S and a residual orthogonal to range(A), S A and S r* are
    # independent, and E[rho^2] - 1 = E tr((A^T S^T S A)^-1 A^T A) = d / (m - d - 1)
    # (the mean of an inverse Wishart matrix).  Simulated here for one fixed A:
    # 20000 sketches, the mean within four standard errors (d / (m - d) or
    # d / m would be more than ten away).
    rng = np.random.default_rng(3)
    n, d, m, T = 64, 4, 16, 20000
    A = rng.standard_normal((n, d))
    Q, _ = np.linalg.qr(A)
    r = rng.standard_normal(n)
    r -= Q @ (Q.T @ r)
    xs = rng.standard_normal(d)
    b = A @ xs + r
    S = rng.standard_normal((T, m, n))
    SA, Sb = S @ A, S @ b
    G = np.einsum("tmi,tmj->tij", SA, SA)
    c = np.einsum("tmi,tm->ti", SA, Sb)
    X = np.linalg.solve(G, c[..., None])[..., 0]
    excess = ((A @ (X - xs).T) ** 2).sum(0) / (r @ r)
    se = excess.std() / math.sqrt(T)
    want = L.gaussian_sketch_ratio(m, d) ** 2 - 1
    assert abs(excess.mean() - want) < 4 * se
    assert abs(d / (m - d) - want) > 10 * se
