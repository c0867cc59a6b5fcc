"""Host logic of the learned sketch (no GPU): the selection between the trained
and the plain sketch, and the Gaussian-sketch reference ratio."""
import math

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


def test_evaluate_reports_both_ratios_per_member():
    members = [_Member(1.1, 1.2), _Member(1.3, 1.0)]
    plain, learned = L.evaluate(_Sketch(), members)
    assert plain == [1.1, 1.3] and learned == [1.2, 1.0]


def test_gaussian_sketch_ratio():
    # E[rho^2] - 1 = d / (m - d - 1) for an m-row Gaussian sketch
    assert L.gaussian_sketch_ratio(2048, 128) == pytest.approx(math.sqrt(1 + 128 / 1919))
    assert L.gaussian_sketch_ratio(10 ** 9, 1) == pytest.approx(1.0, abs=1e-8)
