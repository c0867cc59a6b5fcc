"""Pins for the oracle's seeded map (h, sigma) that defines S = Phi D (paper Section 2).

The C core (128-bit Horner, ``%`` reduction) is checked against: the published
SplitMix64 outputs (tests/golden/splitmix64.txt), the polynomial's definition
evaluated with Python integers as a sum of powers, the vanishing fourth finite
difference of a cubic, interpolation of the coefficients, and the statistical
properties the paper asks of h and D (uniform buckets, fair independent signs).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import hash_bigint as hb

P = (1 << 61) - 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


def test_splitmix64_published_vectors():
    for seed, *outs in _golden():
        g = hb.splitmix64_stream(seed)
        assert [next(g) for _ in outs] == outs


def test_coefficients_are_masked_splitmix_draws():
    # seed 0: the first 8 draws masked to 61 bits (none equals p for this seed)
    seed = 0
    g = hb.splitmix64_stream(seed)
    draws = [next(g) & P for _ in range(8)]
    assert all(c != P for c in draws)
    assert oracle.coeffs(seed) == draws
    cb, cs = hb.coefficients(seed)
    assert cb + cs == draws


@pytest.mark.parametrize("seed", [0, 1, 2, 7, 1234567, 2**63 + 5, 2**64 - 1])
def test_c_core_matches_bigint_definition(seed):
    cb, cs = hb.coefficients(seed)
    assert oracle.coeffs(seed) == cb + cs
    idx = list(range(0, 200)) + [2**31 - 3, 2**31 - 2, 2**31 - 1, 2**40 + 11, P - 1, P, P + 3]
    for i in idx:
        gb, gs = oracle.poly_values(seed, i, 1)
        assert int(gb[0]) == hb.poly(cb, i)
        assert int(gs[0]) == hb.poly(cs, i)


@pytest.mark.parametrize("m", [1, 2, 3, 4096, 65536, 1000003, 2**31 - 1])
def test_bucket_and_sign_match_bigint(m):
    seed = 11
    i0 = 2**31 - 1000
    h, s = oracle.hash(seed, m, i0, 1000)
    hh, ss = hb.hash_rows(seed, m, range(i0, i0 + 1000))
    assert h.tolist() == hh
    assert s.tolist() == ss
    h, s = oracle.hash(seed, m, 0, 3000)
    hh, ss = hb.hash_rows(seed, m, range(3000))
    assert h.tolist() == hh and s.tolist() == ss


def test_cubic_fourth_difference_vanishes():
    # g is a cubic over F_p: its fourth forward difference is 0 mod p
    gb, gs = oracle.poly_values(3, 1000, 64)
    for g in (gb, gs):
        v = [int(t) for t in g]
        for x in range(len(v) - 4):
            d4 = (v[x + 4] - 4 * v[x + 3] + 6 * v[x + 2] - 4 * v[x + 1] + v[x]) % P
            assert d4 == 0


def test_interpolation_recovers_coefficients():
    # values at x = 0..3 determine (c0..c3) by Lagrange interpolation over F_p
    seed = 99
    cb, cs = hb.coefficients(seed)
    gb, gs = oracle.poly_values(seed, 0, 4)
    for vals, c in ((gb, cb), (gs, cs)):
        y = [int(t) for t in vals]
        inv = lambda a: pow(a % P, P - 2, P)
        # Newton forward differences -> monomial coefficients
        d1 = [(y[i + 1] - y[i]) % P for i in range(3)]
        d2 = [(d1[i + 1] - d1[i]) % P for i in range(2)]
        d3 = (d2[1] - d2[0]) % P
        c3 = d3 * inv(6) % P
        c2 = (d2[0] * inv(2) - 3 * c3) % P  # d2(0) = 2 c2 + 6 c3
        c1 = (d1[0] - c3 - c2) % P          # d1(0) = c3 + c2 + c1
        c0 = y[0] % P
        assert [c0, c1, c2, c3] == c


def test_buckets_uniform_and_signs_fair():
    n, m = 1 << 18, 256
    h, s = oracle.hash(5, m, 0, n)
    counts = np.bincount(h, minlength=m)
    chi2 = ((counts - n / m) ** 2 / (n / m)).sum()
    # chi-square with 255 dof: mean 255, sd ~22.6; 6 sd band
    assert chi2 < 255 + 6 * 22.6
    assert abs(s.astype(np.int64).sum()) < 6 * np.sqrt(n)
    # signs and buckets carry no linear dependence on each other
    assert abs(np.corrcoef(h, s)[0, 1]) < 6 / np.sqrt(n)


def test_pairwise_collisions_over_seeds():
    # for fixed rows i != j, P[h(i) = h(j)] = 1/m over the random seed
    m, seeds = 64, 4000
    hits = 0
    for seed in range(seeds):
        h, _ = oracle.hash(seed, m, 10, 2)
        hits += int(h[0] == h[1])
    p = 1.0 / m
    assert abs(hits - seeds * p) < 6 * np.sqrt(seeds * p * (1 - p))


def test_four_sign_products_unbiased_over_seeds():
    # 4-wise independence of sigma: E[s_a s_b s_c s_d] = 0 for distinct rows
    seeds = 4000
    acc = 0
    for seed in range(seeds):
        _, s = oracle.hash(seed, 8, 100, 4)
        acc += int(np.prod(s.astype(np.int64)))
    assert abs(acc) < 6 * np.sqrt(seeds)
