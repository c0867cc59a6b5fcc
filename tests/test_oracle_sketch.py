"""Pins for the oracle's SA / Sb (paper Section 2 and the proof of Lemma "len fixed sparse").

* Brute force: SA equals the explicit m x n matrix S = Phi D times A
  (S[h(i), i] = sigma(i), all other entries 0) on tiny inputs.
* Exact invariants of a matrix with one +-1 per column: the column sums of SA
  equal D-weighted column sums of A, Sb likewise, and row shards add up.
* The paper's expectation E ||S x||^2 = ||x||^2 (proof of Lemma "len fixed
  sparse", eq. "exp") and the second moment from its fourth-moment expansion,
  Var ||S x||^2 = (2/m)(||x||_2^4 - ||x||_4^4) for pairwise uniform h and
  4-wise signs, both checked over many seeds.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W


def _csr(n, d, k, seed):
    return W.csr_uniform(n, d, k, seed)


@pytest.mark.parametrize("n,d,k,m", [(37, 5, 2, 7), (200, 16, 3, 64), (513, 9, 9, 32), (64, 4, 1, 1)])
def test_sa_equals_dense_S_times_A_csr(n, d, k, m):
    A = _csr(n, d, k, seed=n + d)
    b, _ = W.rhs(A, 0.3, seed=5)
    S = oracle.dense_S(seed=17, m=m, n=n)
    SA, Sb = oracle.sketch_csr(A.row_ptr, A.col, A.val, d, b, m, seed=17)
    Ad = A.to_dense().numpy()
    np.testing.assert_allclose(SA, S @ Ad, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Sb, S @ b.double().numpy(), rtol=0, atol=1e-12)


def test_sa_equals_dense_S_times_A_dense_and_vec():
    n, d, m = 301, 7, 19
    A = W.dense_gaussian(n, d, seed=3)
    b = W.dense_gaussian(n, 1, seed=4)[:, 0]
    S = oracle.dense_S(seed=23, m=m, n=n)
    SA, Sb = oracle.sketch_dense(A, b, m, seed=23)
    np.testing.assert_allclose(SA, S @ A.double().numpy(), atol=1e-12)
    np.testing.assert_allclose(Sb, S @ b.double().numpy(), atol=1e-12)
    np.testing.assert_allclose(oracle.sketch_vec(b, m, seed=23), Sb, atol=0)


def test_ragged_and_empty_rows():
    A = W.csr_random_lengths(500, 12, 0, 12, seed=8, empty_frac=0.3)
    S = oracle.dense_S(seed=2, m=40, n=A.n)
    SA, _ = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, None, 40, seed=2)
    np.testing.assert_allclose(SA, S @ A.to_dense().numpy(), atol=1e-12)


def test_column_sums_and_shards():
    n, d, m, seed = 5000, 24, 333, 41
    A = _csr(n, d, 6, seed=1)
    b, _ = W.rhs(A, 0.1, seed=2)
    SA, Sb = oracle.sketch_csr(A.row_ptr, A.col, A.val, d, b, m, seed)
    _, sign = oracle.hash(seed, m, 0, n)
    Ad = A.to_dense().numpy()
    np.testing.assert_allclose(SA.sum(axis=0), (sign[:, None] * Ad).sum(axis=0), atol=1e-9)
    np.testing.assert_allclose(Sb.sum(), float((sign * b.double().numpy()).sum()), atol=1e-9)
    # a row shard hashes with its global row indices; shards sum to the whole
    a = 1777
    P1 = oracle.sketch_csr(*A.rows(0, a).numpy(), d, b[:a], m, seed, i0=0)
    P2 = oracle.sketch_csr(*A.rows(a, n).numpy(), d, b[a:], m, seed, i0=a)
    np.testing.assert_allclose(P1[0] + P2[0], SA, atol=1e-12)
    np.testing.assert_allclose(P1[1] + P2[1], Sb, atol=1e-12)


def test_norm_moments_over_seeds():
    """E||Sx||^2 = ||x||^2 and Var||Sx||^2 = (2/m)(||x||_2^4 - ||x||_4^4)."""
    rng = np.random.default_rng(0)
    n, m, seeds = 300, 16, 6000
    x = rng.standard_normal(n).astype(np.float32)
    xd = x.astype(np.float64)
    n2 = float((xd ** 2).sum())
    n4 = float((xd ** 4).sum())
    vals = np.array([float((oracle.sketch_vec(x, m, s) ** 2).sum()) for s in range(seeds)])
    var_theory = 2.0 / m * (n2 ** 2 - n4)
    # mean: CLT band
    assert abs(vals.mean() - n2) < 5 * np.sqrt(var_theory / seeds)
    # variance: relative band (the sample variance of this heavy-ish tail has rel sd ~0.05 here)
    assert abs(vals.var() / var_theory - 1.0) < 0.2
    # and the paper's (looser) bound Var <= (6/t) ||x||^4 holds
    assert vals.var() <= 6.0 / m * n2 ** 2


def test_frobenius_expectation_matrix():
    # E ||SA||_F^2 = ||A||_F^2 over seeds (proof of Lemma "len fixed sparse")
    A = _csr(400, 6, 3, seed=9)
    fro = float((A.val.double() ** 2).sum())
    vals = []
    for s in range(1500):
        SA, _ = oracle.sketch_csr(A.row_ptr, A.col, A.val, 6, None, 32, s)
        vals.append(float((SA ** 2).sum()))
    vals = np.array(vals)
    assert abs(vals.mean() / fro - 1) < 5 * vals.std() / np.sqrt(len(vals)) / fro


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_all_core_variant_equals_the_plain_loop_bitwise(threads):
    # the all-core variant sums each bucket's rows in the same ascending order
    # as the plain row loop, so its float64 results are identical
    A = W.csr_random_lengths(30001, 24, 0, 20, seed=41, empty_frac=0.1)
    b = torch.randn(A.n, generator=torch.Generator().manual_seed(42))
    for m, seed in ((1000, 3), (7, 5), (65536, 1)):
        SA, Sb = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, m, seed, i0=17)
        SAp, Sbp = oracle.sketch_csr_parallel(A.row_ptr, A.col, A.val, A.d, b, m, seed, i0=17, threads=threads)
        np.testing.assert_array_equal(SA, SAp)
        np.testing.assert_array_equal(Sb, Sbp)
