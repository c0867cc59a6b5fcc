"""Pins for the oracle's generalized sparse embedding (paper Section
"Generalized Sparse Embedding Matrices", "The construction"; Theorem
"general" for the inner sketches B^(i)).

* Two independent forms agree: the row loop of the C core equals the
  explicit matrix built as the paper writes it, block-diagonal(B^(1..q)) times
  the permutation P that groups the rows by h, on tiny inputs.
* Structure of that matrix: each column has kappa entries of magnitude
  1 / sqrt(kappa), all inside the v * kappa rows of block h(i), one in each of
  the kappa v-row segments, where h is the Section 2 map of the seed over q
  buckets (checked against the arbitrary-precision hash).
* The seeds of the inner sketches come from a SplitMix64 stream written out
  separately in Python.
* Special case: q = 1, kappa = 1 is the sparse embedding of Section 2 with v
  rows and the first inner seed.
* E ||S x||^2 = ||x||^2 over seeds, and ||S x||^2 concentrates more tightly
  with kappa (Theorem "general": kappa stacked sketches scaled by
  1 / sqrt(kappa)); the subspace embedding holds on a d-dimensional column
  space once q * v is large (Theorem on generalized embeddings).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import hash_bigint as HB


def _after_coeffs_py(seed, count):
    accepted, out = 0, []
    for z in HB.splitmix64_stream(seed):
        if accepted < 8:
            if (z & HB.P61) != HB.P61:
                accepted += 1
            continue
        out.append(z)
        if len(out) == count:
            return out


@pytest.mark.parametrize("seed,count", [(0, 5), (1, 1), (2**64 - 1, 3), (123456789, 16)])
def test_inner_seeds_follow_the_stream(seed, count):
    assert oracle.general_seeds(seed, count) == _after_coeffs_py(seed, count)


@pytest.mark.parametrize("n,d,k,q,v,kappa,seed", [
    (40, 5, 2, 3, 4, 2, 7), (97, 6, 3, 5, 3, 4, 1), (64, 4, 1, 1, 8, 3, 11),
    (31, 7, 4, 7, 2, 1, 3), (0, 3, 1, 2, 2, 2, 5)])
def test_row_loop_equals_block_diagonal_times_permutation(n, d, k, q, v, kappa, seed):
    if n:
        A = W.csr_uniform(n, d, k, seed=n + 3)
        b, _ = W.rhs(A, 0.2, seed=9)
        Ad, bd = A.to_dense().numpy(), b.double().numpy()
        rp, c, vals = A.row_ptr, A.col, A.val
    else:
        Ad, bd = np.zeros((0, d)), np.zeros(0, np.float32)
        rp, c, vals = np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)
    S = oracle.dense_S_general(seed, q, v, kappa, n)
    assert S.shape == (q * v * kappa, n)
    SA, Sb = oracle.sketch_csr_general(rp, c, vals, d, bd.astype(np.float32), q, v, kappa, seed)
    np.testing.assert_allclose(SA, S @ Ad, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Sb, S @ bd, rtol=0, atol=1e-12)


@pytest.mark.parametrize("q,v,kappa,seed", [(4, 5, 3, 2), (1, 6, 2, 9), (9, 2, 5, 4)])
def test_matrix_structure(q, v, kappa, seed):
    n = 60
    S = oracle.dense_S_general(seed, q, v, kappa, n)
    h, _ = HB.hash_rows(seed, q, range(n))
    seeds = _after_coeffs_py(seed, kappa)
    w = 1.0 / np.sqrt(kappa)
    for i in range(n):
        nz = np.nonzero(S[:, i])[0]
        assert len(nz) == kappa
        np.testing.assert_allclose(np.abs(S[nz, i]), w, rtol=1e-15)
        for bidx in range(kappa):
            hb, sb = HB.bucket_sign(seeds[bidx], v, i)
            r = h[i] * v * kappa + bidx * v + hb
            assert S[r, i] == pytest.approx(sb * w, rel=1e-15)


def test_q1_kappa1_is_the_section2_sketch():
    A = W.csr_uniform(3000, 9, 4, seed=5)
    b, _ = W.rhs(A, 0.3, seed=6)
    seed, v = 77, 40
    s0 = oracle.general_seeds(seed, 1)[0]
    SA, Sb = oracle.sketch_csr_general(A.row_ptr, A.col, A.val, 9, b, 1, v, 1, seed)
    SA0, Sb0 = oracle.sketch_csr(A.row_ptr, A.col, A.val, 9, b, v, s0)
    np.testing.assert_array_equal(SA, SA0)
    np.testing.assert_array_equal(Sb, Sb0)


def test_norm_expectation_and_concentration():
    rng = np.random.default_rng(3)
    n, q, v = 200, 2, 6
    x = rng.standard_normal(n).astype(np.float32)
    n2 = float((x.astype(np.float64) ** 2).sum())
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.zeros(n, np.int32)
    spread = []
    for kappa in (1, 8):
        vals = np.array([float((oracle.sketch_csr_general(rp, col, x, 1, None, q, v, kappa, s)[0] ** 2).sum())
                         for s in range(1500)])
        assert abs(vals.mean() - n2) < 5 * vals.std() / np.sqrt(len(vals))
        spread.append(vals.std())
    # kappa independent sketches averaged: the spread falls by about sqrt(kappa)
    assert spread[1] < 0.6 * spread[0]


def test_subspace_embedding_on_a_column_space():
    n, d = 20000, 6
    A = W.dense_gaussian(n, d, seed=12).double().numpy()
    Q, _ = np.linalg.qr(A)
    rp = np.arange(0, n * d + 1, d, dtype=np.int32)
    col = np.tile(np.arange(d, dtype=np.int32), n)
    SQ, _ = oracle.sketch_csr_general(rp, col, Q.astype(np.float32).ravel(), d, None, 64, 16, 4, 21)
    sv = np.linalg.svd(SQ, compute_uv=False)
    assert 0.8 < sv.min() and sv.max() < 1.2
