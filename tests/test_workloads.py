"""The seeded input generators against their recipes (host logic, CPU).

* fixed-k CSR: exactly k distinct, sorted columns per row in [0, d); with k = 1
  the column frequencies follow p (the exponential-key draw without
  replacement reduces to a draw from p); with Zipf(1.1) over 256 columns and
  k = 16 the inclusion frequencies fall with the column index;
* values N(0,1); b - A x0 is noise * N(0,1);
* ragged rows: lengths in [kmin, kmax] or empty at the requested rate;
* A = U diag(sigma) V^T has the singular values sigma (float32 storage);
* the same seed gives the same data, another seed other data.
"""
import numpy as np
import torch

import workloads as W


def _rows(A):
    rp, col, val = A.numpy()
    return rp, col, val


def test_fixed_k_rows_are_distinct_sorted_in_range():
    for A in (W.csr_uniform(5000, 40, 7, seed=1), W.csr_zipf(5000, 256, 16, 1.1, seed=2)):
        rp, col, _ = _rows(A)
        k = A.nnz // A.n
        np.testing.assert_array_equal(rp, np.arange(A.n + 1) * k)
        C = col.reshape(A.n, k)
        assert (C >= 0).all() and (C < A.d).all()
        assert (np.diff(C, axis=1) > 0).all()   # sorted, hence distinct


def test_single_draw_follows_the_column_distribution():
    n, d = 200000, 256
    p = W.zipf_probs(d, 1.1).numpy()
    assert abs(p[0] - 0.21) < 0.01             # the recipe's column-1 probability
    A = W.csr_zipf(n, d, 1, 1.1, seed=3)
    freq = np.bincount(A.col.numpy(), minlength=d) / n
    sd = np.sqrt(p * (1 - p) / n)
    assert (np.abs(freq - p) <= 5 * sd + 1e-12).all()


def test_zipf_inclusion_falls_with_the_column_index():
    n, d, k = 100000, 256, 16
    A = W.csr_zipf(n, d, k, 1.1, seed=4)
    inc = np.bincount(A.col.numpy(), minlength=d) / n
    assert abs(inc.sum() - k) < 1e-9
    # smoothed over blocks of 16 columns, strictly decreasing
    blocks = inc.reshape(-1, 16).mean(axis=1)
    assert (np.diff(blocks) < 0).all()
    assert inc[0] > 0.9 and inc[-16:].mean() < 0.05


def test_values_and_rhs_noise():
    A = W.csr_uniform(50000, 24, 6, seed=5)
    v = A.val.double().numpy()
    assert abs(v.mean()) < 0.01 and abs(v.var() - 1) < 0.02
    b, x0 = W.rhs(A, 0.25, seed=6)
    r = b.double().numpy() - A.matvec(x0).numpy()
    assert abs(r.std() - 0.25) < 0.005 and abs(r.mean()) < 0.005


def test_ragged_lengths_and_empty_rows():
    n, d = 40000, 30
    A = W.csr_random_lengths(n, d, 2, 9, seed=7, empty_frac=0.1)
    rp, col, _ = _rows(A)
    lens = np.diff(rp)
    assert ((lens == 0) | ((lens >= 2) & (lens <= 9))).all()
    assert abs((lens == 0).mean() - 0.1) < 0.01
    for i in range(0, n, 997):
        c = col[rp[i]:rp[i + 1]]
        assert (np.diff(c) > 0).all() and ((c >= 0) & (c < d)).all()


def test_lowrank_singular_values():
    sigma = W.geometric_sigma(12, 1e-2)
    A = W.dense_lowrank(3000, 12, sigma, seed=8)
    s = np.linalg.svd(A.double().numpy(), compute_uv=False)
    np.testing.assert_allclose(s, sigma.numpy(), rtol=1e-4)


def test_seeds_reproduce_and_differ():
    a1 = W.csr_zipf(1000, 64, 8, 1.1, seed=9)
    a2 = W.csr_zipf(1000, 64, 8, 1.1, seed=9)
    a3 = W.csr_zipf(1000, 64, 8, 1.1, seed=10)
    assert torch.equal(a1.col, a2.col) and torch.equal(a1.val, a2.val)
    assert not torch.equal(a1.col, a3.col)
