"""GPU parity of the map (h, sigma) and of SA / Sb against the float64 oracle.

Hash rows and signs must match bit for bit.  Every SA / Sb entry must agree
with the oracle within 1e-5 of its bucket's absolute sum (sum over the rows i in
the bucket of |A_ij|), the float32 tolerance of the sparse-embedding kernels.
Sizes span several 8192-row tiles with ragged tails; the edge cases are empty
and ragged rows, n < m, m = 1, m not a power of two, wide rows, groups larger
than one shared-memory chunk, and bitwise reproducibility.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


def _abs_bucket_sums(h, rows_abs, m):
    """Sum over rows i with h(i) = j of |row_i| (rows_abs: n x d float64)."""
    out = np.zeros((m,) + rows_abs.shape[1:])
    np.add.at(out, h, rows_abs)
    return out


def _check_sa(SA, SA_o, absum, what):
    SA = SA.detach().cpu().double().numpy()
    err = np.abs(SA - SA_o)
    bound = TOL * absum + 1e-30
    bad = err > bound
    assert not bad.any(), "%s: %d entries out of tolerance, worst err %.3g vs bound %.3g" % (
        what, int(bad.sum()), float(err[bad].max()), float(bound[bad].min()))


def _csr_abs_sums(A, h, m):
    rp, c, v = A.numpy()
    out = np.zeros((m, A.d))
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    np.add.at(out, (h[rows], c), np.abs(v.astype(np.float64)))
    return out


@pytest.mark.parametrize("seed,m,i0,count", [
    (1, 4096, 0, 100000), (7, 65536, 2**31 - 50000, 70001), (3, 1000003, 12345, 33333),
    (2**64 - 1, 1, 0, 5000), (99, 3, 2**40 + 7, 40000)])
def test_hash_bit_exact(cw, seed, m, i0, count):
    bucket, sign = cw.cw_hash(seed, m, i0, count)
    h_o, s_o = oracle.hash(seed, m, i0, count)
    np.testing.assert_array_equal(bucket.cpu().numpy(), h_o)
    np.testing.assert_array_equal(sign.cpu().numpy(), s_o)


def _run_csr(cw, A, b, m, seed, check_b=True):
    Ag = A.to("cuda")
    bg = b.cuda() if b is not None else None
    SA, Sb = cw.cw_sketch_csr(Ag, bg, m, seed)
    cw.device_status()
    SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, m, seed)
    h, _ = oracle.hash(seed, m, 0, A.n)
    _check_sa(SA, SA_o, _csr_abs_sums(A, h, m), "SA")
    if b is not None and check_b:
        absb = _abs_bucket_sums(h, np.abs(b.double().numpy()), m)
        _check_sa(Sb, Sb_o, absb, "Sb")
    return SA, Sb


def test_sketch_csr_tiny_regression_config(cw):
    # n = 65536, d = 32, 8 uniform distinct columns per row, m = 4096, seed 1
    A = W.csr_uniform(65536, 32, 8, seed=1001)
    b, _ = W.rhs(A, 0.1, seed=2001)
    _run_csr(cw, A, b, 4096, 1)


@pytest.mark.parametrize("n,d,k,m,seed", [
    (50001, 256, 16, 1024, 5),     # Zipf-like width, ragged last tile
    (8191, 17, 5, 1000, 2),        # m not a power of two, n < one tile
    (300, 8, 3, 4096, 9),          # n < m: most buckets empty
    (20000, 12, 4, 1, 4),          # a single bucket: many chunks
    (200000, 9, 2, 3, 8),          # three huge buckets
    (70000, 64, 33, 777, 6),       # rows longer than 16 and 32 lanes
])
def test_sketch_csr_shapes(cw, n, d, k, m, seed):
    A = W.csr_uniform(n, d, k, seed=seed + 10)
    b, _ = W.rhs(A, 0.5, seed=seed + 20)
    _run_csr(cw, A, b, m, seed)


def test_sketch_csr_ragged_empty_rows_no_b(cw):
    A = W.csr_random_lengths(30000, 40, 0, 30, seed=3, empty_frac=0.25)
    SA, Sb = _run_csr(cw, A, None, 2048, 11)
    assert Sb is None


def test_sketch_csr_wide_rows_global_accumulator(cw):
    A = W.csr_random_lengths(3000, 5000, 10, 80, seed=4)
    b, _ = W.rhs(A, 0.5, seed=5)
    _run_csr(cw, A, b, 64, 12)


def test_sketch_csr_zipf_columns(cw):
    A = W.csr_zipf(100000, 256, 16, 1.1, seed=1002)
    b, _ = W.rhs(A, 0.01, seed=2002)
    _run_csr(cw, A, b, 8192, 1)


def test_sketch_csr_deterministic(cw):
    A = W.csr_zipf(60000, 128, 16, 1.1, seed=77).to("cuda")
    b = torch.randn(A.n, device="cuda")
    SA1, Sb1 = cw.cw_sketch_csr(A, b, 2048, 5)
    SA2, Sb2 = cw.cw_sketch_csr(A, b, 2048, 5)
    assert torch.equal(SA1, SA2) and torch.equal(Sb1, Sb2)


def test_sketch_csr_row_shards_add_up(cw):
    A = W.csr_uniform(40000, 24, 6, seed=31)
    b, _ = W.rhs(A, 0.1, seed=32)
    m, seed, a = 1500, 3, 17777
    SA, Sb = cw.cw_sketch_csr(A.to("cuda"), b.cuda(), m, seed)
    P1 = cw.cw_sketch_csr_rows(A.rows(0, a).to("cuda"), 0, b[:a].cuda(), m, seed)
    P2 = cw.cw_sketch_csr_rows(A.rows(a, A.n).to("cuda"), a, b[a:].cuda(), m, seed)
    h, _ = oracle.hash(seed, m, 0, A.n)
    _check_sa(P1[0] + P2[0], SA.cpu().double().numpy(), 2 * _csr_abs_sums(A, h, m), "shards SA")
    SA_o, Sb_o = oracle.sketch_csr(A.rows(a, A.n).row_ptr, A.rows(a, A.n).col, A.rows(a, A.n).val, A.d,
                                   b[a:], m, seed, i0=a)
    h2 = h[a:]
    _check_sa(P2[0], SA_o, _csr_abs_sums(A.rows(a, A.n), h2, m), "shard 2 SA")


def test_sketch_csr_empty_matrix(cw):
    A = W.csr_uniform(0, 5, 0, seed=1).to("cuda")
    SA = torch.full((10, 5), 7.0, device="cuda")
    cw.cw_sketch_csr(A, None, 10, 1, SA=SA)
    assert float(SA.abs().max()) == 0.0


def test_sketch_csr_flags_bad_column(cw):
    A = W.csr_uniform(1000, 10, 3, seed=2)
    A.col[5] = 10  # out of range [0, d)
    cw.cw_sketch_csr(A.to("cuda"), None, 64, 1)
    with pytest.raises(cw.CWError):
        cw.device_status()
    cw.device_status()  # flag is cleared


def test_csr_check_finds_every_violation(cw):
    good = W.csr_random_lengths(5000, 40, 0, 40, seed=2, empty_frac=0.1)
    cw.cw_csr_check(good.to("cuda"))
    dup = W.csr_uniform(1000, 10, 3, seed=2)
    dup.col[1] = dup.col[0]
    bad_col = W.csr_uniform(1000, 10, 3, seed=2)
    bad_col.col[7] = -1
    bad_ptr = W.csr_uniform(1000, 10, 3, seed=2)
    bad_ptr.row_ptr[5] = bad_ptr.row_ptr[6] + 1
    long_dup = W.csr_random_lengths(50, 100, 70, 80, seed=3)
    long_dup.col[int(long_dup.row_ptr[3]) + 65] = long_dup.col[int(long_dup.row_ptr[3]) + 2]
    for A in (dup, bad_col, bad_ptr, long_dup):
        with pytest.raises(cw.CWError):
            cw.cw_csr_check(A.to("cuda"))


@pytest.mark.parametrize("n,d,lda,m,seed", [
    (65536, 512, 512, 4096, 1), (30001, 100, 100, 999, 2), (10000, 33, 40, 256, 3),
    (5000, 1500, 1500, 128, 4), (100, 7, 7, 1000, 5), (40000, 4, 4, 1, 6)])
def test_sketch_dense(cw, n, d, lda, m, seed):
    A = W.dense_gaussian(n, lda, seed=seed)
    b = W.dense_gaussian(n, 1, seed=seed + 1)[:, 0].contiguous()
    Ag = A.cuda()
    SA, Sb = cw.cw_sketch_dense(Ag[:, :d], b.cuda(), m, seed, lda=lda) if lda != d else \
        cw.cw_sketch_dense(Ag, b.cuda(), m, seed)
    cw.device_status()
    SA_o, Sb_o = oracle.sketch_dense(A[:, :d].contiguous(), b, m, seed)
    h, _ = oracle.hash(seed, m, 0, n)
    _check_sa(SA, SA_o, _abs_bucket_sums(h, np.abs(A[:, :d].double().numpy()), m), "dense SA")
    _check_sa(Sb, Sb_o, _abs_bucket_sums(h, np.abs(b.double().numpy()), m), "dense Sb")


def test_sketch_vec(cw):
    x = W.dense_gaussian(123457, 1, seed=9)[:, 0].contiguous()
    for m, seed in ((4096, 1), (65536, 2), (7, 3)):
        Sx = cw.cw_sketch_vec(x.cuda(), m, seed)
        Sx_o = oracle.sketch_vec(x, m, seed)
        h, _ = oracle.hash(seed, m, 0, x.numel())
        _check_sa(Sx, Sx_o, _abs_bucket_sums(h, np.abs(x.double().numpy()), m), "Sx")


def test_sketch_csr_full_size_large_sparse_config(cw):
    """n = 2^24, d = 256, 16 Zipf(1.1) columns per row, m = 65536: every entry vs the oracle."""
    n, d, m, seed = 1 << 24, 256, 65536, 1
    A = W.csr_zipf(n, d, 16, 1.1, seed=1002, device="cuda")
    b, _ = W.rhs(A, 0.01, seed=2002)
    SA, Sb = cw.cw_sketch_csr(A, b, m, seed)
    cw.device_status()
    rp, c, v = A.numpy()
    bh = b.cpu()
    SA_o, Sb_o = oracle.sketch_csr(rp, c, v, d, bh, m, seed)
    h, _ = oracle.hash(seed, m, 0, n)
    absA = np.zeros((m, d))
    rows = np.repeat(h, 16)
    np.add.at(absA, (rows, c), np.abs(v.astype(np.float64)))
    _check_sa(SA, SA_o, absA, "C2 SA")
    _check_sa(Sb, Sb_o, _abs_bucket_sums(h, np.abs(bh.double().numpy()), m), "C2 Sb")
