"""GPU parity of the downstream steps against the float64 oracle.

* cw_qr: R (positive diagonal) and c = Q^T Sb of the library's own SA equal the
  oracle's Householder QR of the same matrix to float64 accuracy.
* cw_solve_sketch: the residual ratio rho = ||Ax'-b|| / ||Ax*-b|| of the
  library's x' equals the oracle's (same S, float64 sketch) within 1e-6.
* cw_lsqr_precond: both converge under the same stopping test, iteration
  counts agree within one, and the residual ratios agree within 1e-6.
* cw_leverage: each score within 1e-3 (relative) of the same algorithm run by
  the oracle in float64 (same S, same G), on an A with condition number 1e6;
  the exact scores ||Q_i||^2 bound the estimates within the constant factor
  of Theorem "icml".
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-6


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


def _rho(A, b, x, rn):
    return oracle.residual_ratio_csr(A.row_ptr, A.col, A.val, b, x, rn)


# blocked kernel: one panel, several panels with a ragged last one, d = 1,
# d = 33, d = m; unblocked fallback: 131075 rows do not fit one CTA's panel rows
# in shared memory
@pytest.mark.parametrize("m,d", [(4096, 32), (1000, 17), (300, 300), (20000, 100), (5000, 1), (70001, 33),
                                 (131075, 40)])
def test_qr_matches_oracle_on_same_matrix(cw, m, d):
    SA = W.dense_gaussian(m, d, seed=m + d)
    SA[:, 0] *= 1e3  # uneven column scales
    Sb = W.dense_gaussian(m, 1, seed=7)[:, 0].contiguous()
    R, c = cw.cw_qr(SA.cuda(), Sb.cuda())
    R_o, c_o = oracle.qr_r(SA.double().numpy(), Sb.double().numpy())
    np.testing.assert_allclose(R.cpu().numpy(), R_o, rtol=1e-10, atol=1e-11 * np.abs(R_o).max())
    np.testing.assert_allclose(c.cpu().numpy(), c_o, rtol=1e-9, atol=1e-11 * np.abs(c_o).max())


def test_qr_rank_deficient_is_reported(cw):
    SA = W.dense_gaussian(500, 8, seed=3).cuda()
    SA[:, 5] = 0.0
    with pytest.raises(cw.CWError) as e:
        cw.cw_qr(SA)
    assert e.value.status == -5


def test_solve_sketch_tiny_regression_config(cw):
    # n = 65536, d = 32, 8 uniform distinct columns, m = 4096, seed 1
    n, d, m, seed = 65536, 32, 4096, 1
    A = W.csr_uniform(n, d, 8, seed=1001)
    b, _ = W.rhs(A, 0.1, seed=2001)
    x = cw.cw_solve_sketch(A.to("cuda"), b.cuda(), m, seed).cpu().numpy()
    SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, d, b, m, seed)
    x_o, _ = oracle.solve_sketch(SA_o, Sb_o)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, d, b)
    rho, rho_o = _rho(A, b, x, rn), _rho(A, b, x_o, rn)
    assert abs(rho - rho_o) <= RHO_TOL, (rho, rho_o)
    assert 1.0 <= rho < 1.05


@pytest.mark.parametrize("n,d,k,m,seed", [(30001, 10, 4, 640, 3), (5000, 48, 12, 2304, 4), (100000, 5, 3, 97, 5)])
def test_solve_sketch_shapes(cw, n, d, k, m, seed):
    A = W.csr_uniform(n, d, k, seed=seed)
    b, _ = W.rhs(A, 0.2, seed=seed + 1)
    x, R = cw.cw_solve_sketch(A.to("cuda"), b.cuda(), m, seed, want_R=True)
    SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, d, b, m, seed)
    x_o, R_o = oracle.solve_sketch(SA_o, Sb_o)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, d, b)
    assert abs(_rho(A, b, x.cpu().numpy(), rn) - _rho(A, b, x_o, rn)) <= RHO_TOL
    np.testing.assert_allclose(R.cpu().numpy(), R_o, rtol=1e-4, atol=1e-5 * np.abs(R_o).max())


def test_solve_sketch_dense(cw):
    n, d, m = 40000, 24, 1024
    A = W.dense_lowrank(n, d, W.geometric_sigma(d, 1e-2), seed=11)
    b, _ = W.rhs(A, 0.05, seed=12)
    x = cw.cw_solve_sketch_dense(A.cuda(), b.cuda(), m, 9).cpu().numpy()
    SA_o, Sb_o = oracle.sketch_dense(A, b, m, 9)
    x_o, _ = oracle.solve_sketch(SA_o, Sb_o)
    Ad, bd = A.double().numpy(), b.double().numpy()
    xs = np.linalg.lstsq(Ad, bd, rcond=None)[0]
    rn = np.linalg.norm(Ad @ xs - bd)
    rho = np.linalg.norm(Ad @ x - bd) / rn
    rho_o = np.linalg.norm(Ad @ x_o - bd) / rn
    assert abs(rho - rho_o) <= RHO_TOL


def _lsqr_case(cw, A, b, m, seed, rtol=1e-6):
    x, it, test = cw.cw_lsqr_precond(A.to("cuda") if A.device.type == "cpu" else A,
                                     b.cuda() if b.device.type == "cpu" else b, m, seed, rtol=rtol, max_iter=100)
    rp, c, v = A.numpy()
    bh = b.cpu()
    SA_o, Sb_o = oracle.sketch_csr(rp, c, v, A.d, bh, m, seed)
    x0_o, R_o = oracle.solve_sketch(SA_o, Sb_o)
    x_o, it_o, test_o, conv_o, _ = oracle.lsqr_precond_csr(rp, c, v, A.d, bh, R_o, x0_o, rtol, 100)
    return x.cpu().numpy(), it, test, x_o, it_o, test_o, conv_o


def test_lsqr_matches_oracle_small(cw):
    n, d, m, seed = 1 << 18, 64, 4096, 1
    A = W.csr_zipf(n, d, 16, 1.1, seed=1002)
    b, _ = W.rhs(A, 0.01, seed=2002)
    x, it, test, x_o, it_o, test_o, conv_o = _lsqr_case(cw, A, b, m, seed)
    assert conv_o and test <= 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    xs, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, d, b)
    assert abs(_rho(A, b, x, rn) - _rho(A, b, x_o, rn)) <= RHO_TOL
    np.testing.assert_allclose(x, xs, rtol=1e-5, atol=1e-6 * np.abs(xs).max())


def test_lsqr_ragged_rows(cw):
    A = W.csr_random_lengths(120000, 40, 2, 30, seed=5, empty_frac=0.05)
    b, _ = W.rhs(A, 0.1, seed=6)
    x, it, test, x_o, it_o, test_o, conv_o = _lsqr_case(cw, A, b, 1600, 3)
    assert abs(it - it_o) <= 1
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    assert abs(_rho(A, b, x, rn) - _rho(A, b, x_o, rn)) <= RHO_TOL


@pytest.mark.parametrize("n,d,k,m,seed", [
    (150000, 300, 8, 4096, 7),    # one-CTA Cholesky, last panel 12 columns wide
    (80000, 400, 6, 8192, 8),     # packed triangle too large for one CTA: panel kernels
    (30000, 1, 1, 64, 9),         # a single column
    (50000, 33, 5, 512, 10),      # two panels, the second one column wide
    (60000, 150, 6, 2048, 11)])   # tensor-core Gram with two accumulator blocks, element loads
def test_lsqr_shapes(cw, n, d, k, m, seed):
    A = W.csr_uniform(n, d, k, seed=seed + 40)
    b, _ = W.rhs(A, 0.1, seed=seed + 50)
    x, it, test, x_o, it_o, test_o, conv_o = _lsqr_case(cw, A, b, m, seed)
    assert conv_o and test <= 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    assert abs(_rho(A, b, x, rn) - _rho(A, b, x_o, rn)) <= RHO_TOL


def test_lsqr_badly_scaled_columns_take_the_qr_preconditioner(cw):
    """Columns scaled over four decades: R's diagonal ratio is far above the
    Cholesky route's limit of 300, so the library redoes the iterations from
    the float64 QR preconditioner; the result still matches the oracle."""
    A0 = W.csr_uniform(60000, 48, 6, seed=71)
    scale = torch.pow(10.0, torch.linspace(0, 4, 48, dtype=torch.float64)).to(torch.float32)
    A = W.CSR(A0.n, A0.d, A0.row_ptr, A0.col, A0.val * scale[A0.col.long()])
    b, _ = W.rhs(A, 0.1, seed=72)
    x, it, test, x_o, it_o, test_o, conv_o = _lsqr_case(cw, A, b, 2048, 13)
    assert conv_o and test <= 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    assert abs(_rho(A, b, x, rn) - _rho(A, b, x_o, rn)) <= RHO_TOL


def test_lsqr_is_deterministic(cw):
    """Every sum in the sketch, the preconditioner and the LSQR steps has a
    fixed order: two runs give the same bits."""
    A = W.csr_zipf(1 << 18, 200, 12, 1.1, seed=81, device="cuda")
    b, _ = W.rhs(A, 0.05, seed=82)
    x1, it1, t1 = cw.cw_lsqr_precond(A, b, 8192, 5)
    x2, it2, t2 = cw.cw_lsqr_precond(A, b, 8192, 5)
    assert it1 == it2 and t1 == t2
    assert torch.equal(x1, x2)


def test_lsqr_zero_iterations(cw):
    A = W.csr_uniform(20000, 16, 4, seed=2)
    b, _ = W.rhs(A, 0.5, seed=3)
    x, it, test = cw.cw_lsqr_precond(A.to("cuda"), b.cuda(), 64, 1, rtol=1e-6, max_iter=0, allow_noconv=True)
    assert it == 0
    x_s = cw.cw_solve_sketch(A.to("cuda"), b.cuda(), 64, 1)
    # no iteration: x is the sketch-and-solve start (Cholesky or QR route, float32 R^-1)
    np.testing.assert_allclose(x.cpu().numpy(), x_s.cpu().numpy(), rtol=1e-4, atol=1e-5)


def test_lsqr_max_iter_reports_noconv(cw):
    A = W.csr_uniform(20000, 16, 4, seed=2)
    b, _ = W.rhs(A, 0.5, seed=3)
    x, it, test = cw.cw_lsqr_precond(A.to("cuda"), b.cuda(), 64, 1, rtol=1e-14, max_iter=2, allow_noconv=True)
    assert it == 2 and test > 1e-14


def test_lsqr_full_size_large_sparse_config(cw):
    """n = 2^24, d = 256, 16 Zipf(1.1) columns per row, m = 65536, rtol 1e-6."""
    n, d, m, seed = 1 << 24, 256, 65536, 1
    A = W.csr_zipf(n, d, 16, 1.1, seed=1002, device="cuda")
    b, _ = W.rhs(A, 0.01, seed=2002)
    x, it, test, x_o, it_o, test_o, conv_o = _lsqr_case(cw, A, b, m, seed)
    assert conv_o and test <= 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    rp, c, v = A.numpy()
    bh = b.cpu()
    # exact optimum by the oracle's own LSQR run to 1e-13 (its preconditioned operator is near-orthonormal)
    SA_o, Sb_o = oracle.sketch_csr(rp, c, v, d, bh, m, seed)
    x0_o, R_o = oracle.solve_sketch(SA_o, Sb_o)
    xs, _, _, conv_s, _ = oracle.lsqr_precond_csr(rp, c, v, d, bh, R_o, x0_o, 1e-13, 200)
    rn = oracle.residual_norm_csr(rp, c, v, bh, xs)
    rho = oracle.residual_norm_csr(rp, c, v, bh, x) / rn
    rho_o = oracle.residual_norm_csr(rp, c, v, bh, x_o) / rn
    assert abs(rho - rho_o) <= RHO_TOL and rho >= 1 - 1e-12


def _lev_case(cw, n, d, m, k, kappa, seed):
    A = W.dense_lowrank(n, d, W.geometric_sigma(d, 1.0 / kappa), seed=seed)
    G = W.gaussian(d, k, seed=seed + 1)
    lev = cw.cw_leverage(A.cuda(), m, 1, G.cuda()).cpu().double().numpy()
    SA_o, _ = oracle.sketch_dense(A, None, m, 1)
    R_o, _ = oracle.qr_r(SA_o)
    lev_o = oracle.leverage_same(A, R_o, G.numpy())
    return A, lev, lev_o


def test_leverage_matches_same_algorithm_ill_conditioned(cw):
    A, lev, lev_o = _lev_case(cw, 1 << 16, 64, 4096, 32, 1e6, seed=21)
    rel = np.abs(lev - lev_o) / lev_o
    assert rel.max() <= 1e-3, rel.max()
    # Theorem "icml": constant-factor estimates.  sum(lev)/d is a JL estimate of
    # ||A R^-1||_F^2 / d with relative sd ~ sqrt(2/(k d)) ~ 3% plus the embedding
    # distortion, so the band is a few sd wide.
    u = oracle.leverage_exact(A)
    assert abs(lev.sum() / 64 - 1) < 0.15
    assert 0.8 < np.median(lev / u) < 1.25


def test_leverage_at_the_dense_workload_shape(cw):
    # the dense leverage workload's d, m, k and kappa (d = 512: eight 64-column
    # chunks of the tensor-core product; a 65536 x 512 sketch: sixteen panels of
    # the blocked float64 QR), on 2^17 rows instead of 2^22
    A, lev, lev_o = _lev_case(cw, 1 << 17, 512, 65536, 32, 1e6, seed=23)
    rel = np.abs(lev - lev_o) / lev_o
    assert rel.max() <= 1e-3, rel.max()


@pytest.mark.parametrize("n,d,m,k", [(20001, 100, 1024, 32), (5000, 33, 700, 7), (3000, 520, 2048, 40),
                                     (30001, 200, 2048, 32), (10000, 128, 1024, 7)])
def test_leverage_shapes(cw, n, d, m, k):
    _, lev, lev_o = _lev_case(cw, n, d, m, k, 1e3, seed=n % 97)
    rel = np.abs(lev - lev_o) / lev_o
    assert rel.max() <= 1e-3, rel.max()


def test_leverage_tensor_core_path_runs(cw):
    """k <= 32 with 16-byte aligned rows takes the tcgen05 kernel; other shapes the CUDA-core one."""
    cw.profile_reset()
    cw.profile_enable(True)
    try:
        _lev_case(cw, 4097, 96, 1024, 32, 10.0, seed=5)
        n_tc = cw.profile_get("k_leverage_tc")[0]
        _lev_case(cw, 4097, 33, 1024, 32, 10.0, seed=5)
        n_cc = cw.profile_get("k_leverage")[0]
    finally:
        cw.profile_enable(False)
    assert n_tc == 1 and n_cc == 1
