"""Pins for the oracle's downstream steps: QR / sketch-and-solve, exact least
squares, preconditioned LSQR and leverage scores.

Each function is checked against an independent route or a property the
mathematics fixes:
* R of SA against the Cholesky factor of SA^T SA (the unique upper factor
  with positive diagonal), plus orthogonality and reconstruction;
* x' against an SVD-based least-squares solve and its normal equations;
* streaming TSQR x* against an SVD solve on the dense matrix, and against
  itself with other block sizes;
* LSQR against SciPy's independent LSQR on the same preconditioned operator,
  the true residual of its iterates, and the paper's contraction bound;
* leverage: sum = rank (paper Section 4, sum of u_i = r), the hat-matrix
  diagonal, and the same-algorithm estimator with an exact R and G = sqrt(d) I.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as W


def _problem(n=4000, d=12, k=4, m=256, seed=1, noise=0.1):
    A = W.csr_uniform(n, d, k, seed)
    b, x0 = W.rhs(A, noise, seed + 100)
    SA, Sb = oracle.sketch_csr(A.row_ptr, A.col, A.val, d, b, m, seed=seed)
    return A, b, SA, Sb


def test_qr_r_is_cholesky_factor_and_orthogonal():
    A, b, SA, Sb = _problem()
    R, c = oracle.qr_r(SA, Sb)
    assert np.allclose(np.tril(R, -1), 0)
    assert (np.diag(R) > 0).all()
    L = np.linalg.cholesky(SA.T @ SA)
    np.testing.assert_allclose(R, L.T, rtol=1e-9, atol=1e-9 * np.abs(R).max())
    # c = Q^T Sb with Q = SA R^-1 orthonormal
    Q = sla.solve_triangular(R, SA.T, lower=False, trans="T").T
    np.testing.assert_allclose(Q.T @ Q, np.eye(R.shape[0]), atol=1e-10)
    np.testing.assert_allclose(c, Q.T @ Sb, atol=1e-9 * np.linalg.norm(Sb))


def test_gram_against_qr_and_brute_force():
    """The Gram matrix pinned two ways: R^T R from the Householder QR (LAPACK,
    another algorithm), with the Sb column R^T c and corner ||Sb||^2, and a
    plain triple loop on a tiny case."""
    A, b, SA, Sb = _problem(d=9, m=96)
    G = oracle.gram(SA, Sb)
    R, c = oracle.qr_r(SA, Sb)
    d = SA.shape[1]
    scale = np.abs(G).max()
    np.testing.assert_allclose(G[:d, :d], R.T @ R, atol=1e-12 * scale)
    np.testing.assert_allclose(G[:d, d], R.T @ c, atol=1e-12 * scale)
    np.testing.assert_allclose(G[d, :d], G[:d, d], rtol=0, atol=0)
    assert abs(G[d, d] - float(np.dot(Sb.astype(np.float64), Sb.astype(np.float64)))) <= 1e-12 * scale
    np.testing.assert_array_equal(oracle.gram(SA), G[:d, :d])
    X = np.random.default_rng(3).standard_normal((5, 3))
    y = np.random.default_rng(4).standard_normal(5)
    Gt = oracle.gram(X, y)
    for i in range(4):
        for j in range(4):
            s = 0.0
            for r in range(5):
                u = X[r, i] if i < 3 else y[r]
                v = X[r, j] if j < 3 else y[r]
                s += u * v
            assert abs(Gt[i, j] - s) <= 1e-12


def test_solve_sketch_matches_svd_lstsq():
    A, b, SA, Sb = _problem()
    x, R = oracle.solve_sketch(SA, Sb)
    x_svd = np.linalg.lstsq(SA, Sb, rcond=None)[0]
    np.testing.assert_allclose(x, x_svd, rtol=1e-10, atol=1e-12)
    g = SA.T @ (SA @ x - Sb)
    assert np.linalg.norm(g) < 1e-9 * np.linalg.norm(SA) ** 2 * np.linalg.norm(x)


def test_exact_lstsq_csr_matches_svd_and_block_size():
    A, b, _, _ = _problem(n=3000, d=10)
    Ad = A.to_dense().numpy()
    bd = b.double().numpy()
    xs, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b, block=512)
    x_svd = np.linalg.lstsq(Ad, bd, rcond=None)[0]
    np.testing.assert_allclose(xs, x_svd, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(rn, np.linalg.norm(Ad @ x_svd - bd), rtol=1e-10)
    xs2, rn2 = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b, block=7)
    np.testing.assert_allclose(xs2, xs, rtol=1e-10, atol=1e-12)
    xd, rnd = oracle.lstsq_exact_dense(Ad.astype(np.float32), b)
    np.testing.assert_allclose(xd, xs, rtol=1e-10, atol=1e-12)


def test_residual_ratio_sketch_and_solve_band():
    # rho = ||Ax'-b|| / ||Ax*-b|| >= 1, and close to 1 for m >> d (Theorem "lin reg")
    A, b, SA, Sb = _problem(n=20000, d=8, m=1024)
    x, _ = oracle.solve_sketch(SA, Sb)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    rho = oracle.residual_ratio_csr(A.row_ptr, A.col, A.val, b, x, rn)
    assert 1.0 <= rho < 1.05


def _scipy_lsqr_same(A, b, R, x0, tol, iters):
    Ad = sp.csr_matrix((A.val.double().numpy(), A.col.numpy(), A.row_ptr.numpy()), shape=(A.n, A.d))
    op = spla.LinearOperator((A.n, A.d),
                             matvec=lambda v: Ad @ sla.solve_triangular(R, v, lower=False),
                             rmatvec=lambda u: sla.solve_triangular(R, Ad.T @ u, lower=False, trans="T"),
                             dtype=np.float64)
    bd = b.double().numpy()
    r0 = bd - Ad @ x0
    out = spla.lsqr(op, r0, atol=0, btol=0, conlim=0, iter_lim=iters)
    return x0 + sla.solve_triangular(R, out[0], lower=False), out


def test_lsqr_matches_scipy_iterates():
    A, b, SA, Sb = _problem(n=6000, d=10, m=128, seed=3)
    x0, R = oracle.solve_sketch(SA, Sb)
    for iters in (1, 2, 3, 5):
        x, it, _, _, _ = oracle.lsqr_precond_csr(A.row_ptr, A.col, A.val, A.d, b, R, x0, rtol=0.0,
                                                 max_iter=iters)
        xs, _ = _scipy_lsqr_same(A, b, R, x0, 0.0, iters)
        assert it == iters
        np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-12)


def test_lsqr_estimates_equal_true_residuals_and_converge():
    A, b, SA, Sb = _problem(n=8000, d=16, m=512, seed=4)
    x0, R = oracle.solve_sketch(SA, Sb)
    xs, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    x, it, test2, conv, hist = oracle.lsqr_precond_csr(A.row_ptr, A.col, A.val, A.d, b, R, x0,
                                                       rtol=1e-10, max_iter=100)
    assert conv and test2 <= 1e-10
    # rnorm estimate = true ||b - A x|| at the returned iterate
    true_r = oracle.residual_norm_csr(A.row_ptr, A.col, A.val, b, x)
    assert abs(hist[-1][0] - true_r) <= 1e-9 * true_r
    # the estimate of ||(AR^-1)^T r|| is the true one
    r = b.double().numpy() - oracle.csr_matvec(A.row_ptr, A.col, A.val, x)
    ar = sla.solve_triangular(R, oracle.csr_rmatvec(A.row_ptr, A.col, A.val, A.d, r), lower=False, trans="T")
    assert abs(np.linalg.norm(ar) - hist[-1][1]) <= 1e-6 * np.linalg.norm(ar) + 1e-12 * true_r
    np.testing.assert_allclose(x, xs, rtol=1e-7, atol=1e-9)
    # rnorm decreases monotonically
    rs = [h[0] for h in hist]
    assert all(rs[i + 1] <= rs[i] * (1 + 1e-12) for i in range(len(rs) - 1))


def test_lsqr_contraction_matches_embedding_quality():
    # Section 7.6: kappa(R^T A^T A R) <= ((1+e0)/(1-e0))^2, so the normal-equation
    # residual contracts fast; measure e0 from the singular values of A R^-1.
    A, b, SA, Sb = _problem(n=20000, d=16, m=2048, seed=6)
    x0, R = oracle.solve_sketch(SA, Sb)
    Ad = A.to_dense().numpy()
    sv = np.linalg.svd(Ad @ np.linalg.inv(R), compute_uv=False)
    e0 = max(sv.max() - 1, 1 - sv.min())
    assert e0 < 0.5
    x, it, test2, conv, hist = oracle.lsqr_precond_csr(A.row_ptr, A.col, A.val, A.d, b, R, x0,
                                                       rtol=1e-6, max_iter=100)
    kappa = (sv.max() / sv.min())
    rate = (kappa - 1) / (kappa + 1)
    # CG bound on the error in the A-norm: ~ 2 rate^k; 1e-6 reached well within
    bound_iters = int(np.ceil(np.log(1e-6 / 2) / np.log(rate))) + 2
    assert conv and it <= bound_iters


def test_lsqr_identity_preconditioner_is_plain_lsqr():
    A, b, _, _ = _problem(n=3000, d=8, seed=7)
    R = np.eye(8)
    x, it, _, _, _ = oracle.lsqr_precond_csr(A.row_ptr, A.col, A.val, 8, b, R, np.zeros(8), 0.0, 4)
    Ad = sp.csr_matrix((A.val.double().numpy(), A.col.numpy(), A.row_ptr.numpy()), shape=(A.n, 8))
    xs = spla.lsqr(Ad, b.double().numpy(), atol=0, btol=0, conlim=0, iter_lim=4)[0]
    np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-12)


def test_leverage_exact_sum_and_hat_matrix():
    A = W.dense_lowrank(3000, 12, W.geometric_sigma(12, 1e-3), seed=5)
    u = oracle.leverage_exact(A)
    assert abs(u.sum() - 12) < 1e-9
    Ad = A.double().numpy()
    hat = np.einsum("ij,ij->i", Ad @ np.linalg.inv(Ad.T @ Ad), Ad)
    np.testing.assert_allclose(u, hat, rtol=1e-6, atol=1e-12)
    assert (u >= 0).all() and (u <= 1 + 1e-12).all()


def test_leverage_same_with_exact_R_identity_G_is_exact():
    A = W.dense_lowrank(2000, 10, W.geometric_sigma(10, 1e-4), seed=6)
    Ad = A.double().numpy()
    R = np.linalg.qr(Ad, mode="r")
    R = np.sign(np.diag(R))[:, None] * R
    G = np.sqrt(10.0) * np.eye(10)
    lev = oracle.leverage_same(A, R, G)
    np.testing.assert_allclose(lev, oracle.leverage_exact(A), rtol=1e-7, atol=1e-14)
    lev_rows = oracle.leverage_same(A, R, G, rows=[0, 17, 1999])
    np.testing.assert_allclose(lev_rows, lev[[0, 17, 1999]], rtol=1e-12)


def test_leverage_sketch_constant_factor():
    # Theorem "icml": u'_i = (1 +- eps) u_i for a subspace embedding and a JL Pi_2
    n, d, m, k = 20000, 8, 4096, 64
    A = W.dense_lowrank(n, d, W.geometric_sigma(d, 1e-2), seed=9)
    SA, _ = oracle.sketch_dense(A, None, m, seed=1)
    R, _ = oracle.qr_r(SA)
    G = W.gaussian(d, k, seed=2).numpy()
    lev = oracle.leverage_same(A, R, G)
    u = oracle.leverage_exact(A)
    ratio = lev / u
    assert 0.85 < np.median(ratio) < 1.15
    assert abs(lev.sum() / d - 1) < 0.1


def test_distortion_reported_in_band():
    A, b, SA, _ = _problem(n=20000, d=8, m=4096, seed=2)
    Ad = A.to_dense().numpy()
    R_A = np.linalg.qr(Ad, mode="r")
    sv = oracle.distortion(SA, R_A)
    assert 0.7 < sv.min() <= sv.max() < 1.3


def test_distortion_identity_and_injective_sketch_are_isometries():
    # S = I: SA R_A^-1 = Q has orthonormal columns, every singular value is 1.
    # A hash without collisions makes S a signed row selection, S Q keeps
    # orthonormal columns, so again all ones.  A transposed or lower-triangular
    # R, or R in place of its inverse, breaks both.
    rng = np.random.default_rng(5)
    Ad = rng.standard_normal((60, 7)) @ np.diag([1.0, 3.0, 0.2, 10.0, 1.5, 0.5, 4.0])
    R_A = np.linalg.qr(Ad, mode="r")
    np.testing.assert_allclose(oracle.distortion(Ad, R_A), np.ones(7), rtol=0, atol=1e-12)
    m = 1 << 20
    for seed in range(1, 50):
        h, _ = oracle.hash(seed, m, 0, Ad.shape[0])
        if len(set(h.tolist())) == Ad.shape[0]:
            break
    else:
        pytest.fail("no collision-free seed")
    rp = np.arange(0, Ad.size + 1, Ad.shape[1], dtype=np.int32)
    col = np.tile(np.arange(Ad.shape[1], dtype=np.int32), Ad.shape[0])
    SA, _ = oracle.sketch_csr(rp, col, Ad.ravel().astype(np.float32), Ad.shape[1], None, m, seed=seed)
    Af = Ad.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(oracle.distortion(SA, np.linalg.qr(Af, mode="r")), np.ones(7), rtol=0, atol=1e-10)


def test_distortion_equals_generalized_eigenvalues():
    # The singular values of SA R_A^-1 squared are the eigenvalues of
    # R_A^-T (SA^T SA) R_A^-1, i.e. the generalized eigenvalues of the pencil
    # (SA^T SA, A^T A): a route with no triangular factor at all.
    A, b, SA, _ = _problem(n=3000, d=6, m=64, seed=9)
    Ad = A.to_dense().numpy().astype(np.float64)
    R_A = np.linalg.qr(Ad, mode="r")
    lam = sla.eigh(SA.T @ SA, Ad.T @ Ad, eigvals_only=True)
    want = np.sort(np.sqrt(lam))[::-1]
    got = oracle.distortion(SA, R_A)
    np.testing.assert_allclose(got, want, rtol=1e-9)
    assert got.max() > 1.05 and got.min() < 0.95   # m = 64 distorts visibly
