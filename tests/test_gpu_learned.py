"""The learned + random sketches: their training gradients, the library's
sketched-solve backward and loss constants, and residual ratios, all against
the float64 oracle.

* cw_solve_sketched_backward: for L = c^T x'(SA, Sb) (x' the sketch-and-solve
  solution), the library's dL/dSA and dL/dSb equal central differences of the
  oracle's Householder solve; the normal-equations route (cw_gram +
  cw_normal_solve) gives the oracle's R and x' too.
* cw_normal_solve / cw_excess_residual: x* and ||A x* - b|| from the bordered
  Gram matrix equal the oracle's QR of [A | b], and rho^2 - 1 equals the
  oracle's residual ratio of a given x.
* The gradient of rho^2 - 1 with respect to the learned values, per column
  (LearnedSketch) and tied per bucket (TiedSketch), equals central
  differences of the same loss computed end to end by the oracle (oracle
  sketches, oracle Householder solve, exact x* by QR of [A | b]).
* After training, the residual ratio of the learned + random sketch on a
  held-out matrix of the full-size family (n = 2^20, d = 128, m = 2048) is the
  one the oracle computes for the same values (to 1e-5), and so is the plain
  sparse embedding's.
* select_or_fallback keeps the trained sketch exactly when its mean ratio on
  the selection members is below the plain one, and the Selection solves new
  matrices with the sketch it chose.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


def _oracle_ratio(A, b, v, mh, seed_L, seed_R):
    SA_L, Sb_L = oracle.sketch_dense_values(A, b, mh, seed_L, v)
    SA_R, Sb_R = oracle.sketch_dense(A, b, mh, seed_R)
    x, _ = oracle.solve_sketch(np.vstack([SA_L, SA_R]), np.concatenate([Sb_L, Sb_R]))
    _, rstar = oracle.lstsq_exact_dense(A, b)
    r = A.double().numpy() @ x - b.double().numpy()
    return float(np.linalg.norm(r)) / rstar


def test_solve_backward_matches_oracle_finite_differences(cw):
    m, d = 96, 7
    g = torch.Generator().manual_seed(5)
    SA = torch.randn(m, d, generator=g)
    Sb = torch.randn(m, generator=g)
    c = torch.randn(d, dtype=torch.float64, generator=g)
    x, R = cw.cw_solve_sketched(SA.cuda(), Sb.cuda())
    xo, Ro = oracle.solve_sketch(SA.double().numpy(), Sb.double().numpy())
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-12 * np.abs(xo).max())
    np.testing.assert_allclose(R.cpu().numpy(), Ro, rtol=0, atol=1e-12 * np.abs(Ro).max())
    # the normal-equations route: the same R and x' up to the 3xTF32 Gram's rounding
    xn, r2n, Rn = cw.cw_normal_solve(cw.cw_gram(SA.cuda(), Sb.cuda()), want_R=True)
    np.testing.assert_allclose(Rn.cpu().numpy(), Ro, rtol=0, atol=1e-4 * np.abs(Ro).max())
    np.testing.assert_allclose(xn.cpu().numpy(), xo, rtol=0, atol=1e-4 * np.abs(xo).max())
    rr = float(np.linalg.norm(SA.double().numpy() @ xo - Sb.double().numpy()))
    assert abs(float(r2n) ** 0.5 - rr) <= 1e-4 * rr
    gSA, gSb = cw.cw_solve_sketched_backward(SA.cuda(), Sb.cuda(), R, x, c.cuda())
    gSA, gSb = gSA.cpu().double().numpy(), gSb.cpu().double().numpy()
    M0, y0, cn = SA.double().numpy(), Sb.double().numpy(), c.numpy()

    def L(M, y):
        return float(cn @ oracle.solve_sketch(M, y)[0])
    eps = 1e-6
    gscale = max(np.abs(gSA).max(), np.abs(gSb).max())
    for (i, j) in [(0, 0), (5, 3), (m - 1, d - 1), (40, 2), (17, 6)]:
        Mp, Mm = M0.copy(), M0.copy()
        Mp[i, j] += eps
        Mm[i, j] -= eps
        fd = (L(Mp, y0) - L(Mm, y0)) / (2 * eps)
        assert abs(fd - gSA[i, j]) <= 1e-5 * gscale, (i, j, fd, gSA[i, j])
    for i in [0, 33, m - 1]:
        yp, ym = y0.copy(), y0.copy()
        yp[i] += eps
        ym[i] -= eps
        fd = (L(M0, yp) - L(M0, ym)) / (2 * eps)
        assert abs(fd - gSb[i]) <= 1e-5 * gscale, (i, fd, gSb[i])


def test_normal_solve_and_excess_match_oracle(cw):
    from paper_1207_6365_gb300 import learned as L
    V, sig = W.family_basis(16, seed=7)
    A, b = W.family_matrix(3, 20000, V, sig)
    st = L.MatrixStats(A.cuda(), b.cuda())
    xo, rstar = oracle.lstsq_exact_dense(A, b)
    np.testing.assert_allclose(st.xstar.cpu().numpy(), xo, rtol=0, atol=1e-4 * np.abs(xo).max())
    assert abs(float(st.rstar2) ** 0.5 - rstar) <= 1e-5 * rstar
    # rho of a perturbed solution, against the oracle's residual norm
    xt = torch.as_tensor(xo) + 0.05 * torch.randn(16, dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    rho = st.ratio(xt.cuda())
    rho_o = float(np.linalg.norm(A.double().numpy() @ xt.numpy() - b.double().numpy())) / rstar
    assert abs(rho - rho_o) <= 1e-5 * rho_o, (rho, rho_o)


def test_normal_solve_reports_rank_deficiency(cw):
    A = torch.randn(500, 6, generator=torch.Generator().manual_seed(1))
    A[:, 4] = A[:, 1]
    b = torch.randn(500, generator=torch.Generator().manual_seed(2))
    G = cw.cw_gram(A.cuda(), b.cuda())
    with pytest.raises(cw.CWError) as e:
        cw.cw_normal_solve(G)
    assert e.value.status == -5  # CW_ERR_RANK


def test_training_gradient_matches_oracle_finite_differences(cw):
    from paper_1207_6365_gb300 import learned as L
    n, d, m = 4096, 8, 64
    V, sig = W.family_basis(d, seed=7)
    A, b = W.family_matrix(0, n, V, sig)
    Ag, bg = A.cuda(), b.cuda()
    sk = L.LearnedSketch(n, m, seed_L=11, seed_R=12)
    with torch.no_grad():
        sk.v.mul_(1.0 + 0.3 * torch.rand(n, generator=torch.Generator(device="cuda").manual_seed(1),
                                          device="cuda"))
    st = L.MatrixStats(Ag, bg)
    loss = st.excess(sk.solve(Ag, bg))
    loss.backward()
    g = sk.v.grad.cpu().double().numpy()
    v = sk.v.detach().cpu()

    def oloss(vv):
        rho = _oracle_ratio(A, b, vv, m // 2, 11, 12)
        return rho * rho - 1.0
    assert abs(float(loss.detach()) - oloss(v)) <= 1e-4 * abs(oloss(v))
    # coordinates with the largest gradients, plus a few others
    idx = list(np.argsort(-np.abs(g))[:6]) + [0, 1000, 4095]
    for i in idx:
        eps = 2.0 ** -8
        vp, vm = v.clone(), v.clone()
        vp[i] += eps
        vm[i] -= eps
        fd = (oloss(vp) - oloss(vm)) / (float(vp[i]) - float(vm[i]))
        assert abs(fd - g[i]) <= 2e-3 * np.abs(g).max(), (i, fd, g[i])


def test_tied_gradient_matches_oracle_finite_differences(cw):
    """Values tied per bucket: v_i = w_{h(i)} sigma(i); the oracle sees only v."""
    from paper_1207_6365_gb300 import learned as L
    n, d, m = 6000, 8, 64
    mh = m // 2
    V, sig = W.family_basis(d, seed=7)
    A, b = W.family_matrix(1, n, V, sig)
    sk = L.TiedSketch(m, seed_L=11, seed_R=12)
    w0 = 1.0 + 0.3 * torch.rand(mh, generator=torch.Generator().manual_seed(3))
    with torch.no_grad():
        sk.w.copy_(w0.cuda())
    mem = sk.member(A.cuda(), b.cuda())
    loss = sk.loss(mem)
    loss.backward()
    g = sk.w.grad.cpu().double().numpy()
    # training through the normal equations gives the same gradient up to rounding
    skn = L.TiedSketch(m, seed_L=11, seed_R=12, method="normal")
    with torch.no_grad():
        skn.w.copy_(w0.cuda())
    skn.loss(mem).backward()
    gn = skn.w.grad.cpu().double().numpy()
    assert np.abs(gn - g).max() <= 1e-3 * np.abs(g).max()
    h, sgn = oracle.hash(11, mh, 0, n)
    sgn = np.asarray(sgn, dtype=np.float64)

    def oloss(w):
        v = torch.as_tensor((np.asarray(w, dtype=np.float32)[h] * sgn).astype(np.float32))
        rho = _oracle_ratio(A, b, v, mh, 11, 12)
        return rho * rho - 1.0
    w = w0.numpy().astype(np.float64)
    assert abs(float(loss.detach()) - oloss(w)) <= 1e-4 * abs(oloss(w))
    for k in list(np.argsort(-np.abs(g))[:4]) + [0, mh - 1]:
        eps = 2.0 ** -8
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (oloss(wp) - oloss(wm)) / (2 * eps)
        assert abs(fd - g[k]) <= 2e-3 * np.abs(g).max(), (k, fd, g[k])
    # the tied solve is the values sketch with v = w[h] sigma
    with torch.no_grad():
        x_t = sk.solve(A.cuda(), b.cuda())
        SA_L, Sb_L = cw.SketchValues.apply(sk.values(n), A.cuda(), b.cuda(), mh, 11)
        SA_R, Sb_R = cw.cw_sketch_dense(A.cuda(), b.cuda(), mh, 12)
        x_v, _ = cw.cw_solve_sketched(torch.cat([SA_L, SA_R]), torch.cat([Sb_L, Sb_R]))
    np.testing.assert_allclose(x_t.cpu().numpy(), x_v.cpu().numpy(), rtol=0,
                               atol=1e-5 * float(x_v.abs().max()))


def test_learned_sketch_trains_and_is_judged_by_the_oracle_at_full_size(cw):
    from paper_1207_6365_gb300 import learned as L
    n, d, m = 1 << 20, 128, 2048
    V, sig = W.family_basis(d, seed=7, device="cuda")
    sk = L.LearnedSketch(n, m, seed_L=11, seed_R=12)

    def member(k):
        A, b = W.family_matrix(k, n, V, sig, device="cuda")
        return sk.member(A, b, m, seed_P=13)
    train_set = [member(k) for k in range(4)]
    hist = L.train(sk, train_set, epochs=2, lr=1e-3)
    assert all(np.isfinite(hist))
    del train_set
    # the oracle judges the sketch at a seeded v (its inputs never come from the
    # library): the hash signs of S_L times 1 + 0.1 N(0,1)
    _, sgn = oracle.hash(11, m // 2, 0, n)
    gen = torch.Generator().manual_seed(21)
    v_eval = torch.as_tensor(np.asarray(sgn, dtype=np.float32)) * (1 + 0.1 * torch.randn(n, generator=gen))
    with torch.no_grad():
        sk.v.copy_(v_eval.to(sk.v.device))
    mem = member(100000)
    rho_gpu = sk.ratio(mem)
    Ah, bh = mem.A.cpu(), mem.b.cpu()
    rho_o = _oracle_ratio(Ah, bh, v_eval, m // 2, 11, 12)
    assert abs(rho_gpu - rho_o) <= 1e-5 * rho_o, (rho_gpu, rho_o)
    SA, Sb = oracle.sketch_dense(Ah, bh, m, 13)
    x, _ = oracle.solve_sketch(SA, Sb)
    _, rstar = oracle.lstsq_exact_dense(Ah, bh)
    rho_plain_o = float(np.linalg.norm(Ah.double().numpy() @ x - bh.double().numpy())) / rstar
    assert abs(mem.plain - rho_plain_o) <= 1e-5 * rho_plain_o, (mem.plain, rho_plain_o)


def test_tied_sketch_select_or_fallback(cw):
    from paper_1207_6365_gb300 import learned as L
    n, d, m = 1 << 16, 32, 256
    V, sig = W.family_basis(d, seed=7, device="cuda")
    sk = L.TiedSketch(m, seed_L=11, seed_R=12, method="normal")

    def member(k):
        A, b = W.family_matrix(k, n, V, sig, device="cuda")
        return sk.member(A, b, m, seed_P=13)
    train_set = [member(k) for k in range(12)]
    selection = [member(200000 + k) for k in range(6)]
    hist = L.train(sk, train_set, epochs=3, lr=1e-2)
    assert len(hist) == 3 and all(np.isfinite(hist))
    assert not torch.equal(sk.w.detach(), torch.ones_like(sk.w))
    sel = L.select_or_fallback(sk, selection, m, seed_P=13)
    plain, learned = L.evaluate(sk, selection)
    assert sel.mean_plain == pytest.approx(np.mean(plain), rel=1e-12)
    assert sel.mean_learned == pytest.approx(np.mean(learned), rel=1e-12)
    assert sel.use_learned == (np.mean(learned) < np.mean(plain))
    # the Selection solves a new matrix with the sketch it chose
    A, b = W.family_matrix(300000, n, V, sig, device="cuda")
    x = sel.solve(A, b)
    if sel.use_learned:
        with torch.no_grad():
            ref = sk.solve(A, b)
    else:
        ref = cw.cw_solve_sketch_dense(A, b, m, 13)
    assert torch.equal(x, ref)
    # both branches exist: a Selection forced either way
    for use in (True, False):
        s2 = L.Selection(sk, use, m, 13, 0.0, 0.0)
        assert s2.name == ("learned" if use else "plain")
        assert s2.solve(A, b).shape == (d,)
