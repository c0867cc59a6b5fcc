"""The learned + random sketch: its training gradient and its residual ratios
against the float64 oracle.

* The gradient of rho^2 - 1 with respect to the learned values (library
  forward and backward kernels + a float64 QR in torch) equals central
  differences of the same loss computed end to end by the float64 oracle
  (oracle sketches, oracle Householder solve, exact x* by QR of [A | b]).
* After training, the residual ratio of the learned + random sketch on a
  held-out matrix of the full-size family (n = 2^20, d = 128, m = 2048) is the
  one the float64 oracle computes for the same values (to 1e-5), and so is the
  plain CountSketch's.
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


def test_learned_sketch_trains_and_is_judged_by_the_oracle_at_full_size(cw):
    from paper_1207_6365_gb300 import learned as L
    n, d, m = 1 << 20, 128, 2048
    V, sig = W.family_basis(d, seed=7, device="cuda")
    sk = L.LearnedSketch(n, m, seed_L=11, seed_R=12)

    def member(k):
        A, b = W.family_matrix(k, n, V, sig, device="cuda")
        return A, b, L.MatrixStats(A, b), sk.random_half(A, b)
    train_set = [member(k) for k in range(4)]
    hist = L.train(sk, train_set, epochs=2, lr=1e-3)
    assert all(np.isfinite(hist))
    # the oracle judges the sketch at a seeded v (its inputs never come from the
    # library): the hash signs of S_L times 1 + 0.1 N(0,1)
    _, sgn = oracle.hash(11, m // 2, 0, n)
    gen = torch.Generator().manual_seed(21)
    v_eval = torch.as_tensor(np.asarray(sgn, dtype=np.float32)) * (1 + 0.1 * torch.randn(n, generator=gen))
    with torch.no_grad():
        sk.v.copy_(v_eval.to(sk.v.device))
    A, b, st, rh = member(100000)
    with torch.no_grad():
        rho_gpu = st.ratio(sk.solve(A, b, rh))
        rho_plain = L.plain_ratio(A, b, st, m, seed_P=13)
    Ah, bh = A.cpu(), b.cpu()
    rho_o = _oracle_ratio(Ah, bh, v_eval, m // 2, 11, 12)
    assert abs(rho_gpu - rho_o) <= 1e-5 * rho_o, (rho_gpu, rho_o)
    SA, Sb = oracle.sketch_dense(Ah, bh, m, 13)
    x, _ = oracle.solve_sketch(SA, Sb)
    _, rstar = oracle.lstsq_exact_dense(Ah, bh)
    rho_plain_o = float(np.linalg.norm(Ah.double().numpy() @ x - bh.double().numpy())) / rstar
    assert abs(rho_plain - rho_plain_o) <= 1e-5 * rho_plain_o, (rho_plain, rho_plain_o)
