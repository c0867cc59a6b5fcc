"""GPU parity of the sketch with values and of its backward kernel against the
float64 oracle, and the autograd wrapper against finite differences.

Forward: every SA / Sb entry within 1e-5 of its bucket's sum of |v_i A_ij|;
v = sigma reproduces cw_sketch_csr / cw_sketch_dense bit for bit.  Backward:
every gv_i within 1e-5 of sum_k |gSA[h(i), c_k] A_ik| + |gSb[h(i)] b_i|.
Autograd: the gradient of a loss through SketchValues equals the oracle's
float64 gradient and central differences of the oracle's float64 forward.
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


def _check(got, want, bound, what):
    got = got.detach().cpu().double().numpy()
    err = np.abs(got - want)
    bad = err > TOL * bound + 1e-30
    assert not bad.any(), "%s: %d out of tolerance, worst %.3g" % (what, int(bad.sum()), float(err.max()))


@pytest.mark.parametrize("n,d,k,m,seed", [(50001, 64, 8, 1024, 3), (9000, 17, 5, 999, 2), (300, 8, 3, 4096, 9),
                                          (20000, 40, 33, 64, 4)])
def test_csr_values_forward_and_backward(cw, n, d, k, m, seed):
    A = W.csr_uniform(n, d, k, seed=seed + 1)
    b, _ = W.rhs(A, 0.3, seed=seed + 2)
    g = torch.Generator().manual_seed(seed)
    v = torch.randn(n, generator=g)
    Ag, bg, vg = A.to("cuda"), b.cuda(), v.cuda()
    SA, Sb = cw.cw_sketch_csr_values(Ag, bg, m, seed, vg)
    cw.device_status()
    SA_o, Sb_o = oracle.sketch_csr_values(A.row_ptr, A.col, A.val, d, b, m, seed, v)
    h, _ = oracle.hash(seed, m, 0, n)
    rp, c, vals = A.numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    absA = np.zeros((m, d))
    np.add.at(absA, (h[rows], c), np.abs(v.numpy()[rows] * vals).astype(np.float64))
    absb = np.zeros(m)
    np.add.at(absb, h, np.abs(v.numpy() * b.numpy()).astype(np.float64))
    _check(SA, SA_o, absA, "SA")
    _check(Sb, Sb_o, absb, "Sb")
    G = torch.randn(m, d, generator=g)
    gb = torch.randn(m, generator=g)
    gv = cw.cw_sketch_values_backward_csr(Ag, bg, m, seed, G.cuda(), gb.cuda())
    gv_o = oracle.sketch_values_backward_csr(A.row_ptr, A.col, A.val, d, b, m, seed, G.double().numpy(),
                                             gb.double().numpy())
    bound = np.zeros(n)
    np.add.at(bound, rows, np.abs(G.double().numpy()[h[rows], c] * vals))
    bound += np.abs(gb.double().numpy()[h] * b.double().numpy())
    _check(gv, gv_o, bound, "gv")


@pytest.mark.parametrize("n,d,lda,m,seed", [(65536, 128, 128, 2048, 1), (10001, 33, 40, 256, 2), (4000, 5, 5, 7, 3)])
def test_dense_values_forward_and_backward(cw, n, d, lda, m, seed):
    A = W.dense_gaussian(n, lda, seed=seed)
    b = W.dense_gaussian(n, 1, seed=seed + 1)[:, 0].contiguous()
    g = torch.Generator().manual_seed(seed)
    v = torch.randn(n, generator=g)
    Ag = A.cuda()[:, :d]
    SA, Sb = cw.cw_sketch_dense_values(Ag, b.cuda(), m, seed, v.cuda())
    Ad = A[:, :d].contiguous()
    SA_o, Sb_o = oracle.sketch_dense_values(Ad, b, m, seed, v)
    h, _ = oracle.hash(seed, m, 0, n)
    absA = np.zeros((m, d))
    np.add.at(absA, h, np.abs(v.double().numpy()[:, None] * Ad.double().numpy()))
    absb = np.zeros(m)
    np.add.at(absb, h, np.abs(v.double().numpy() * b.double().numpy()))
    _check(SA, SA_o, absA, "SA")
    _check(Sb, Sb_o, absb, "Sb")
    G = torch.randn(m, d, generator=g)
    gb = torch.randn(m, generator=g)
    gv = cw.cw_sketch_values_backward_dense(Ag, b.cuda(), m, seed, G.cuda(), gb.cuda())
    gv_o = oracle.sketch_values_backward_dense(Ad, b, m, seed, G.double().numpy(), gb.double().numpy())
    bound = (np.abs(G.double().numpy()[h] * Ad.double().numpy())).sum(1) + np.abs(gb.double().numpy()[h] *
                                                                                    b.double().numpy())
    _check(gv, gv_o, bound, "gv")


def test_values_equal_to_signs_reproduce_the_sketch_bit_for_bit(cw):
    A = W.csr_zipf(80000, 64, 12, 1.1, seed=5)
    b, _ = W.rhs(A, 0.1, seed=6)
    m, seed = 2048, 7
    _, s = oracle.hash(seed, m, 0, A.n)
    sig = torch.from_numpy(s.astype(np.float32)).cuda()
    Ag, bg = A.to("cuda"), b.cuda()
    SA1, Sb1 = cw.cw_sketch_csr_values(Ag, bg, m, seed, sig)
    SA0, Sb0 = cw.cw_sketch_csr(Ag, bg, m, seed)
    assert torch.equal(SA1, SA0) and torch.equal(Sb1, Sb0)
    D = W.dense_gaussian(50000, 96, seed=8).cuda()
    _, s2 = oracle.hash(seed, m, 0, 50000)
    sig2 = torch.from_numpy(s2.astype(np.float32)).cuda()
    bd = bg[:50000].contiguous()
    SA1, Sb1 = cw.cw_sketch_dense_values(D, bd, m, seed, sig2)
    SA0, Sb0 = cw.cw_sketch_dense(D, bd, m, seed)
    assert torch.equal(SA1, SA0) and torch.equal(Sb1, Sb0)


def test_autograd_matches_oracle_gradient_and_finite_differences(cw):
    n, d, m, seed = 3000, 12, 64, 11
    A = W.dense_gaussian(n, d, seed=4)
    b = W.dense_gaussian(n, 1, seed=5)[:, 0].contiguous()
    g = torch.Generator().manual_seed(0)
    v = torch.randn(n, generator=g)
    W1 = torch.randn(m, d, generator=g, dtype=torch.float64)
    w2 = torch.randn(m, generator=g, dtype=torch.float64) * 0.1
    vg = v.cuda().requires_grad_(True)
    SA, Sb = cw.SketchValues.apply(vg, A.cuda(), b.cuda(), m, seed)
    L = 0.5 * (SA.double() ** 2).sum() + (W1.cuda() * SA.double()).sum() + torch.tanh((w2.cuda() * Sb.double()).sum())
    L.backward()
    gv = vg.grad.cpu().double().numpy()
    # the oracle's gradient at the same v
    SA_o, Sb_o = oracle.sketch_dense_values(A, b, m, seed, v)
    G = SA_o + W1.numpy()
    gb = (1 - np.tanh(w2.numpy() @ Sb_o) ** 2) * w2.numpy()
    gv_o = oracle.sketch_values_backward_dense(A, b, m, seed, G, gb)
    assert np.abs(gv - gv_o).max() <= 1e-4 * (np.abs(gv_o).max() + 1)

    def loss(vv):
        S_A, S_b = oracle.sketch_dense_values(A, b, m, seed, vv)
        return 0.5 * (S_A ** 2).sum() + (W1.numpy() * S_A).sum() + np.tanh(w2.numpy() @ S_b)
    # finite differences of the float64 oracle forward (values rounded to float32 by its input
    # type, so the step is taken in exactly representable amounts)
    for i in range(0, n, 397):
        eps = 2.0 ** -10
        vp, vm = v.clone(), v.clone()
        vp[i] += eps
        vm[i] -= eps
        fd = (loss(vp) - loss(vm)) / (float(vp[i]) - float(vm[i]))
        assert abs(fd - gv[i]) <= 1e-3 * (abs(fd) + 1), (i, fd, gv[i])
