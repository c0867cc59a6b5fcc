"""Pins for the oracle's sketch with values and its gradient.

S(v) has the one entry of column i at row h(i) (Section 2's map) with value
v_i; SA(v) and Sb(v) are linear in v and dL/dv_i = <dL/dSA[h(i)], A_i> +
dL/dSb[h(i)] b_i.  Pinned by:
* v = sigma gives the Section 2 sketch (exactly);
* SA(v) = S(v) A with S(v) written out explicitly (tiny inputs), CSR and dense;
* the gradient is the transpose of the linear map: <G, SA(dv)> + <g, Sb(dv)>
  = <gv(G, g), dv> for random G, g, dv;
* central finite differences in float64 of a nonlinear loss through the
  oracle's forward, CSR and dense.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W


def _signs(seed, m, n):
    return oracle.hash(seed, m, 0, n)[1].astype(np.float32)


def test_values_equal_to_the_signs_give_the_section2_sketch():
    A = W.csr_uniform(4000, 12, 5, seed=3)
    b, _ = W.rhs(A, 0.2, seed=4)
    m, seed = 97, 13
    SA, Sb = oracle.sketch_csr_values(A.row_ptr, A.col, A.val, 12, b, m, seed, _signs(seed, m, A.n))
    SA0, Sb0 = oracle.sketch_csr(A.row_ptr, A.col, A.val, 12, b, m, seed)
    np.testing.assert_array_equal(SA, SA0)
    np.testing.assert_array_equal(Sb, Sb0)
    Ad = W.dense_gaussian(3000, 7, seed=5)
    SAd, Sbd = oracle.sketch_dense_values(Ad, b[:3000], m, seed, _signs(seed, m, 3000))
    SAd0, Sbd0 = oracle.sketch_dense(Ad, b[:3000], m, seed)
    np.testing.assert_allclose(SAd, SAd0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Sbd, Sbd0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,d,k,m", [(40, 6, 3, 7), (300, 9, 4, 33), (64, 5, 5, 1)])
def test_values_sketch_equals_explicit_S_of_v(n, d, k, m):
    A = W.csr_uniform(n, d, k, seed=n)
    b, _ = W.rhs(A, 0.2, seed=1)
    v = torch.randn(n, generator=torch.Generator().manual_seed(n + 1))
    S = oracle.dense_S_values(21, m, n, v)
    SA, Sb = oracle.sketch_csr_values(A.row_ptr, A.col, A.val, d, b, m, 21, v)
    np.testing.assert_allclose(SA, S @ A.to_dense().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(Sb, S @ b.double().numpy(), rtol=0, atol=1e-12)
    Ad = A.to_dense().float()
    SAd, Sbd = oracle.sketch_dense_values(Ad, b, m, 21, v)
    np.testing.assert_allclose(SAd, S @ Ad.double().numpy(), rtol=0, atol=1e-12)


def test_gradient_is_the_transpose_of_the_linear_map():
    n, d, m, seed = 700, 10, 41, 8
    A = W.csr_uniform(n, d, 4, seed=2)
    b, _ = W.rhs(A, 0.2, seed=3)
    g = np.random.default_rng(0)
    G = g.standard_normal((m, d))
    gb = g.standard_normal(m)
    dv = g.standard_normal(n).astype(np.float32)
    SA, Sb = oracle.sketch_csr_values(A.row_ptr, A.col, A.val, d, b, m, seed, dv)
    lhs = float((G * SA).sum() + (gb * Sb).sum())
    gv = oracle.sketch_values_backward_csr(A.row_ptr, A.col, A.val, d, b, m, seed, G, gb)
    assert abs(lhs - float(gv @ dv.astype(np.float64))) <= 1e-10 * (abs(lhs) + 1)
    Ad = A.to_dense().float()
    SAd, Sbd = oracle.sketch_dense_values(Ad, b, m, seed, dv)
    lhs_d = float((G * SAd).sum() + (gb * Sbd).sum())
    gvd = oracle.sketch_values_backward_dense(Ad, b, m, seed, G, gb)
    assert abs(lhs_d - float(gvd @ dv.astype(np.float64))) <= 1e-10 * (abs(lhs_d) + 1)
    np.testing.assert_allclose(gvd, gv, rtol=0, atol=1e-10)


def _loss(SA, Sb, W1, w2):
    # a nonlinear loss of both outputs
    return 0.5 * float((SA * SA).sum()) + float((W1 * SA).sum()) + float(np.tanh(w2 @ Sb))


def _loss_grad(SA, Sb, W1, w2):
    return SA + W1, (1.0 - np.tanh(w2 @ Sb) ** 2) * w2


@pytest.mark.parametrize("dense", [False, True])
def test_gradient_matches_central_differences(dense):
    n, d, m, seed = 60, 5, 9, 4
    A = W.csr_uniform(n, d, 3, seed=7)
    b, _ = W.rhs(A, 0.2, seed=8)
    g = np.random.default_rng(1)
    W1 = g.standard_normal((m, d))
    w2 = g.standard_normal(m) * 0.1
    v = g.standard_normal(n)
    Ad = A.to_dense().float()

    def fwd(vv):
        # float64 forward of S(v) A (values kept in float64 through the explicit matrix)
        S = oracle.dense_S_values(seed, m, n, np.zeros(n))
        h, _ = oracle.hash(seed, m, 0, n)
        S[h, np.arange(n)] = vv
        return S @ Ad.double().numpy(), S @ b.double().numpy()

    SA, Sb = fwd(v)
    G, gb = _loss_grad(SA, Sb, W1, w2)
    if dense:
        gv = oracle.sketch_values_backward_dense(Ad, b, m, seed, G, gb)
    else:
        gv = oracle.sketch_values_backward_csr(A.row_ptr, A.col, A.val, d, b, m, seed, G, gb)
    eps = 1e-6
    for i in range(0, n, 7):
        e = np.zeros(n)
        e[i] = eps
        fd = (_loss(*fwd(v + e), W1, w2) - _loss(*fwd(v - e), W1, w2)) / (2 * eps)
        assert abs(fd - gv[i]) <= 1e-6 * (abs(gv[i]) + 1), (i, fd, gv[i])
