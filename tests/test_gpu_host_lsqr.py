"""cw_lsqr_precond_host: the preconditioned LSQR for A and b in host memory.

The call copies A to the device in row chunks and sketches each chunk as it
lands (SA = sum of S_k A_k over the chunks, with the hash at global row
indices), then runs the same preconditioner and LSQR as cw_lsqr_precond.
Checked against the float64 oracle (same S, same stopping rule): the
iteration count within one, the residual ratio ||A x - b|| / ||A x* - b||
within 1e-6 of the oracle's; the result does not depend on where the chunks
fall (compared with the device-pointer call); two calls give the same x bit
for bit.  Edge cases: ragged and empty rows, fewer rows than chunks, page-locked
and ordinary host memory.
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


def _host(A, b, pinned):
    if not pinned:
        return A, b
    return W.CSR(A.n, A.d, A.row_ptr.pin_memory(), A.col.pin_memory(), A.val.pin_memory()), b.pin_memory()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("case", ["zipf", "ragged", "tiny"])
def test_host_lsqr_matches_oracle(cw, case, pinned):
    if case == "zipf":
        A = W.csr_zipf(1 << 18, 64, 16, 1.1, seed=1002)
        b, _ = W.rhs(A, 0.01, seed=2002)
        m, seed = 4096, 1
    elif case == "ragged":
        A = W.csr_random_lengths(120000, 40, 0, 30, seed=5, empty_frac=0.05)
        b, _ = W.rhs(A, 0.1, seed=6)
        m, seed = 1600, 3
    else:  # fewer rows than chunks
        A = W.csr_uniform(6, 3, 2, seed=7)
        b, _ = W.rhs(A, 0.1, seed=8)
        m, seed = 16, 2
    Ah, bh = _host(A, b, pinned)
    x, it, test = cw.cw_lsqr_precond_host(Ah, bh, m, seed, rtol=1e-6, max_iter=100, allow_noconv=(case == "tiny"))
    x = x.numpy()
    rp, c, v = A.numpy()
    SA_o, Sb_o = oracle.sketch_csr(rp, c, v, A.d, b, m, seed)
    x0_o, R_o = oracle.solve_sketch(SA_o, Sb_o)
    x_o, it_o, test_o, conv_o, _ = oracle.lsqr_precond_csr(rp, c, v, A.d, b, R_o, x0_o, 1e-6, 100)
    _, rn = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
    if case != "tiny":
        assert abs(it - it_o) <= 1, (it, it_o)
    assert abs(_rho(A, b, x, rn) - _rho(A, b, x_o, rn)) <= RHO_TOL
    # the device-pointer call on the same data: same solution up to LSQR's tolerance
    xd, itd, _ = cw.cw_lsqr_precond(A.to("cuda"), b.cuda(), m, seed, rtol=1e-6, max_iter=100,
                                    allow_noconv=(case == "tiny"))
    assert abs(_rho(A, b, x, rn) - _rho(A, b, xd.cpu().numpy(), rn)) <= RHO_TOL
    # deterministic
    x2, _, _ = cw.cw_lsqr_precond_host(Ah, bh, m, seed, rtol=1e-6, max_iter=100, allow_noconv=(case == "tiny"))
    assert np.array_equal(x, x2.numpy())
