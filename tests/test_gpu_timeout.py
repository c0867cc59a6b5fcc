"""A bounded device-side wait that runs out reports CW_ERR_TIMEOUT and leaves
the context usable.

The library's cooperative kernels (the float64 QR, the batch's persistent
solve, the LSQR step) separate their phases with a grid barrier whose wait
gives up after a bounded number of polls, flags the call and returns.
cw_selftest_barrier_timeout runs that same barrier with blocks that wait for
one arrival more than the grid has, with a short poll limit (about a
millisecond): every block's wait runs out.  No kernel is left waiting, and an
ordinary sketch right after must still match the float64 oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CW_ERR_TIMEOUT = -7


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


@pytest.mark.parametrize("blocks", [1, 8, 152])
def test_grid_barrier_wait_runs_out_and_the_context_stays_usable(cw, blocks):
    st = cw.load().cw_selftest_barrier_timeout(blocks, 1 << 14, cw._stream())
    assert st == CW_ERR_TIMEOUT, cw.status_string(st)
    A = W.csr_uniform(20000, 16, 6, seed=7)
    b, _ = W.rhs(A, 0.1, seed=8)
    SA, Sb = cw.cw_sketch_csr(A.to("cuda"), b.cuda(), 512, 3)
    cw.device_status()
    SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, 512, 3)
    assert np.abs(SA.cpu().double().numpy() - SA_o).max() <= 1e-5 * (np.abs(SA_o).max() + 1)
    assert np.abs(Sb.cpu().double().numpy() - Sb_o).max() <= 1e-5 * (np.abs(Sb_o).max() + 1)
