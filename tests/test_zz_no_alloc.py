"""cw_sketch_csr_noalloc: the CSR sketch for callers that cannot allocate.

Callers running under an allocator that owns all device memory, or on paths
where a pool allocation could block, use this entry point; its scratch is a
static device array inside the library.  The test calls it through the C ABI
twice in a row (different shapes and seeds, so the second call reuses the
array after the first one) and checks both results against cw_sketch_csr
within the sketch tolerance (1e-5 of each bucket's absolute sum), then checks
that a problem too large for the array is rejected with CW_ERR_SHAPE.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _noalloc(cw, A, b, m, seed):
    SA = torch.full((m, A.d), float("nan"), device="cuda")
    Sb = torch.full((m,), float("nan"), device="cuda") if b is not None else None
    c = cw._csr(A)
    st = cw.load().cw_sketch_csr_noalloc(ctypes.byref(c), cw._ptr(b), m, seed, cw._ptr(SA), cw._ptr(Sb),
                                         cw._stream())
    torch.cuda.synchronize()
    return st, SA, Sb


def _bound(A, b, m, seed):
    rp, col, val = A.numpy()
    h, _ = oracle.hash(seed, m, 0, A.n)
    absA = np.zeros((m, A.d))
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    np.add.at(absA, (h[rows], col), np.abs(val.astype(np.float64)))
    absb = np.zeros(m)
    if b is not None:
        np.add.at(absb, h, np.abs(b.cpu().double().numpy()))
    return TOL * absA + 1e-30, TOL * absb + 1e-30


def test_noalloc_matches_sketch_csr_twice():
    import paper_1207_6365_gb300 as cw
    cw.load()
    cases = [
        (W.csr_zipf(200000, 256, 16, 1.1, seed=11, device="cuda"), 4096, 1),
        (W.csr_random_lengths(77777, 40, 0, 30, seed=12, empty_frac=0.1, device="cuda"), 1000, 2),
    ]
    for A, m, seed in cases:
        b = torch.randn(A.n, device="cuda")
        st, SA, Sb = _noalloc(cw, A, b, m, seed)
        assert st == 0, cw.status_string(st)
        SA_ref, Sb_ref = cw.cw_sketch_csr(A, b, m, seed)
        torch.cuda.synchronize()
        bA, bb = _bound(A, b, m, seed)
        assert (np.abs(SA.cpu().double().numpy() - SA_ref.cpu().double().numpy()) <= bA).all()
        assert (np.abs(Sb.cpu().double().numpy() - Sb_ref.cpu().double().numpy()) <= bb).all()


def test_noalloc_rejects_problems_beyond_its_array():
    import paper_1207_6365_gb300 as cw
    cw.load()
    A = W.csr_uniform(1 << 20, 8, 2, seed=3, device="cuda")  # 28 MiB of scratch > 24 MiB
    st, SA, _ = _noalloc(cw, A, None, 4096, 1)
    assert st == -2
    assert torch.isnan(SA).all()  # nothing was launched
