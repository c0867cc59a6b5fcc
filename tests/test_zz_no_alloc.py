"""cw_sketch_csr_noalloc: the CSR sketch for callers that cannot allocate.

Some callers cannot allocate device memory while they run: code under an
allocator that owns all of the device's memory, latency-critical paths where
a pool allocation could block, or hosts whose allocator must not be entered
again.  cw_sketch_csr_noalloc serves them with scratch taken from a static
device array inside the library.

The tests call it through the C ABI, two calls in a row with different shapes
and seeds, so the second call reuses the array after the first.  Each result
must equal cw_sketch_csr bit for bit, because both run the same kernels in the
same fixed order.  It must also agree with the float64 oracle within the
sketch tolerance (1e-5 of each bucket's absolute sum).  The default memory
pool's reserved and used bytes must not change across the call.  A problem
too large for the array must be rejected before anything is launched.  A
column index out of range must be reported by cw_noalloc_status and then
cleared.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
CW_ERR_SHAPE, CW_ERR_DEVICE = -2, -9


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
    np.add.at(absb, h, np.abs(b.double().numpy()))
    return TOL * absA + 1e-30, TOL * absb + 1e-30


class _Pool:
    """Reserved and used bytes of the current device's default memory pool
    (the pool cw_sketch_csr allocates its scratch from), read through the
    CUDA driver API."""

    RESERVED_CURRENT, USED_CURRENT = 0x5, 0x7  # CU_MEMPOOL_ATTR_{RESERVED,USED}_MEM_CURRENT

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def read(self):
        out = []
        for attr in (self.RESERVED_CURRENT, self.USED_CURRENT):
            v = ctypes.c_uint64()
            assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
            out.append(v.value)
        return tuple(out)


def test_noalloc_matches_sketch_csr_and_oracle_twice():
    import paper_1207_6365_gb300 as cw
    cw.load()
    cases = [
        (W.csr_zipf(200000, 256, 16, 1.1, seed=11), 4096, 1),
        (W.csr_random_lengths(77777, 40, 0, 30, seed=12, empty_frac=0.1), 1000, 2),
    ]
    pool = _Pool()
    for A, m, seed in cases:
        b = torch.randn(A.n, generator=torch.Generator().manual_seed(seed + 100))
        Ag, bg = A.to("cuda"), b.cuda()
        SA_ref, Sb_ref = cw.cw_sketch_csr(Ag, bg, m, seed)
        torch.cuda.synchronize()
        before = pool.read()
        st, SA, Sb = _noalloc(cw, Ag, bg, m, seed)
        after = pool.read()
        assert st == 0, cw.status_string(st)
        assert before == after, "the default memory pool changed across the call: %s -> %s" % (before, after)
        assert torch.equal(SA, SA_ref) and torch.equal(Sb, Sb_ref)
        SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, m, seed)
        bA, bb = _bound(A, b, m, seed)
        assert (np.abs(SA.cpu().double().numpy() - SA_o) <= bA).all()
        assert (np.abs(Sb.cpu().double().numpy() - Sb_o) <= bb).all()
        assert load_status(cw) == 0


def load_status(cw):
    return cw.load().cw_noalloc_status(cw._stream())


def test_noalloc_rejects_problems_beyond_its_array():
    import paper_1207_6365_gb300 as cw
    cw.load()
    # 1.2 M rows with b need about 33.6 MB of scratch (28 bytes a row), well
    # beyond the 24 MiB array
    A = W.csr_uniform(1200000, 8, 2, seed=3, device="cuda")
    b = torch.ones(A.n, device="cuda")
    st, SA, Sb = _noalloc(cw, A, b, 4096, 1)
    assert st == CW_ERR_SHAPE
    assert torch.isnan(SA).all() and torch.isnan(Sb).all()  # nothing was launched


def test_noalloc_reports_and_clears_a_column_out_of_range():
    import paper_1207_6365_gb300 as cw
    cw.load()
    assert load_status(cw) == 0
    A = W.csr_uniform(5000, 10, 3, seed=21)
    A.col[17] = 10  # one past the last column: the kernel skips it and flags it
    b = torch.randn(A.n)
    st, SA, _ = _noalloc(cw, A.to("cuda"), b.cuda(), 256, 4)
    assert st == 0
    assert load_status(cw) == CW_ERR_DEVICE
    assert load_status(cw) == 0  # read once, then cleared
    cw.device_status()  # the ordinary calls' flag is a different word
