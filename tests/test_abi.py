"""The C-ABI library loads and exports every function include/cw.h declares.

Runs without a GPU: loading libcw.so needs only the CUDA runtime library, and
the argument checks below return before any device call.
"""
import ctypes
import os
import re

import pytest

import paper_1207_6365_gb300 as cw

HEADER = cw.HEADER


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cw_sketch_csr", "cw_sketch_dense", "cw_sketch_vec", "cw_solve_sketch", "cw_lsqr_precond",
              "cw_leverage", "cw_hash", "cw_qr", "cw_gram", "cw_sketch_csr_general"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = cw.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(cw.EXPORTS) <= set(_declared())


def test_status_strings_and_version():
    lib = cw.load()
    assert lib.cw_version() >= 100
    for code in range(-9, 1):
        assert cw.status_string(code).startswith("CW_")
    assert "unknown" in cw.status_string(-42)


def test_host_side_validation_rejects_bad_arguments():
    lib = cw.load()
    null = None
    # m < 1, negative counts, overflowing index ranges: rejected before any launch
    assert lib.cw_hash(1, 0, 0, 10, null, null, null) == -2
    assert lib.cw_hash(1, 10, -1, 10, null, null, null) == -3
    assert lib.cw_hash(1, 10, 2**62, 10, null, null, null) == -3
    assert lib.cw_sketch_csr(null, null, 10, 1, null, null, null) == -1
    # the host-memory LSQR checks row_ptr's ends before touching the device
    rp = (ctypes.c_int32 * 3)(0, 2, 3)
    hc = cw._CSR()
    hc.n, hc.d, hc.nnz = 2, 2, 4
    hc.row_ptr = ctypes.cast(rp, ctypes.c_void_p)
    hc.col = ctypes.c_void_p(16)
    hc.val = ctypes.c_void_p(16)
    xh = (ctypes.c_double * 2)()
    assert lib.cw_lsqr_precond_host(ctypes.byref(hc), ctypes.c_void_p(16), 8, 1, 1e-6, 10, xh, None, None,
                                    null) == -1
    # the barrier self-test checks its arguments before touching the device
    assert lib.cw_selftest_barrier_timeout(0, 100, null) == -1
    assert lib.cw_selftest_barrier_timeout(2, 0, null) == -1
    assert lib.cw_selftest_barrier_timeout(2, (1 << 24) + 1, null) == -1
    c = cw._CSR()
    c.n, c.d, c.nnz = 10, 4, 10
    assert lib.cw_sketch_csr(ctypes.byref(c), null, 0, 1, ctypes.c_void_p(16), null, null) == -2
    assert lib.cw_sketch_csr(ctypes.byref(c), null, 1 << 20, 1, ctypes.c_void_p(16), null, null) == -2
    c.nnz = 2**31
    assert lib.cw_sketch_csr(ctypes.byref(c), null, 8, 1, ctypes.c_void_p(16), null, null) == -3
    c.nnz = 10
    assert lib.cw_sketch_csr_general(ctypes.byref(c), null, 1 << 10, 1 << 10, 1, 1, ctypes.c_void_p(16), null,
                                     null) == -2
    assert lib.cw_sketch_csr_general(ctypes.byref(c), null, 4, 4, 0, 1, ctypes.c_void_p(16), null, null) == -2
    assert lib.cw_sketch_csr_general(ctypes.byref(c), null, 1 << 19, 1, 4096, 1, ctypes.c_void_p(16), null,
                                     null) == -3
    assert lib.cw_sketch_csr_general(null, null, 4, 4, 1, 1, null, null, null) == -1
    assert lib.cw_sketch_dense(null, 10, 4, 2, null, 8, 1, ctypes.c_void_p(16), null, null) == -1
    assert lib.cw_sketch_dense(ctypes.c_void_p(16), 10, 4, 2, null, 8, 1, ctypes.c_void_p(16), null, null) == -2
    assert lib.cw_qr(ctypes.c_void_p(16), 4, 8, null, null, null, null) == -2
    assert lib.cw_gram(null, 4, 8, null, ctypes.c_void_p(16), null) == -1
    assert lib.cw_gram(ctypes.c_void_p(16), 4, 8, null, null, null) == -1
    assert lib.cw_gram(ctypes.c_void_p(16), 4, 0, null, ctypes.c_void_p(16), null) == -2
    assert lib.cw_gram(ctypes.c_void_p(16), 4, 1025, null, ctypes.c_void_p(16), null) == -2
    assert lib.cw_gram(ctypes.c_void_p(16), 0, 8, null, ctypes.c_void_p(16), null) == -2
    it = ctypes.c_int32(0)
    ft = ctypes.c_double(0)
    c.nnz = 10
    assert lib.cw_lsqr_precond(ctypes.byref(c), ctypes.c_void_p(16), 64, 1, -1.0, 10, ctypes.c_void_p(16),
                               ctypes.byref(it), ctypes.byref(ft), null) == -1
    assert lib.cw_leverage(ctypes.c_void_p(16), 100, 8, 8, 64, 1, 0, ctypes.c_void_p(16), ctypes.c_void_p(16),
                           null) == -2
    # the segment read probe: pointers, a power-of-two segment count, 1..8 CTAs per SM
    p16 = ctypes.c_void_p(16)
    assert lib.cw_probe_gather64(null, 64, 64, 0, 4, p16, null) == -1
    assert lib.cw_probe_gather64(p16, 64, 64, 0, 4, null, null) == -1
    assert lib.cw_probe_gather64(p16, 48, 64, 0, 4, p16, null) == -2
    assert lib.cw_probe_gather64(p16, 0, 64, 0, 4, p16, null) == -2
    assert lib.cw_probe_gather64(p16, 64, -1, 0, 4, p16, null) == -2
    assert lib.cw_probe_gather64(p16, 1 << 41, 64, 0, 4, p16, null) == -3
    assert lib.cw_probe_gather64(p16, 64, 64, 0, 0, p16, null) == -1
    assert lib.cw_probe_gather64(p16, 64, 64, 1, 9, p16, null) == -1
    assert lib.cw_probe_gather64(p16, 64, 0, 0, 4, p16, null) == 0   # nothing to read: no launch


def test_built_for_sm103a():
    from paper_1207_6365_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_batch_plan_rejects_bad_arguments_before_any_launch():
    lib = cw.load()
    plan = ctypes.c_void_p(None)
    assert lib.cw_batch_create(None, 1, 0, None, ctypes.byref(plan)) == -1
    arr = (cw._BatchProblem * 1)()
    assert lib.cw_batch_create(arr, 0, 0, None, ctypes.byref(plan)) == -1
    arr[0].A.n, arr[0].A.d, arr[0].A.nnz, arr[0].m = 10, 200, 10, 40000   # d > 128
    arr[0].x = 16
    assert lib.cw_batch_create(arr, 1, 0, None, ctypes.byref(plan)) == -2
    arr[0].A.d, arr[0].m = 16, 8                                           # m < d
    assert lib.cw_batch_create(arr, 1, 0, None, ctypes.byref(plan)) == -2
    arr[0].m = 64
    arr[0].x = None                                                        # no output
    assert lib.cw_batch_create(arr, 1, 0, None, ctypes.byref(plan)) == -1
    assert plan.value is None
    assert lib.cw_batch_destroy(None) == 0
