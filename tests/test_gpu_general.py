"""GPU parity of the generalized sparse embedding (paper Section "Generalized
Sparse Embedding Matrices") against the float64 oracle.

Every SA / Sb entry must agree with the oracle within 1e-5 of its output
row's absolute sum (sum over the rows i that land there of |A_ij| /
sqrt(kappa)), the float32 tolerance of the sparse-embedding kernels.  Cases
cover q * v a power of two and not, kappa = 1 and large kappa, ragged and
empty rows, wide rows (the accumulator in the output row itself), no b, the
empty matrix, and the special case q = kappa = 1, which must equal the
Section 2 sketch of the first inner seed bit for bit.
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


def _out_rows(n, q, v, kappa, seed):
    """(kappa, n) output row of each (inner sketch, input row) from the oracle's hashes."""
    h, _ = oracle.hash(seed, q, 0, n)
    seeds = oracle.general_seeds(seed, kappa)
    rows = np.empty((kappa, n), np.int64)
    for bidx in range(kappa):
        hb, _ = oracle.hash(seeds[bidx], v, 0, n)
        rows[bidx] = h.astype(np.int64) * v * kappa + bidx * v + hb
    return rows


def _bounds(A, b, q, v, kappa, seed):
    t = q * v * kappa
    rp, c, vals = A.numpy()
    rows = _out_rows(A.n, q, v, kappa, seed)
    w = 1.0 / np.sqrt(kappa)
    rid = np.repeat(np.arange(A.n), np.diff(rp))
    absA = np.zeros((t, A.d))
    absb = np.zeros(t)
    for bidx in range(kappa):
        np.add.at(absA, (rows[bidx][rid], c), w * np.abs(vals.astype(np.float64)))
        if b is not None:
            np.add.at(absb, rows[bidx], w * np.abs(b.double().numpy()))
    return absA, absb


def _check(got, want, absum, what):
    got = got.detach().cpu().double().numpy()
    err = np.abs(got - want)
    bound = TOL * absum + 1e-30
    bad = err > bound
    assert not bad.any(), "%s: %d entries out of tolerance, worst err %.3g vs bound %.3g" % (
        what, int(bad.sum()), float(err[bad].max()), float(bound[bad].min()))


def _run(cw, A, b, q, v, kappa, seed):
    SA, Sb = cw.cw_sketch_csr_general(A.to("cuda"), b.cuda() if b is not None else None, q, v, kappa, seed)
    cw.device_status()
    SA_o, Sb_o = oracle.sketch_csr_general(A.row_ptr, A.col, A.val, A.d, b, q, v, kappa, seed)
    absA, absb = _bounds(A, b, q, v, kappa, seed)
    _check(SA, SA_o, absA, "SA")
    if b is not None:
        _check(Sb, Sb_o, absb, "Sb")
    return SA, Sb


@pytest.mark.parametrize("n,d,k,q,v,kappa,seed", [
    (50001, 64, 8, 64, 16, 4, 3),      # q v a power of two, ragged last tile
    (30011, 17, 5, 37, 11, 3, 8),      # q v = 407, not a power of two
    (20000, 12, 4, 1, 32, 1, 4),       # one block, one inner sketch
    (9000, 8, 3, 300, 2, 9, 2),        # many blocks of 2 rows, kappa = 9
    (4000, 33, 33, 5, 7, 2, 6),        # rows longer than 32 lanes
    (120000, 256, 16, 1024, 16, 4, 1), # the bench's q, v, kappa
    (40000, 24, 6, 50, 9, 8, 11),      # kappa = 8
    (30000, 40, 5, 8, 512, 4, 12),     # wide inner sketches (v kappa = 2048 rows a block)
])
def test_general_shapes(cw, n, d, k, q, v, kappa, seed):
    A = W.csr_uniform(n, d, k, seed=seed + 40)
    b, _ = W.rhs(A, 0.3, seed=seed + 41)
    _run(cw, A, b, q, v, kappa, seed)


def test_general_ragged_empty_rows_no_b(cw):
    A = W.csr_random_lengths(25000, 40, 0, 30, seed=5, empty_frac=0.3)
    SA, Sb = _run(cw, A, None, 20, 8, 3, 13)
    assert Sb is None


def test_general_wide_rows(cw):
    A = W.csr_random_lengths(3000, 5000, 10, 80, seed=4)
    b, _ = W.rhs(A, 0.5, seed=5)
    _run(cw, A, b, 4, 4, 2, 12)


def test_general_q1_kappa1_equals_section2_sketch(cw):
    A = W.csr_zipf(80000, 64, 12, 1.1, seed=3)
    b, _ = W.rhs(A, 0.1, seed=4)
    seed, v = 19, 2048
    s0 = oracle.general_seeds(seed, 1)[0]
    Ag, bg = A.to("cuda"), b.cuda()
    SA, Sb = cw.cw_sketch_csr_general(Ag, bg, 1, v, 1, seed)
    SA0, Sb0 = cw.cw_sketch_csr(Ag, bg, v, s0)
    assert torch.equal(SA, SA0) and torch.equal(Sb, Sb0)


def test_general_deterministic_and_empty(cw):
    A = W.csr_zipf(60000, 128, 16, 1.1, seed=77).to("cuda")
    b = torch.randn(A.n, device="cuda")
    r1 = cw.cw_sketch_csr_general(A, b, 16, 32, 5, 9)
    r2 = cw.cw_sketch_csr_general(A, b, 16, 32, 5, 9)
    assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])
    E = W.csr_uniform(0, 5, 0, seed=1).to("cuda")
    SA = torch.full((2 * 3 * 4, 5), 7.0, device="cuda")
    cw.cw_sketch_csr_general(E, None, 2, 3, 4, 1, SA=SA)
    torch.cuda.synchronize()
    assert float(SA.abs().max()) == 0.0


def test_general_rejects_bad_shapes(cw):
    A = W.csr_uniform(100, 4, 2, seed=1).to("cuda")
    SA = torch.zeros(8, 4, device="cuda")
    for q, v, kappa in ((1 << 10, 1 << 10, 1), (0, 4, 1), (2, 0, 1), (2, 4, 0)):
        with pytest.raises(cw.CWError):
            cw.cw_sketch_csr_general(A, None, q, v, kappa, 1, SA=SA)
