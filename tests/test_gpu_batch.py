"""GPU parity of the batched sketch-and-solve (many independent problems of
uneven n and d in one graph launch) against the float64 oracle.

For every problem: each SA / Sb entry within 1e-5 of its bucket's absolute sum
(the sketch tolerance), x' equal to the float64 least-squares solution of the
batch's own float32 SA (the oracle's Householder QR of that SA) to 1e-9, and
the residual ratio ||A x' - b|| / ||A x* - b|| equal to the oracle's (oracle
SA, oracle QR) to 1e-6.  Edge cases: empty and rank-deficient problems,
d = 1, m = d, n < m, an ill-conditioned problem that must go to the QR
fallback, determinism, graph and direct launches agreeing, and the autotuner
with its cache file.
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


def _check_sketch(A, b, m, seed, SA, Sb):
    SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, m, seed)
    h, _ = oracle.hash(seed, m, 0, A.n)
    rp, c, v = A.numpy()
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    absA = np.zeros((m, A.d))
    np.add.at(absA, (h[rows], c), np.abs(v.astype(np.float64)))
    absb = np.zeros(m)
    np.add.at(absb, h, np.abs(b.double().numpy()))
    err = np.abs(SA.cpu().double().numpy() - SA_o)
    assert (err <= TOL * absA + 1e-30).all(), "SA out of tolerance"
    errb = np.abs(Sb.cpu().double().numpy() - Sb_o)
    assert (errb <= TOL * absb + 1e-30).all(), "Sb out of tolerance"
    return SA_o, Sb_o


def _make(shapes):
    probs, cpu = [], []
    for s in shapes:
        A, b = W.batch_problem(s)
        cpu.append((A, b, s["m"], s["seed"]))
        probs.append((A.to("cuda"), b.cuda(), s["m"], s["seed"]))
    return probs, cpu


def test_batch_matches_oracle(cw):
    shapes = W.batch_shapes(24, seed=5, log2n=(9, 13), dset=(4, 16, 33, 64, 128))
    probs, cpu = _make(shapes)
    B = cw.Batch(probs, keep_sketch=True)
    B.run()
    st = B.finish()
    assert st == [0] * len(probs), st
    for p, (A, b, m, seed) in enumerate(cpu):
        SA_o, Sb_o = _check_sketch(A, b, m, seed, B.SA[p], B.Sb[p])
        x = B.x[p].cpu().numpy()
        # the float64 least-squares solution of the batch's own float32 SA
        x_same, _ = oracle.solve_sketch(B.SA[p].cpu().double().numpy(), B.Sb[p].cpu().double().numpy())
        assert np.abs(x - x_same).max() <= 1e-9 * np.abs(x_same).max(), p
        # residual ratio against the oracle end to end
        x_o, _ = oracle.solve_sketch(SA_o, Sb_o)
        _, rstar = oracle.lstsq_exact_csr(A.row_ptr, A.col, A.val, A.d, b)
        rho = oracle.residual_ratio_csr(A.row_ptr, A.col, A.val, b, x, rstar)
        rho_o = oracle.residual_ratio_csr(A.row_ptr, A.col, A.val, b, x_o, rstar)
        assert abs(rho - rho_o) <= 1e-6 * rho_o, (p, rho, rho_o)
    B.close()


def test_batch_edge_cases(cw):
    shapes = [dict(n=0, d=8, m=64, kmin=1, kmax=8, seed=1),       # empty: rank deficient
              dict(n=5, d=8, m=64, kmin=8, kmax=8, seed=2),       # n < d: rank deficient
              dict(n=3000, d=1, m=4, kmin=1, kmax=1, seed=3),     # d = 1
              dict(n=5000, d=16, m=16, kmin=4, kmax=16, seed=4),  # m = d
              dict(n=700, d=128, m=65536, kmin=4, kmax=32, seed=5),  # n << m
              dict(n=20000, d=20, m=1600, kmin=4, kmax=20, seed=6)]
    probs, cpu = _make(shapes)
    B = cw.Batch(probs, keep_sketch=True)
    B.run()
    st = B.finish()
    assert st[0] == 4 and st[1] == 4, st
    assert all(s == 0 for s in st[2:]), st
    assert float(B.x[0].abs().max()) == 0.0
    for p in range(2, len(cpu)):
        A, b, m, seed = cpu[p]
        _check_sketch(A, b, m, seed, B.SA[p], B.Sb[p])
        x_same, _ = oracle.solve_sketch(B.SA[p].cpu().double().numpy(), B.Sb[p].cpu().double().numpy())
        x = B.x[p].cpu().numpy()
        assert np.abs(x - x_same).max() <= 1e-9 * np.abs(x_same).max(), p
    B.close()


def _collinear(n, d, eps, seed):
    """Dense-pattern CSR whose column 1 is column 0 plus eps * N(0,1)."""
    g = torch.Generator().manual_seed(seed)
    V = torch.randn(n, d, generator=g, dtype=torch.float64)
    V[:, 1] = V[:, 0] + eps * torch.randn(n, generator=g, dtype=torch.float64)
    row_ptr = (torch.arange(n + 1) * d).to(torch.int32)
    col = torch.arange(d, dtype=torch.int32).repeat(n)
    A = W.CSR(n, d, row_ptr, col, V.reshape(-1).to(torch.float32))
    b = (V @ torch.ones(d, dtype=torch.float64) + 0.1 * torch.randn(n, generator=g, dtype=torch.float64))
    return A, b.to(torch.float32)


def test_batch_ill_conditioned_problem_goes_to_the_qr(cw):
    A, b = _collinear(6000, 8, 1e-6, 3)
    A2, b2 = W.batch_problem(dict(n=6000, d=8, m=256, kmin=2, kmax=8, seed=9))
    probs = [(A.to("cuda"), b.cuda(), 256, 11), (A2.to("cuda"), b2.cuda(), 256, 9)]
    B = cw.Batch(probs, keep_sketch=True)
    B.run()
    st = B.finish()
    assert st == [3, 0], st
    for p in range(2):
        x_same, _ = oracle.solve_sketch(B.SA[p].cpu().double().numpy(), B.Sb[p].cpu().double().numpy())
        x = B.x[p].cpu().numpy()
        assert np.abs(x - x_same).max() <= 1e-6 * np.abs(x_same).max(), p
    B.close()


def test_batch_deterministic_graph_and_direct_agree(cw):
    shapes = W.batch_shapes(40, seed=8, log2n=(10, 14), dset=(16, 32, 64))
    probs, _ = _make(shapes)
    B1 = cw.Batch(probs)
    B2 = cw.Batch(probs, eager=True)
    assert B1.info()["graph"] == 1 and B2.info()["graph"] == 0
    B1.run()
    assert B1.finish() == [0] * 40
    x1 = [x.clone() for x in B1.x]
    B1.run()
    B1.finish()
    B2.run()
    B2.finish()
    for p in range(40):
        assert torch.equal(x1[p], B1.x[p])
        assert torch.equal(x1[p], B2.x[p])
    B1.close()
    B2.close()


def test_batch_autotune_and_cache(cw, tmp_path, monkeypatch):
    shapes = W.batch_shapes(16, seed=9, log2n=(10, 13), dset=(16, 64))
    probs, _ = _make(shapes)
    monkeypatch.setenv("CW_TUNE_CACHE", str(tmp_path / "tune.txt"))
    B = cw.Batch(probs, autotune=True)
    info = B.info()
    assert info["tuned"] == 1 and info["slab"] in (512, 1024, 2048, 4096)
    B.run()
    assert B.finish() == [0] * 16
    B2 = cw.Batch(probs, autotune=True)
    assert B2.info()["tuned"] == 2 and B2.info()["slab"] == info["slab"]
    B.close()
    B2.close()
