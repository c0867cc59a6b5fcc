"""GPU parity of the batched sketch-and-solve (many independent problems of
uneven n and d in one graph launch) against the float64 oracle.

For every problem: each SA / Sb entry within 1e-5 of its bucket's absolute sum
(the sketch tolerance), x' within four times the first-order perturbation
bound of the oracle's solution (its own float64 sketch and Householder QR),
the perturbation being the float32 summation error of each SA entry, and
the residual ratio ||A x' - b|| / ||A x* - b|| equal to the oracle's (oracle
SA, oracle QR) to 1e-6.  Edge cases: empty and rank-deficient problems,
d = 1, m = d, n < m, an ill-conditioned problem that must go to the QR
fallback, determinism, graph and direct launches agreeing, and the autotuner
with its cache file.  Every variant the autotuner can choose (segmented sum
with 16 or 32 lanes per row, or over whole 16- or 8-bucket ranges; slabs of
512 and 4096 bucket rows; one or two CTAs per SM) is forced through the tune
cache and checked the same way, on a set that includes a problem of the
workload's largest shape (n = 2^18, d = 128, m = 65536).
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
    """The batch's SA, Sb against the oracle's; returns the oracle's sketch and
    the float32 rounding bounds E, Eb of the batch's entries (see _x_bound)."""
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
    # an entry of SA is a float32 sum over the rows of its bucket: in any order
    # within (k - 1) u sum |terms| of the exact sum (k rows, u = 2^-24), plus
    # the rounding of the inputs' products by the signs (exact)
    k = np.bincount(h, minlength=m).astype(np.float64)
    E = (k[:, None] * 2.0 ** -24) * absA
    Eb = k * 2.0 ** -24 * absb
    return SA_o, Sb_o, E, Eb


def _x_bound(SA_o, Sb_o, x_o, E, Eb):
    """First-order bound on |x - x_o| for x = argmin ||SA x - Sb|| when
    |SA - SA_o| <= E and |Sb - Sb_o| <= Eb entrywise:
        x - x_o ~ -P (dSA x_o - dSb) + (SA_o^T SA_o)^-1 dSA^T r_o,  P = SA_o^+,
    with r_o = Sb_o - SA_o x_o; each term bounded with absolute values."""
    P = np.linalg.pinv(SA_o)
    Ginv = np.linalg.inv(SA_o.T @ SA_o)
    r_o = Sb_o - SA_o @ x_o
    return np.abs(P) @ (E @ np.abs(x_o) + Eb) + np.abs(Ginv) @ (E.T @ np.abs(r_o))


def _check_x(x, SA_o, Sb_o, E, Eb, p):
    """x against the oracle's solve of its own sketch: within four times the
    first-order bound (second-order terms, the solver's own rounding)."""
    x_o, _ = oracle.solve_sketch(SA_o, Sb_o)
    bound = _x_bound(SA_o, Sb_o, x_o, E, Eb)
    err = np.abs(x - x_o)
    assert (err <= 4 * bound + 1e-8 * np.abs(x_o).max()).all(), (p, float((err / (bound + 1e-300)).max()))
    return x_o


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
        SA_o, Sb_o, E, Eb = _check_sketch(A, b, m, seed, B.SA[p], B.Sb[p])
        x = B.x[p].cpu().numpy()
        x_o = _check_x(x, SA_o, Sb_o, E, Eb, p)
        # residual ratio against the oracle end to end
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
        SA_o, Sb_o, E, Eb = _check_sketch(A, b, m, seed, B.SA[p], B.Sb[p])
        _check_x(B.x[p].cpu().numpy(), SA_o, Sb_o, E, Eb, p)
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
    for p, (A_, b_, m_, seed_) in enumerate(((A, b, 256, 11), (A2, b2, 256, 9))):
        SA_o, Sb_o, E, Eb = _check_sketch(A_, b_, m_, seed_, B.SA[p], B.Sb[p])
        _check_x(B.x[p].cpu().numpy(), SA_o, Sb_o, E, Eb, p)
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


# ---------------------------------------------------------------- every tuned variant against the oracle

def _fnv(h, v):
    # FNV-1a over the eight little-endian bytes of v (the tune cache's key)
    for k in range(8):
        h ^= (v >> (8 * k)) & 0xFF
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _shape_key(cpu):
    h = 1469598103934665603
    h = _fnv(h, len(cpu))
    h = _fnv(h, torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    for A, _, m, _ in cpu:
        for v in (A.n, A.d, A.nnz, m):
            h = _fnv(h, v)
    return h


_VARIANT_SET = {}


def _variant_set():
    """Problems of uneven n and d, one of them at the workload's largest shape,
    with the oracle's sketch, its bounds and solution (computed once)."""
    if not _VARIANT_SET:
        shapes = W.batch_shapes(10, seed=13, log2n=(9, 14), dset=(16, 33, 64, 128))
        shapes.append(dict(n=1 << 18, d=128, m=65536, kmin=4, kmax=32, seed=77))
        probs, cpu = _make(shapes)
        ref = []
        for A, b, m, seed in cpu:
            SA_o, Sb_o = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, m, seed)
            h, _ = oracle.hash(seed, m, 0, A.n)
            rp, c, v = A.numpy()
            rows = np.repeat(np.arange(A.n), np.diff(rp))
            absA = np.zeros((m, A.d))
            np.add.at(absA, (h[rows], c), np.abs(v.astype(np.float64)))
            absb = np.zeros(m)
            np.add.at(absb, h, np.abs(b.double().numpy()))
            k = np.bincount(h, minlength=m).astype(np.float64)
            E, Eb = (k[:, None] * 2.0 ** -24) * absA, k * 2.0 ** -24 * absb
            x_o, _ = oracle.solve_sketch(SA_o, Sb_o)
            ref.append(dict(SA_o=SA_o, Sb_o=Sb_o, absA=absA, absb=absb,
                            bound=_x_bound(SA_o, Sb_o, x_o, E, Eb), x_o=x_o))
        _VARIANT_SET.update(probs=probs, cpu=cpu, ref=ref)
    return _VARIANT_SET


@pytest.mark.parametrize("cps", [1, 2])
@pytest.mark.parametrize("slab", [512, 4096])
@pytest.mark.parametrize("lpr", [16, 32, 0, -8])
def test_batch_every_tuned_variant_matches_oracle(cw, tmp_path, monkeypatch, lpr, slab, cps):
    V = _variant_set()
    cache = tmp_path / "tune.txt"
    cache.write_text("batch %x %d %d %d\n" % (_shape_key(V["cpu"]), slab, cps, lpr))
    monkeypatch.setenv("CW_TUNE_CACHE", str(cache))
    B = cw.Batch(V["probs"], autotune=True, keep_sketch=True)
    info = B.info()
    assert info["tuned"] == 2, info  # taken from the cache, not re-tuned
    assert (info["slab"], info["ctas_per_sm"], info["lanes_per_row"]) == (slab, cps, lpr), info
    B.run()
    assert B.finish() == [0] * len(V["probs"])
    for p, R in enumerate(V["ref"]):
        err = np.abs(B.SA[p].cpu().double().numpy() - R["SA_o"])
        assert (err <= TOL * R["absA"] + 1e-30).all(), ("SA", p)
        errb = np.abs(B.Sb[p].cpu().double().numpy() - R["Sb_o"])
        assert (errb <= TOL * R["absb"] + 1e-30).all(), ("Sb", p)
        x = B.x[p].cpu().numpy()
        err_x = np.abs(x - R["x_o"])
        assert (err_x <= 4 * R["bound"] + 1e-8 * np.abs(R["x_o"]).max()).all(), ("x", p)
    B.close()
