"""Two ranks on CPU (gloo): the row-shard semantics of the sketch and of
LSQR's per-iteration exchange, and bench.py's cross-rank timing reductions.

Each rank sketches its contiguous block of rows with the global row index
(the float64 oracle stands in for the GPU kernels, which run one per box);
the partials summed in rank order must equal the sketch of the whole matrix,
and be bitwise identical on both ranks.
"""
import json
import multiprocessing as mp
import os
import socket

import numpy as np

import oracle
import workloads as W
import _multirank_workers as workers


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(target, world, out_dir):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, str(out_dir))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]


def test_row_range_partitions():
    from paper_1207_6365_gb300 import shards
    for n, world in ((10, 3), (0, 2), (7, 7), (5, 8), (2**24 + 1, 4)):
        got = [shards.row_range(n, world, r) for r in range(world)]
        assert got[0][0] == 0 and got[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
        sizes = [r1 - r0 for r0, r1 in got]
        assert max(sizes) - min(sizes) <= 1


def test_sharded_sketch_two_ranks(tmp_path):
    _run(workers.sharded_sketch, 2, tmp_path)
    A = W.csr_random_lengths(30001, 24, 0, 12, seed=5, empty_frac=0.1)
    b, _ = W.rhs(A, 0.1, seed=6)
    SA, Sb = oracle.sketch_csr(A.row_ptr, A.col, A.val, A.d, b, 777, 3)
    for name, full in (("SA", SA), ("Sb", Sb)):
        r0 = np.load(tmp_path / ("%s_0.npy" % name))
        r1 = np.load(tmp_path / ("%s_1.npy" % name))
        assert np.array_equal(r0, r1)                      # same bits on both ranks
        np.testing.assert_allclose(r0, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    import torch
    z = torch.randn(A.n, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    g = oracle.csr_rmatvec(A.row_ptr, A.col, A.val, A.d, z.numpy())
    g0, g1 = np.load(tmp_path / "g_0.npy"), np.load(tmp_path / "g_1.npy")
    assert np.array_equal(g0, g1)
    np.testing.assert_allclose(g0, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


def test_bench_reductions_two_ranks(tmp_path):
    _run(workers.bench_reductions, 2, tmp_path)
    for r in range(2):
        res = json.load(open(os.path.join(tmp_path, "red_%d.json" % r)))
        assert res["max"] == 11.0 and res["sum"] == 201.0
        assert res["env"] == [2, r, r]
