"""Rank bodies for the two-rank gloo tests (imported by spawned processes)."""
import json
import os

import numpy as np
import torch
import torch.distributed as dist


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = os.environ["LOCAL_RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def sharded_sketch(rank, world, port, out_dir):
    """Oracle partial sketches of each rank's rows, summed in rank order."""
    import oracle
    import workloads as W
    from paper_1207_6365_gb300 import shards
    _init(rank, world, port)
    A = W.csr_random_lengths(30001, 24, 0, 12, seed=5, empty_frac=0.1)
    b, _ = W.rhs(A, 0.1, seed=6)
    m, seed = 777, 3
    r0, r1 = shards.row_range(A.n, world, rank)
    P = A.rows(r0, r1)
    SA_k, Sb_k = oracle.sketch_csr(P.row_ptr, P.col, P.val, A.d, b[r0:r1], m, seed, i0=r0)
    SA = shards.sum_in_rank_order(torch.from_numpy(np.ascontiguousarray(SA_k)))
    Sb = shards.sum_in_rank_order(torch.from_numpy(np.ascontiguousarray(Sb_k)))
    # LSQR's per-iteration exchange: A^T z over the row blocks
    z = torch.randn(A.n, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    g_k = oracle.csr_rmatvec(P.row_ptr, P.col, P.val, A.d, z[r0:r1].numpy())
    g = shards.sum_in_rank_order(torch.from_numpy(np.ascontiguousarray(g_k)))
    np.save(os.path.join(out_dir, "SA_%d.npy" % rank), SA.numpy())
    np.save(os.path.join(out_dir, "Sb_%d.npy" % rank), Sb.numpy())
    np.save(os.path.join(out_dir, "g_%d.npy" % rank), g.numpy())
    dist.destroy_process_group()


def bench_reductions(rank, world, port, out_dir):
    """bench.py's barrier / max-over-ranks / sum-over-ranks on gloo."""
    import bench
    _init(rank, world, port)
    bench.barrier(world)
    mx = bench.max_over_ranks(10.0 + rank, world)
    sm = bench.sum_over_ranks(100 + rank, world)
    with open(os.path.join(out_dir, "red_%d.json" % rank), "w") as f:
        json.dump({"max": mx, "sum": sm, "env": bench.dist_env()}, f)
    dist.destroy_process_group()
