"""Row shards of one problem over several ranks.

The sketch is linear in the rows: S A = sum over row blocks A_k of S_k A_k,
where S_k is the block of columns of S for the rows of A_k (Section 3: column
i of S holds sigma(i) in row h(i), independently of the other rows).  A rank
sketches its contiguous block of rows with the global hash, passing the
block's first global row index i0 (cw_sketch_csr_rows), and the m x d
partials are added in rank order, so every rank holds the same sum in every
run.  Preconditioned LSQR needs one more exchange per iteration: the d-vector
A^T z and two scalars, summed the same way.

The exchange uses torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch


def row_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [r0, r1) of the n rows owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(int(n), world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def sum_in_rank_order(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of `t` over the ranks of `group`, added in rank order 0, 1, 2, ...

    All ranks gather every partial and add them in the same order, so the
    result is bitwise the same on every rank and from run to run (an
    all-reduce may add in an order that depends on the ring or tree)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out
