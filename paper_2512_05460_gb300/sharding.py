"""Host logic for running the path on several GPUs (one process per GPU).

Queries are independent, so a batch is sharded by contiguous query ranges
with no data-path collective (weak scaling).  A single query too large for
one GPU is split on median-of-means block boundaries (Eq. final-estimator):
rank r computes the block means of its blocks with pw_query_blocks (the same
walks the whole query would run), the means are gathered in block order to
rank 0, and pw_block_median gives the unsharded estimate bit for bit.  The
only collectives are this gather and a max over ranks of the timing.
"""

from __future__ import annotations

import numpy as np


def shard_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of `count` items owned by `rank`; sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_blocks(G: int, rank: int, world: int) -> tuple[int, int]:
    """Median-of-means blocks [g0, g1) of one query owned by `rank`."""
    return shard_range(G, rank, world)


def gather_block_means(local_means, G: int, group=None):
    """Gather every rank's block means to rank 0, in block order.  Returns the
    G means on rank 0 and None elsewhere (torch.distributed, any backend that
    supports all_gather of CPU tensors, e.g. gloo)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    g0, g1 = shard_blocks(G, rank, world)
    local = np.asarray(local_means, dtype=np.float64)
    if local.size != g1 - g0:
        raise ValueError("local block means do not match this rank's block range")
    width = -(-G // world)
    buf = torch.full((width,), float("nan"), dtype=torch.float64)
    buf[: local.size] = torch.from_numpy(local)
    parts = [torch.empty(width, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    if rank != 0:
        return None
    out = []
    for r in range(world):
        a, b = shard_blocks(G, r, world)
        out.append(parts[r][: b - a].numpy())
    return np.concatenate(out)


def sharded_query(graph_handle: int, s: int, t: int, eps: float, L: int, seed: int, G: int, params=None,
                  group=None):
    """One query split across the ranks of `group`; the estimate on rank 0."""
    import torch.distributed as dist

    from . import probewalk as pw

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    g0, g1 = shard_blocks(G, rank, world)
    local = pw.pw_query_blocks(graph_handle, s, t, eps, L, g0, g1, seed, params)
    means = gather_block_means(local, G, group)
    return pw.pw_block_median(means) if rank == 0 else None


def max_over_ranks(x: float, group=None) -> float:
    """Max of a host scalar over the ranks (the timing reduction of the bench)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
