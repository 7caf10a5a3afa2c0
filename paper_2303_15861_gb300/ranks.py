"""Placement of independent work on ranks, one process per GPU (torchrun environment).

The batched workload is a set of independent instances: each rank takes a contiguous block
of them and advances it on its own GPU, with no data exchange. Only the timing uses a
collective (the slowest rank's time, the total work), outside the timed region.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the torchrun environment (1 process by default)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, rank: int, world: int):
    """Contiguous block [lo, hi) of `count` units for `rank` of `world`; block sizes differ
    by at most one and the blocks cover every unit once."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError("bad rank, world or count")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_scalar(value: float, op: str, dist=None, device=None) -> float:
    """value reduced over the ranks ("max" or "sum"); the value itself without a process group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
