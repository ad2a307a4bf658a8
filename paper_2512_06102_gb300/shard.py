"""Sharding a batch of grids over ranks (one process per GPU).

Grids are independent (Section 3: each grid evolves on its own), so a batch
splits into contiguous ranges of grids with no exchange in the data path;
ranges are balanced by cell count, since the step's cost grows with cells.
The only collective is the sum of the calibration gradient (Section 4): the
calibration loss is a sum over grids, so each rank differentiates the loss of
its own grids and the parameter gradients are added.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(cells_per_env, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) ranges of grids, one per rank, splitting the
    running cell count as evenly as whole grids allow (rank r's range ends at
    the first grid whose running count reaches (r + 1) / world of the total).
    Every grid lands in exactly one range; ranges may be empty when there are
    fewer grids than ranks."""
    c = np.asarray(cells_per_env, np.int64).reshape(-1)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = c.shape[0]
    cum = np.cumsum(c)
    total = int(cum[-1]) if n else 0
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left")) + 1 if n else 0
        k = min(max(k, bounds[-1]), n)
        bounds.append(k)
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def allreduce_sum_(t):
    """In-place sum over the ranks of the default process group (no-op when
    torch.distributed is not initialised or has one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
