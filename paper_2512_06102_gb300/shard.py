"""Sharding a batch of grids over ranks (one process per GPU).

Grids are independent (Section 3: each grid evolves on its own), so a batch
splits into contiguous ranges of grids with no exchange in the data path;
ranges are balanced by cell count, since the step's cost grows with cells.
The only collective is in calibration (Section 4).  Its loss is a mean over
the whole batch; each rank evaluates its share of it (the sums over its own
grids divided by the whole batch's counts), so the shares, and their
parameter gradients, add up over ranks to the whole batch's loss and
gradient.  One all-reduce per iteration carries the gradient and the loss
together; a rank whose range is empty contributes zeros.
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


def global_count(n_local: int) -> int:
    """Sum of n_local over the ranks (n_local itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return int(n_local)
    t = torch.tensor([int(n_local)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def reduce_loss_and_grad_(grad, loss) -> float:
    """Sum this rank's share of the loss and its gradient over the ranks with
    one all-reduce.  grad (float64, any device the backend takes) is
    overwritten by the sum; the summed loss is returned."""
    import torch
    buf = torch.cat([grad.reshape(-1).to(torch.float64),
                     torch.as_tensor(loss, dtype=torch.float64, device=grad.device).reshape(1)])
    allreduce_sum_(buf)
    grad.copy_(buf[:-1].reshape(grad.shape).to(grad.dtype))
    return float(buf[-1].item())
