"""Sharding of a trace job over ranks (one process per GPU).

Views are independent: each rank traces a contiguous share of them with no
exchange.  The adjoint of a shared grid needs one exchange: every rank
accumulates the gradient of its own views (the mip adjoint is linear, so it
commutes with the sum) and the level-0 gradients are summed over ranks.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Contiguous share of `items` for `rank` (sizes differ by at most one)."""
    n = len(items)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return items[lo:hi]


def reduce_gradient(grad, group=None):
    """Sums a level-0 gradient tensor over the ranks of `group` in place."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
