"""Data parallelism over views for the training step.

A training step renders a set of views of one scene and differentiates a
per-view loss; the views are independent, so each rank renders its share of
them, and the one exchange step is the sum of the per-view parameter
gradients across ranks (an all-reduce).  Forward-only rendering of
independent views needs no exchange at all.  These helpers are host logic
only: the rendering and the adjoint run in the library's kernels.
"""
from __future__ import annotations

import math


def shard(items, rank: int, world: int) -> list:
    """The items rank `rank` of `world` handles: every world-th one."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return list(items)[rank::world]


def ring_view(rank: int, width: int, height: int, radius: float = 3.0, n_ring: int = 8):
    """The camera of rank `rank` on a ring around the origin (rank 0 looks
    from (radius, 0, 0)); every rank renders its own view of the scene."""
    from . import inputs
    ang = 2 * math.pi * rank / n_ring
    return inputs.look_at((radius * math.cos(ang), radius * math.sin(ang), 0.0), width, height)


def sum_gradients(grads: dict, group=None) -> dict:
    """All-reduce (sum) every gradient tensor in place, in a fixed key order
    so that all ranks issue the same sequence of collectives."""
    import torch.distributed as dist
    for k in sorted(grads):
        dist.all_reduce(grads[k], op=dist.ReduceOp.SUM, group=group)
    return grads
