"""Sharding of the pair set across ranks (one process per GPU).

Pairs are independent, so the forward (linking and travel times) shards by
emitter with no exchange; the adjoint is a sum over pairs, so each rank
scatters its own pairs and one all-reduce (sum) of the grid gradient
completes it. Only host-side index bookkeeping lives here.
"""
from __future__ import annotations

import numpy as np


def emitters_of(rank: int, world: int, n_tx: int) -> np.ndarray:
    """Contiguous, balanced block of emitters for `rank`."""
    if not (0 <= rank < world) or n_tx < 2:
        raise ValueError("bad rank/world/n_tx")
    lo = (n_tx * rank) // world
    hi = (n_tx * (rank + 1)) // world
    return np.arange(lo, hi)


def shard_pairs(rank: int, world: int, n_tx: int) -> np.ndarray:
    """(e, r) pairs with e in this rank's emitter block, emitter-major, int32 [P, 2]."""
    e = emitters_of(rank, world, n_tx)
    if e.size == 0:
        return np.zeros((0, 2), np.int32)
    ee = np.repeat(e, n_tx - 1)
    rr = np.tile(np.arange(n_tx - 1), e.size)
    rr = rr + (rr >= ee)
    return np.stack([ee, rr], 1).astype(np.int32)


def global_index(pairs: np.ndarray, n_tx: int) -> np.ndarray:
    """Index of each (e, r) in the emitter-major list of all pairs."""
    e, r = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    return e * (n_tx - 1) + r - (r > e)


def allreduce_sum(tensor, group=None):
    """Sum a gradient over ranks in place (torch.distributed)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
