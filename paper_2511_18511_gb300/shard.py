"""Sharding across ranks (one process per GPU).

ToF: pairs are independent, so the forward (linking and travel times) shards
by emitter with no exchange; the adjoint is a sum over pairs, so each rank
scatters its own pairs and one all-reduce (sum) of the grid gradient
completes it.

Ray-Born: the frequencies are independent, so each rank holds every
transducer's maps and applies the Born map for its own block of frequencies;
one all-gather assembles d[f, e, r]. The adjoint is a sum over frequencies,
so each rank back-projects its block of the data and one all-reduce (sum) of
the grid perturbation completes it. Only host-side bookkeeping lives here.
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


def frequencies_of(rank: int, world: int, n_freq: int) -> np.ndarray:
    """Contiguous, balanced block of frequency indices for `rank` (empty when
    there are fewer frequencies than ranks)."""
    if not (0 <= rank < world) or n_freq < 0:
        raise ValueError("bad rank/world/n_freq")
    lo = (n_freq * rank) // world
    hi = (n_freq * (rank + 1)) // world
    return np.arange(lo, hi)


def allgather_frequencies(local, n_freq: int, group=None):
    """Assemble the per-rank blocks d[f_block, ...] (complex or real tensors, the
    blocks of frequencies_of in rank order) into d[n_freq, ...] on every rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return local
    world = dist.get_world_size(group)
    sizes = [len(frequencies_of(r, world, n_freq)) for r in range(world)]
    width = max(sizes)
    real = torch.view_as_real(local) if local.is_complex() else local
    pad = torch.zeros((width,) + tuple(real.shape[1:]), dtype=real.dtype, device=real.device)
    pad[: real.shape[0]] = real
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    full = torch.cat([p[:n] for p, n in zip(parts, sizes)])
    return torch.view_as_complex(full.contiguous()) if local.is_complex() else full

