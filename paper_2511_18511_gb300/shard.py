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


def shard_pairs(rank: int, world: int, n_tx: int, longest_first: bool = False) -> np.ndarray:
    """(e, r) pairs with e in this rank's emitter block, int32 [P, 2]:
    emitter-major, or with longest_first ordered by ring offset from the
    diameter outwards (the longest chords first, as the library's queue serves
    the implicit all-pairs list), so that a linking launch ends on its
    shortest rays."""
    e = emitters_of(rank, world, n_tx)
    if e.size == 0:
        return np.zeros((0, 2), np.int32)
    ee = np.repeat(e, n_tx - 1)
    rr = np.tile(np.arange(n_tx - 1), e.size)
    rr = rr + (rr >= ee)
    pairs = np.stack([ee, rr], 1).astype(np.int32)
    if longest_first:
        off = (pairs[:, 1] - pairs[:, 0]) % n_tx
        far = np.minimum(off, n_tx - off)          # ring distance: n_tx / 2 is the diameter
        pairs = pairs[np.lexsort((pairs[:, 0], -far))]
    return pairs


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



class ShardedToF:
    """One ToF inversion step (link + misfit adjoint) of a single problem
    split over ranks by emitter: every rank links and back-projects its own
    pairs, and one all-reduce (sum) of the grid gradient completes the step.

    link(pairs, c) -> (theta, tof) and adjoint(pairs, c, theta, tof, tof_meas)
    -> g (the gradient of the misfit with residual tof - tof_meas) are the
    per-rank operators (the CUDA library's on GPUs, the oracle's in the CPU
    tests), so that both run this same step."""

    def __init__(self, rank: int, world: int, n_tx: int, link=None, adjoint=None, allreduce=allreduce_sum,
                 link_adjoint=None):
        self.rank, self.world, self.n_tx = rank, world, n_tx
        self.pairs = shard_pairs(rank, world, n_tx, longest_first=True)
        self.link, self.adjoint, self.allreduce = link, adjoint, allreduce
        # optional fused operator link_adjoint(pairs, c, tof_meas) -> (theta, tof, g)
        self.link_adjoint = link_adjoint

    def step(self, c, tof_meas):
        """tof_meas: measured times of this rank's pairs (in self.pairs order);
        returns (g summed over ranks, theta, tof) of the misfit 0.5 |T - T_meas|^2."""
        if self.link_adjoint is not None:
            theta, tof, g = self.link_adjoint(self.pairs, c, tof_meas)
        else:
            theta, tof = self.link(self.pairs, c)
            g = self.adjoint(self.pairs, c, theta, tof, tof_meas)
        return self.allreduce(g), theta, tof
