"""Host logic of the multi-GPU form: independent replicas, one process per GPU.

The transmission sum shards over (E, k, column) items with no exchange between them,
so N GPUs run N replicas of the single-GPU engine on disjoint item sets.  The only
collective is the timing: the job's time is the maximum over ranks, and the whole-job
rate is the units all ranks processed divided by that time.  Nothing here touches the
solver's data path; the functions run unchanged on the gloo backend (CPU tensors) and
on NCCL (device tensors).
"""

from __future__ import annotations

import numpy as np


def step_items(n_energy: int, reps, n_rhs: int, count: int, step: int, rank: int, world: int, seed: int = 2000):
    """Items (energy index, k index, column) of one step for one rank.

    One seeded sample of count * world distinct (E, k-representative, column) triples
    is drawn per step (the same on every rank) and rank r takes every world-th entry
    starting at r, so the ranks' items are disjoint and together form the sample.
    """
    reps = np.asarray(reps, np.int64)
    total = int(n_energy) * len(reps) * int(n_rhs)
    need = int(count) * int(world)
    if need > total:
        raise ValueError("more items than distinct (E, k, column) triples")
    rng = np.random.default_rng(seed + step)
    flat = rng.choice(total, size=need, replace=False)
    mine = flat[rank::world]
    col = mine % n_rhs
    rest = mine // n_rhs
    k = reps[rest % len(reps)]
    e = rest // len(reps)
    return e.astype(np.int64), k.astype(np.int32), col.astype(np.int64)


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the value itself
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling: every
    rank processes the same number of units)."""
    if seconds_max <= 0:
        raise ValueError("non-positive time")
    return units_per_rank * world / seconds_max
