"""Host logic for running the solver on several GPUs (one process per GPU).

Runs never interact (Sec. II B: the repetitions are independent), so the
work shards by runs with no collective on the data path: every rank solves
its own runs with its own seed stream, and the only exchange is the final
reduction of the per-rank best answers (an all-gather of a few scalars and
one spin vector per rank).  Nothing here touches device memory.
"""
from __future__ import annotations

import numpy as np

SEED_STRIDE = 1_000_003  # distinct SplitMix64 key per rank


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's share of the runs (64-bit, distinct per rank)."""
    return (int(seed) + SEED_STRIDE * int(rank)) & 0xFFFFFFFFFFFFFFFF


def split_runs(R: int, world: int, rank: int):
    """Strong-scaling split of R runs: (first run, count) of this rank."""
    base, extra = divmod(int(R), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def reduce_best(energy, spins, group=None):
    """Global best over ranks of per-run best energies.

    energy: (R_local,) energies of this rank's runs; spins: (R_local, N).
    Returns (best energy, rank, local run index, spins) on every rank.  Ties
    go to the lowest rank, then the lowest run index.  With no process group
    (or world size 1) this is the local argmin."""
    energy = np.asarray(energy, dtype=np.float64)
    spins = np.asarray(spins, dtype=np.int8)
    r = int(np.argmin(energy)) if energy.size else -1
    local = (float(energy[r]) if r >= 0 else float("inf"), r)
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return local[0], 0, local[1], spins[r].copy() if r >= 0 else None
    world = dist.get_world_size(group)
    gathered = [None] * world
    dist.all_gather_object(gathered, (local[0], local[1], spins[r].tolist() if r >= 0 else None), group=group)
    best_rank = min(range(world), key=lambda k: (gathered[k][0], k, gathered[k][1]))
    e, run, s = gathered[best_rank]
    return e, best_rank, run, (np.array(s, dtype=np.int8) if s is not None else None)


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a scalar over ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
