"""Sharding a job's disorder samples over ranks, one process per GPU.

Disorder samples are independent (Sec. 2.1, Sec. 3): the replica exchange and the
Houdayer move act inside one sample.  So a job splits into contiguous sample ranges, and
no data moves between the ranks while they run.  Every random word is keyed by the
job-wide sample index (a shard's sample_offset plus the local index), so the shards
together evolve exactly as the whole job on one device.  The only collective is the
reduction of the timed region's duration to its maximum over ranks.
"""
from __future__ import annotations

import os
from typing import Tuple


def dist_env() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def weak_shard(workload, rank: int):
    """Rank `rank`'s job when every rank runs `workload.n_samples` samples: samples
    rank*S .. rank*S + S - 1 of one job of world_size * S samples."""
    return workload.with_(sample_offset=workload.sample_offset + rank * workload.n_samples)


def strong_shard(workload, world_size: int, rank: int):
    """Rank `rank`'s contiguous part of the job's samples when the job is split over
    `world_size` ranks (sizes differ by at most one sample)."""
    S = workload.n_samples
    lo, hi = rank * S // world_size, (rank + 1) * S // world_size
    return workload.with_(n_samples=hi - lo, sample_offset=workload.sample_offset + lo)


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of `x` over the ranks of the default process group (x itself when no
    group is running)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
