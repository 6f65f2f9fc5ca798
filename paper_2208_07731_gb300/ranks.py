"""Host logic of runs with one process per GPU (torchrun): every rank decomposes
its own orbital pair (independent problems, like the k-points or spin channels
of one system), so the data path has no collective; only the timing crosses
ranks: the job's time is the maximum over ranks and its throughput counts the
units of all ranks."""
from __future__ import annotations

import dataclasses
import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (1 process without one)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_workload(base, rank: int):
    """The rank's own problem: the same sizes with the seed offset by 1000 per rank."""
    return dataclasses.replace(base, seed=base.seed + 1000 * int(rank))


def max_over_ranks(x: float, device=None) -> float:
    """max of x over the ranks of the default process group (x itself without one)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling: fixed work per rank)."""
    return float(units_per_rank) * int(world) / float(max_seconds)
