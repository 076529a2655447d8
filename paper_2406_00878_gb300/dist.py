"""Replica runs on several GPUs of one node (one process per GPU).

A single all-at-once solve does not shard: its level chain is sequential in time and a
spatial split would need a halo exchange across GPUs in every sweep. Independent
problems do: runs with N > 1 give every rank its own problems (replicas of the
benchmark workload, or a round-robin share of a batch) and exchange nothing on the data
path. The only collectives are the barrier around the timed region and the maximum
of the per-rank times (the job takes as long as its slowest rank).
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def env() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, rank: int, world_size: int) -> List[int]:
    """Indices of the items rank `rank` owns: i = rank, rank + N, rank + 2N, ..."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError(f"rank {rank} outside a world of {world_size}")
    return list(range(rank, count, world_size))


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the value itself without a process group).
    `device`: where the reduction tensor lives (a CUDA device for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def job_throughput(units_per_rank: Sequence[float], seconds_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    if not seconds_max > 0:
        raise ValueError("time must be positive")
    return float(sum(units_per_rank)) / seconds_max
