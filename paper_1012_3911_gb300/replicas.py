"""Multi-GPU bookkeeping of the benchmark: independent replicas.

A single lattice would shard only through an all-to-all transpose between the
real-space and momentum-space passes; independent problems shard with no
data-path collective.  So on N GPUs every rank propagates its own copy of the
workload (weak scaling), the ranks meet only at barriers around the timed
region, and the job's time is the slowest rank's.  These helpers hold that
logic so that it can be exercised with CPU (gloo) process groups.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The maximum of a per-rank number (time) over all ranks; `dist` is
    torch.distributed with an initialised group, or None for one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, split_steps: int, bench_steps: int, world: int, max_ms: float) -> float:
    """Whole-job grid-pt-steps/s: the points all ranks advanced, over the
    slowest rank's time."""
    if max_ms <= 0:
        raise ValueError("time must be positive")
    return world * points_per_rank * split_steps * bench_steps / (max_ms * 1e-3)
