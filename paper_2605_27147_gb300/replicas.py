"""Replica bookkeeping for runs on several GPUs of one node.

A single instance's merge tree does not shard without an exchange step, so
several GPUs run independent replicas: every rank sorts its own inputs (a
fixed amount of work per GPU: weak scaling) and there is no collective on the
data path.  The only cross-rank steps are the timing ones here: the job's time
is the slowest rank's, and the job's rate counts the units every rank did.
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The largest of every rank's `ms` (this rank's own value without a
    process group).  `device` is where the reduction tensor lives: the rank's
    GPU for NCCL, None (CPU) for gloo."""
    if dist is None:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, job_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    if job_ms <= 0.0:
        raise ValueError("the job's time must be positive")
    return units_per_rank * world / (job_ms / 1000.0)


def replica_seed(base: int, rank: int) -> int:
    """Seed of a rank's inputs when replicas should sort different data."""
    return base + 1_000_003 * rank
