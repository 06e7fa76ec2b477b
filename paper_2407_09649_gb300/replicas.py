"""Multi-GPU runs of independent work (one process per GPU, no data-path collective).

GP instances and query batches are independent, so N GPUs run N replicas of the workload,
each on its own inputs (weak scaling).  The only communication is the timing barrier and
the max-over-ranks of the elapsed time, so the aggregate throughput is
    (units processed by all ranks) / (slowest rank's time).
"""
from __future__ import annotations

import os


def rank_env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(units: float, seconds: float, world_size: int, device=None):
    """Whole-job throughput: every rank's units summed, divided by the max elapsed time.
    Uses torch.distributed when world_size > 1 (any backend), else returns the local value."""
    if world_size <= 1:
        return units / seconds, seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds, units], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t[1:].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tot.item()) / float(mx.item()), float(mx.item())
