"""Replica runs on several GPUs of one node.

The hot path shards by source and mode with no exchange between fields, so a
multi-GPU job runs one replica of the workload per rank (weak scaling) and
only its timing is combined: the job time is the slowest rank's, and the job
throughput counts every rank's fields.
"""
from __future__ import annotations


def job_throughput(local_seconds: float, units_per_rank: int, group=None, device=None):
    """(units/s of the whole job, slowest rank's seconds).

    Without an initialised process group this is the single-process value."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units_per_rank / local_seconds, local_seconds
    world = dist.get_world_size(group)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    slowest = float(t.item())
    return world * units_per_rank / slowest, slowest


def shard(items, rank: int, world: int):
    """Contiguous, balanced slice of ``items`` for ``rank`` (sizes differ by <= 1)."""
    n = len(items)
    lo = rank * n // world
    hi = (rank + 1) * n // world
    return items[lo:hi]
