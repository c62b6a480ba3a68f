"""Rank bookkeeping for runs over several GPUs (one process per GPU).

The sensor-model path shards by independent units (filters, particles,
maps) with no exchange between them, so a multi-GPU run is weak scaling:
every rank weights its own copy of the workload (drawn from a rank-dependent
seed), the ranks meet only at the barriers around the timed region, and the
whole-job throughput is the units of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def seed_offset(rank: int) -> int:
    """Seed offset of a rank's workload: rank 0 draws the single-GPU inputs."""
    return rank


def init(backend: str, world: int):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world: int, value: float, device="cpu") -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world: int, value: float, device="cpu") -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(world: int, local_units: float, local_seconds: float, device="cpu") -> float:
    """Units of all ranks per second of the slowest rank."""
    units = sum_over_ranks(world, local_units, device)
    seconds = max_over_ranks(world, local_seconds, device)
    return units / seconds
