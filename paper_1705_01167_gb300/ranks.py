"""Rank bookkeeping for runs over several GPUs (one process per GPU).

The sensor-model path shards by independent units (filters, particles,
maps) with no exchange between them.  A multi-GPU run is weak scaling by
default: every rank weights its own copy of the workload (drawn from a
rank-dependent seed), the ranks meet only at the barriers around the timed
region, and the whole-job throughput is the units of all ranks over the
slowest rank's time.  Strong scaling splits one workload's filters across
the ranks (`partition`, balanced by particle count; every rank holds its own
copy of the CDDT); the log-weights come back to every rank with one
all-gather into local buffers (`gather_filters`), the exchange that
resampling across ranks would need.
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


def partition(counts, world: int):
    """Split filters of the given particle counts over `world` ranks:
    largest first, each to the rank with the fewest particles so far (ties
    to the lower rank).  Returns per rank its filter indices, ascending.
    The heaviest rank carries at most 4/3 of the best possible split plus
    one filter (the longest-processing-time bound)."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for f in sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(f)
        load[r] += int(counts[f])
    return [sorted(o) for o in out]


def gather_filters(world: int, rank: int, parts, counts, local, device="cpu"):
    """Every filter's values on every rank: `local` holds this rank's filters
    (parts[rank], in that order, counts[f] values each, concatenated); the
    result holds all filters in filter order.  One all-gather of equal-sized
    local buffers (padded to the largest rank's share)."""
    import torch
    if world <= 1:
        return local
    import torch.distributed as dist
    sizes = [sum(int(counts[f]) for f in parts[r]) for r in range(world)]
    cap = max(sizes)
    buf = torch.zeros(cap, dtype=local.dtype, device=device)
    buf[:local.numel()] = local.reshape(-1).to(device)
    got = [torch.empty(cap, dtype=local.dtype, device=device) for _ in range(world)]
    dist.all_gather(got, buf)
    starts = [0]
    for c in counts:
        starts.append(starts[-1] + int(c))
    out = torch.empty(starts[-1], dtype=local.dtype, device=device)
    for r in range(world):
        off = 0
        for f in parts[r]:
            out[starts[f]:starts[f + 1]] = got[r][off:off + int(counts[f])]
            off += int(counts[f])
    return out
