"""The multi-GPU bookkeeping (weak scaling, no data-path collective) on two
gloo ranks on the CPU: per-rank inputs differ, the map does not, and the
whole-job rate is the units of all ranks over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_1705_01167_gb300 import ranks as RK
    from paper_1705_01167_gb300 import workloads as WL
    w, r, _ = RK.env()
    RK.init("gloo", w)
    wl = WL.corridor2000(steps=3, particles=64, sweep=0, seed_offset=RK.seed_offset(r))
    RK.barrier(w)
    rate = RK.whole_job_rate(w, local_units=100.0 * (r + 1), local_seconds=1.0 + r)
    out.put((r, rate, float(wl["parts"].sum()), int(wl["grid"].sum()), RK.max_over_ranks(w, 10.0 * r)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, rate0, s0, g0, m0), (r1, rate1, s1, g1, m1) = res
    assert rate0 == rate1 == pytest.approx(300.0 / 2.0)  # (100 + 200) units / max(1, 2) s
    assert g0 == g1            # the same map on every rank
    assert s0 != s1            # rank-dependent particles
    assert m0 == m1 == 10.0


def _split_worker(rank, world, port, counts, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch
    from paper_1705_01167_gb300 import ranks as RK
    w, r, _ = RK.env()
    RK.init("gloo", w)
    parts = RK.partition(counts, w)
    # this rank's "log-weights": filter f's particle i gets f * 100000 + i
    local = torch.cat([torch.arange(counts[f], dtype=torch.float64) + 100000.0 * f for f in parts[r]]) \
        if parts[r] else torch.zeros(0, dtype=torch.float64)
    full = RK.gather_filters(w, r, parts, counts, local)
    out.put((r, parts, full.numpy()))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_partition_covers_and_balances():
    """Every filter goes to exactly one rank, and the heaviest rank carries
    no more than the longest-processing-time bound (4/3 of the mean share
    plus one filter)."""
    from paper_1705_01167_gb300 import ranks as RK
    rs = np.random.default_rng(12)
    for world in (1, 2, 3, 4, 8):
        for n in (1, 5, 64, 200):
            counts = rs.integers(500, 10001, n)
            parts = RK.partition(counts, world)
            flat = sorted(f for p in parts for f in p)
            assert flat == list(range(n))
            loads = [int(sum(counts[f] for f in p)) for p in parts]
            assert max(loads) <= 4 / 3 * counts.sum() / world + counts.max()
            if n >= 8 * world:
                assert max(loads) <= 1.05 * counts.sum() / world + counts.max() / 2
    # equal filters deal out round-robin
    assert RK.partition([10] * 6, 3) == [[0, 3], [1, 4], [2, 5]]


def test_split_filters_gather_on_two_gloo_ranks():
    """Strong scaling on two gloo ranks: the 64 filters of the batched
    workload's particle counts split by partition, each rank's values, and
    the all-gather that returns every filter's values to every rank in
    filter order."""
    counts = [int(m) for m in np.random.default_rng(13).integers(500, 10001, 64)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, counts, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.concatenate([np.arange(c, dtype=np.float64) + 100000.0 * f for f, c in enumerate(counts)])
    assert res[0][1] == res[1][1]
    assert sorted(res[0][1][0] + res[0][1][1]) == list(range(64))
    for _, _, full in res:
        assert np.array_equal(full, want)


def test_single_rank_is_identity():
    from paper_1705_01167_gb300 import ranks as RK
    assert RK.whole_job_rate(1, 50.0, 2.0) == 25.0
    assert RK.max_over_ranks(1, 3.0) == 3.0
    assert RK.seed_offset(0) == 0
