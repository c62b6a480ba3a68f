"""Benchmark: CDDT ray casts per second fused with the beam sensor model.

Default workload (`--workload corridor2000`): a seeded 2000 x 2000
recursive-division map (walls 1-3 cells, doors 3-20, ~8 % occupied),
theta_disc = 200, max range 1000 cells.  A ground-truth pose random-walks for
200 filter steps; each step has 2500 particles drawn around it and its own
61-beam, 270-degree scan.  One benchmark step weights all 200 filter steps
(500,000 particles x 61 beams = 30.5 M ray casts) in one persistent batched
launch; the CDDT (288 MB with its search trees) is resident in HBM and L2
is flushed (a 256 MB write) between steps.  Extra keys report the same work
as 200 per-filter launches, as a CUDA graph, with the binary-search layout,
on the pruned CDDT and on the 16-bit store, with uniform particles, as a
full filter step (motion, sensor model, resampling), end to end from
page-locked host buffers, a 10 M-query random and a 50 M-state grid sweep
with per-warp latency, the paper's comparison casters (lookup table, ray
marching, Bresenham) on both samples (`methods`), one filter step of the
paper's one-robot setting through the C ABI (`single_filter_step`), the CPU
oracle, and compact measurements of the other four configurations
(`configs`: rects256, batched64, diff2000, update4000; skip with
--no-configs).  `roofline.binding` states the fused kernel's fraction of the
limit that binds it (the L1 data pipe), from ncu's wavefront count on the
current kernel source.
`clocks` summarises timestamped nvidia-smi samples (every 200 ms, or
CDDT_CLOCKS_MS; raw samples kept in CDDT_CLOCKS_DIR when set) over the
timed region, or the nearest ones when the region is shorter than the
sampling period (`clocks.basis`).

Other workloads (same JSON line, `config.name` names them):
  rects256      256 x 256 rectangles, theta_disc 108: one 1000-particle filter
  batched64     64 maps 512^2..4096^2, theta_disc 100..360, 500..10000
                particles each: one persistent launch vs 64 per-filter launches
  diff2000      forward + adjoint, 4096 x 61 and 1024 x 1081 beams, with 10
                gradient refinement steps, in one launch (cddt_plan_refine),
                beside the step-by-step loop
  update4000    4000 x 4000, theta_disc 360: 10^4 cell writes through
                cddt_update_cells, then 100,000 particles x 61 beams

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl {cddt,reference}]

`--impl reference` times the CPU oracle (the paper's plain CDDT: sorted
bins, binary search, float64 beam model) on the default workload on the
host cores.  Under torchrun every rank runs its own copy of the workload
(particles drawn from a rank-dependent seed: weak scaling) and the step time
is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1705_01167_gb300 import synth, workloads as WL  # noqa: E402

METRIC = "ray casts/s fused w/ sensor model on 1 GB300, % of L2/HBM gather roofline"
UNIT = "ray casts/s"
WORKLOAD_TEXT = {
    "corridor2000": ("corridor 2000x2000 (~8% occupied, walls 1-3, doors 3-20), theta_disc 200, max range 1000; "
                     "200 filter steps x 2500 particles x 61 beams (270 deg) per benchmark step, one batched launch"),
    "rects256": "rectangles 256x256 (~17% occupied), theta_disc 108, max range 300; 1000 particles x 61 beams",
    "batched64": ("64 corridor maps 512^2..4096^2, theta_disc 100..360, 500..10000 particles x 61 beams each; "
                  "one persistent launch"),
    "diff2000": ("corridor 2000x2000, theta_disc 200; forward + adjoint for 4096 x 61 and 1024 x 1081 beams "
                 "with 10 gradient refinement steps (11 evaluations), one launch"),
    "update4000": ("corridor 4000x4000, theta_disc 360, max range 1000; 10^4 cell writes per step through "
                   "cddt_update_cells, then 100,000 particles x 61 beams"),
}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # the raw samples go to CDDT_CLOCKS_DIR when set (to keep them), else
        # to the temporary directory; the JSON line carries their summary
        out_dir = os.environ.get("CDDT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms",
                                          os.environ.get("CDDT_CLOCKS_MS", "200")],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, window=None):
        """Median SM clock and active throttle reasons over the samples taken
        inside `window` (wall-clock start and end of the timed region); when
        the region is shorter than the sampling period and holds none, over
        the last sample before it and the first after it (said in "basis")."""
        import datetime
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                t = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((t, float(p[2]), float(p[3]),
                             [n for n, v in zip(names, p[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        basis = "all samples"
        use = rows
        if window is not None:
            t0, t1 = window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if inside:
                use, basis = inside, "samples inside the timed region"
            else:
                before = [r for r in rows if r[0] < t0][-1:]
                after = [r for r in rows if r[0] > t1][:1]
                if before or after:
                    use, basis = before + after, "nearest samples before and after the timed region"
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted({n for r in use for n in r[3]}), "samples": len(use), "basis": basis,
                "region_ms": None if window is None else round(1e3 * (window[1] - window[0]), 3)}


# ------------------------------------------------------------------ roofline helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Device-code files that define each profiled kernel; a recorded ncu traffic
# figure is reported only while these files are unchanged.
KERNEL_SOURCES = {
    "batched_kernel": ("cddt_internal.cuh", "cddt_sensor.cuh", "cddt_batched_f32.cu"),
    "calc_range_kernel": ("cddt_internal.cuh", "cddt_query.cu"),
    "refine_kernel": ("cddt_internal.cuh", "cddt_sensor.cuh", "cddt_refine.cu"),
}
# recorded workloads of the same kernel (another launch shape or input)
KERNEL_OF = {"batched_kernel_uniform": "batched_kernel"}


def kernel_source_sha(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1705_01167_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded(kernel: str):
    """The committed ncu counts of a profiled kernel (profiles/traffic.json),
    when they were taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("source_sha") != kernel_source_sha(KERNEL_OF.get(kernel, kernel)):
        return None
    return d


def recorded_traffic(kernel: str, launch_units: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch's units, when it was taken on the current kernel source."""
    d = recorded(kernel)
    return None if d is None else d["dram_bytes_per_unit"] * launch_units


def algorithmic_bytes(work: dict, P: int) -> int:
    """Algorithmic bytes of one sensor launch: per search 8 B of bin offsets
    plus 4 B per probe of a sorted binary search (ceil(log2(k_b + 1)) probes),
    4 B per paired reverse beam, 12 B pose + 1 B occupancy + 4 B log-weight
    per particle."""
    return 8 * work["traversals"] + 4 * work["probes"] + 4 * work["paired"] + 17 * P


def sector_bytes(work: dict, P: int) -> int:
    """Sector bytes of one sensor launch: 32 B per sector a sorted-CSR binary
    search touches (the bin's offsets, the probes while the range spans more
    than one sector, the last sector) plus 17 B per particle."""
    return 32 * work["sectors"] + 17 * P


def gather_bandwidth(G, torch, dev):
    """Random 32-byte sector gather bandwidth (GB/s) of HBM (a 4 GiB buffer,
    well beyond L2) and of L2 (a 32 MiB buffer), timed with CUDA events."""
    out = {}
    for name, nbytes, reads in (("hbm", 4 << 30, 1 << 27), ("l2", 32 << 20, 1 << 27)):
        buf = torch.empty(nbytes // 4, dtype=torch.int32, device=dev).fill_(1)
        sink = torch.zeros(1, dtype=torch.int64, device=dev)
        G.gather_probe(buf, reads, 7, sink)
        torch.cuda.synchronize()
        ts = []
        for i in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            G.gather_probe(buf, reads, 11 + i, sink)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = reads * 32 / (statistics.median(ts) * 1e-3) / 1e9
        del buf
    torch.cuda.empty_cache()
    return out


def add_work(acc: dict, w: dict):
    for k, v in w.items():
        acc[k] = acc.get(k, 0) + v
    return acc


# ------------------------------------------------------------------ ranks

from paper_1705_01167_gb300 import ranks as RK  # noqa: E402


def dist_setup():
    world, rank, local = RK.env()
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        RK.init("nccl", world)
    return world, rank, local


def barrier(world):
    RK.barrier(world)


def max_over_ranks(world, v: float) -> float:
    return RK.max_over_ranks(world, v, device="cuda")


class Timer:
    """Device time of a step with CUDA events on the launching stream, L2
    flushed (a 256 MB write) before every step, barriers around the region."""

    def __init__(self, world, dev):
        import torch
        self.torch = torch
        self.world = world
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def __call__(self, fn, k, w):
        torch = self.torch
        stream = torch.cuda.current_stream()
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        barrier(self.world)
        torch.cuda.synchronize()
        t0 = time.time()
        for i in range(k):
            self.flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        self.window = (t0, time.time())
        barrier(self.world)
        return [a.elapsed_time(b) for a, b in ev]


def host_cpu() -> dict:
    """The timing host's CPU: logical cores and the model lscpu reports."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": os.uname().machine}


def base_line(args, world, value, ms_step, workload, extra_config=None):
    cfg = {"workload": WORKLOAD_TEXT[workload], "name": workload, "l2": "flushed between steps (256 MB write)",
           "inputs": "resident in HBM"}
    if extra_config:
        cfg.update(extra_config)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": getattr(args, "scaling", "weak") if workload == "corridor2000" else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg}


# ------------------------------------------------------------------ oracle arm

def cpu_oracle_run(o, parts, bo, obs, steps, cores, max_range):
    """The CPU oracle (sorted bins, binary search, float64 beam model) over
    `steps` filter steps on `cores` host threads: (seconds, ray casts)."""
    from oracle import oracle as O
    m = O.beam_model(max_range)
    t0 = time.perf_counter()
    for t in range(steps):
        o.sensor_weights(parts[t], bo, obs[t], m, nthreads=cores)
    return time.perf_counter() - t0, steps * parts.shape[1] * bo.size


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    w = WL.corridor2000(sweep=0)
    o = O.OracleCDDT(w["grid"], w["theta_disc"], w["max_range"])
    r = o.calc_range(WL.gt_queries(w["gt"], w["beam_off"]), nthreads=cores).reshape(len(w["gt"]), -1)
    obs = np.clip(r + w["noise"], 0, w["max_range"]).astype(np.float32)
    sample = 40  # filter steps per benchmark step: a bounded sample of the 200
    for _ in range(args.warmup):
        cpu_oracle_run(o, w["parts"], w["beam_off"], obs, sample, cores, w["max_range"])
    tot, rays = 0.0, 0
    for _ in range(args.steps):
        dt, n = cpu_oracle_run(o, w["parts"], w["beam_off"], obs, sample, cores, w["max_range"])
        tot += dt
        rays += n
    value = rays / tot
    line = base_line(args, 1, value, 1e3 * tot / args.steps, "corridor2000",
                     {"sample": f"{sample} of 200 filter steps per benchmark step"})
    line.update({"impl": "reference", "n_gpus": args.gpus,
                 "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"{sample} filter steps x 2500 particles x 61 beams per step"},
                 "cpu_host": host_cpu(),
                 "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU workloads

def bench_corridor(args, G, torch, dev, world, rank):
    w = WL.corridor2000(seed_offset=RK.seed_offset(rank))
    bo, D, mr = w["beam_off"], w["D"], w["max_range"]
    S, P = w["parts"].shape[:2]
    B = bo.size
    grid = torch.from_numpy(w["grid"]).to(dev)
    t0 = time.perf_counter()
    d = G.CDDT(grid, w["theta_disc"], mr)
    torch.cuda.synchronize()
    build_wall = time.perf_counter() - t0
    st0 = d.stats()
    # observations: cast from each step's ground-truth pose, plus noise
    r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], bo)).to(dev)).cpu().numpy()
    obs = np.clip(r.reshape(S, B) + w["noise"], 0, mr).astype(np.float32)
    parts_d = torch.from_numpy(w["parts"].reshape(-1, 3)).to(dev).contiguous()
    bo_d = torch.from_numpy(bo).to(dev)
    obs_d = torch.from_numpy(obs).to(dev).contiguous()
    logw_d = torch.empty(S * P, dtype=torch.float32, device=dev)
    m = G.beam_model(mr)

    def filters_for(handle, parts=None):
        parts = parts_d if parts is None else parts
        return [dict(map=handle, particles=parts[t * P:(t + 1) * P], beam_off=bo_d, obs=obs_d[t],
                     model=m, logw=logw_d[t * P:(t + 1) * P], pair_offset=D) for t in range(S)]

    plan = G.Plan(filters_for(d))
    shape = plan.autotune()
    timed = Timer(world, dev)
    rays_per_step = S * P * B
    strong = args.scaling == "strong" and world > 1
    if strong:  # this rank's share of the 200 filters (every rank holds the CDDT)
        mine = RK.partition([P] * S, world)[rank]
        plan_t = G.Plan([filters_for(d)[t] for t in mine])
        plan_t.set_shape(**shape)
    else:
        plan_t = plan
    with ClockSampler(dev.index) as clk:
        ms = timed(plan_t.run, args.steps, args.warmup)
    clocks = clk.summary(timed.window)
    ms_step = max_over_ranks(world, statistics.mean(ms))
    # whole-job rate: every rank's ray casts over the slowest rank's time
    value = (rays_per_step if strong else world * rays_per_step) / (ms_step * 1e-3)
    if strong:
        plan_t.close()

    work = {}
    for t in range(S):
        add_work(work, d.sensor_work(parts_d[t * P:(t + 1) * P], bo_d, D))
    alg = algorithmic_bytes(work, S * P)
    peak, peak_kind = measured_peaks()
    achieved = alg / (ms_step * 1e-3) / 1e9
    # the sorted-CSR sector count against this GPU's random-sector gather
    # bandwidth (the store, 288 MB, is larger than L2: the HBM figure)
    sec = sector_bytes(work, S * P)
    gbw = gather_bandwidth(G, torch, dev)

    extra = {}
    k2 = max(3, args.steps // 2)
    ms_g = timed(plan.launch_graph, k2, 2)
    extra["graph_rays_per_s"] = rays_per_step / (statistics.mean(ms_g) * 1e-3)

    # a full filter step (Section I): the odometry motion model, the sensor
    # weights of the 200 filters and low-variance resampling, on two particle
    # buffers that swap roles every step, each direction one CUDA graph
    rs_m = synth.Stream(synth.SEED_PARTICLES + 77 + RK.seed_offset(rank))
    seg_d = torch.arange(0, S * P + 1, P, dtype=torch.int64, device=dev)
    odom_d = torch.from_numpy(np.stack([rs_m.normal(S) * 0.5 + 1.0, rs_m.normal(S) * 0.1,
                                        rs_m.normal(S) * 0.02], 1).astype(np.float32)).to(dev)
    noise_d = torch.from_numpy((rs_m.normal(3 * S * P) * 0.05).astype(np.float32).reshape(-1, 3)).to(dev)
    u0_d = torch.from_numpy(rs_m.uniform(S).astype(np.float32)).to(dev)
    buf_a = parts_d.clone()
    buf_b = torch.empty_like(buf_a)
    scratch_d = torch.empty(S * P, dtype=torch.float64, device=dev)
    plans_m = [G.Plan(filters_for(d, buf)) for buf in (buf_a, buf_b)]
    for pl in plans_m:
        pl.set_shape(**shape)
        pl.run()
    graphs = []
    for src, dst, pl in ((buf_a, buf_b, plans_m[0]), (buf_b, buf_a, plans_m[1])):
        def mcl_step(src=src, dst=dst, pl=pl):
            G.motion(src, seg_d, odom_d, noise_d)
            pl.run()
            G.resample(src, logw_d, seg_d, u0_d, out=dst, scratch=scratch_d)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            mcl_step()
        torch.cuda.current_stream().wait_stream(side)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            mcl_step()
        graphs.append(gr)
    flip = [0]

    def mcl():
        graphs[flip[0]].replay()
        flip[0] ^= 1
    ms_m = timed(mcl, k2, 2)
    extra["mcl_step"] = {"ms": statistics.mean(ms_m),
                         "rays_per_s": rays_per_step / (statistics.mean(ms_m) * 1e-3),
                         "steps": "motion model + sensor weights + low-variance resampling of 200 filters x "
                                  "2500 particles, one CUDA graph"}
    for pl in plans_m:
        pl.close()
    del buf_a, buf_b, scratch_d, noise_d

    # the uniform-particle variant (global localization: each filter's
    # particles spread over the whole free space)
    upart = np.stack([synth.uniform_particles(w["grid"], P, seed=synth.SEED_PARTICLES + 5000 + t
                                              + 100000 * RK.seed_offset(rank)) for t in range(S)])
    upart_d = torch.from_numpy(upart.reshape(-1, 3)).to(dev).contiguous()
    plan_u = G.Plan([dict(map=d, particles=upart_d[t * P:(t + 1) * P], beam_off=bo_d, obs=obs_d[t], model=m,
                          logw=logw_d[t * P:(t + 1) * P], pair_offset=D) for t in range(S)])
    shape_u = plan_u.autotune()
    ms_u = timed(plan_u.run, k2, 2)
    extra["uniform_particles_rays_per_s"] = rays_per_step / (statistics.mean(ms_u) * 1e-3)
    extra["uniform_particles_shape"] = shape_u
    # its roofline: algorithmic bytes over the same HBM copy peak, and the
    # DRAM bytes ncu counted per particle (its gathers leave the caches)
    work_u = {}
    for t in range(S):
        add_work(work_u, d.sensor_work(upart_d[t * P:(t + 1) * P], bo_d, D))
    alg_u = algorithmic_bytes(work_u, S * P)
    mean_s = statistics.mean(ms_u) * 1e-3
    rec_u = recorded("batched_kernel_uniform")
    dram_u = None if rec_u is None else rec_u["dram_bytes_per_unit"] * S * P
    extra["uniform_particles_roofline"] = {
        "bound": "hbm", "achieved": alg_u / mean_s / 1e9, "peak": peak, "unit": "GB/s",
        "frac": alg_u / mean_s / 1e9 / peak, "traffic": dram_u, "peak_kind": peak_kind,
        "algorithmic_bytes_per_launch": alg_u, "sector_bytes_per_launch": sector_bytes(work_u, S * P),
        "dram_gbs": None if dram_u is None else dram_u / mean_s / 1e9,
        "dram_frac": None if dram_u is None else dram_u / mean_s / 1e9 / peak}
    plan_u.close()

    def sequential():
        for t in range(S):
            d.sensor_weights(parts_d[t * P:(t + 1) * P], bo_d, obs_d[t], m, D, logw=logw_d[t * P:(t + 1) * P])
    ms_s = timed(sequential, k2, 2)
    extra["sequential_rays_per_s"] = rays_per_step / (statistics.mean(ms_s) * 1e-3)
    extra["batched_speedup_vs_sequential"] = statistics.mean(ms_s) / statistics.mean(ms)

    # one filter step of the paper's one-robot setting (Section VI: 2500
    # particles x 61 beams, 40 Hz on one CPU thread there), through the C ABI:
    # a one-filter plan launched as a CUDA graph (device time per step), the
    # same with the motion model and resampling in the graph, and the wall
    # time of one cddt_sensor_weights call from the host to its completion
    f0 = filters_for(d)[0]
    plan1 = G.Plan([f0])
    shape1 = plan1.autotune()
    ms1 = timed(plan1.launch_graph, 50, 5)
    seg1 = torch.tensor([0, P], dtype=torch.int64, device=dev)
    odo1, u01 = odom_d[:1].contiguous(), u0_d[:1].contiguous()
    src1 = parts_d[:P].clone()
    dst1 = torch.empty_like(src1)
    noise1 = torch.from_numpy((rs_m.normal(3 * P) * 0.05).astype(np.float32).reshape(-1, 3)).to(dev)
    scr1 = torch.empty(P, dtype=torch.float64, device=dev)
    plan1m = G.Plan([dict(f0, particles=src1)])
    plan1m.set_shape(**shape1)

    def step1():
        G.motion(src1, seg1, odo1, noise1)
        plan1m.run()
        G.resample(src1, f0["logw"], seg1, u01, out=dst1, scratch=scr1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step1()
    torch.cuda.current_stream().wait_stream(side)
    gr1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr1):
        step1()
    ms1m = timed(gr1.replay, 50, 5)
    for _ in range(20):
        d.sensor_weights(f0["particles"], bo_d, f0["obs"], m, D, logw=f0["logw"])
    torch.cuda.synchronize()
    n_calls = 200
    t0 = time.perf_counter()
    for _ in range(n_calls):
        d.sensor_weights(f0["particles"], bo_d, f0["obs"], m, D, logw=f0["logw"])
        torch.cuda.synchronize()
    call_us = (time.perf_counter() - t0) / n_calls * 1e6
    extra["single_filter_step"] = {
        "particles": P, "beams": B, "sensor_graph_us": statistics.mean(ms1) * 1e3,
        "mcl_step_graph_us": statistics.mean(ms1m) * 1e3, "sensor_call_wall_us": call_us,
        "shape": shape1, "steps_per_s_graph": 1e3 / statistics.mean(ms1),
        "note": "device time per CUDA-graph launch (L2 flushed before each); the call's wall time includes "
                "the Python binding, the C-ABI argument checks, the launch and a stream synchronize"}
    plan1.close()
    plan1m.close()
    del src1, dst1, noise1, scr1

    d.set_search(G.SEARCH_BINARY)
    ms_b = timed(plan.run, k2, 2)
    extra["binary_search_launch_groups"] = plan.groups()
    d.set_search(G.SEARCH_TREE)
    extra["binary_search_rays_per_s"] = rays_per_step / (statistics.mean(ms_b) * 1e-3)

    sw = torch.from_numpy(w["sweep"]).to(dev)
    out = torch.empty(sw.shape[0], dtype=torch.float32, device=dev)
    ms_u = timed(lambda: d.calc_range_many(sw, out=out), 5, 2)
    ms_o = timed(lambda: d.calc_range_many(sw, sort_by_slice=True, out=out), 5, 2)
    extra["sweep_rays_per_s"] = sw.shape[0] / (statistics.mean(ms_u) * 1e-3)
    extra["sweep_sorted_rays_per_s"] = sw.shape[0] / (statistics.mean(ms_o) * 1e-3)
    # the "grid" benchmark of Section V: every 4th cell centre in x and y and
    # 200 headings (50 M states, x fastest)
    gq = torch.from_numpy(WL.grid_states(grid.shape[1], grid.shape[0], 4, 200)).to(dev)
    gout = torch.empty(gq.shape[0], dtype=torch.float32, device=dev)
    ms_grid = timed(lambda: d.calc_range_many(gq, out=gout), 5, 2)
    extra["grid_sweep_rays_per_s"] = gq.shape[0] / (statistics.mean(ms_grid) * 1e-3)
    # per-warp latency (32 consecutive queries, one per lane) of 1 M random and
    # 1 M grid states, the GPU counterpart of the paper's per-query violins
    lat = {}
    for name, qs in (("random", sw[:1 << 20]), ("grid", gq[:1 << 20])):
        d.calc_range_timed(qs)
        _, cyc = d.calc_range_timed(qs)
        c = cyc.double().cpu().numpy()
        lat[name] = {"p25": float(np.percentile(c, 25)), "median": float(np.median(c)),
                     "p75": float(np.percentile(c, 75)), "p99": float(np.percentile(c, 99)), "mean": float(c.mean())}
    extra["warp_latency_cycles"] = lat

    # the paper's comparison: a 16-bit lookup table of every state, built on
    # the GPU from this CDDT; the same sensor model over table reads (all 200
    # filters in one launch) and the same 10 M sweep
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    lut = G.Lut(d)
    ev1.record()
    torch.cuda.synchronize()
    seg_l = torch.arange(0, S * P + 1, P, dtype=torch.int64, device=dev)
    ms_lut = timed(lambda: lut.sensor_weights(parts_d, seg_l, bo_d, obs_d, m, logw=logw_d), k2, 2)
    lut_out = torch.empty(sw.shape[0], dtype=torch.float32, device=dev)
    ms_lsw = timed(lambda: lut.calc_range_many(sw, out=lut_out), 5, 2)
    extra["lut"] = {"build_ms": ev0.elapsed_time(ev1), "bytes": lut.info()["bytes"],
                    "cddt_store_bytes": st0["store_bytes"],
                    "sensor_rays_per_s": rays_per_step / (statistics.mean(ms_lut) * 1e-3),
                    "sweep_rays_per_s": sw.shape[0] / (statistics.mean(ms_lsw) * 1e-3),
                    "grid_sweep_rays_per_s": gq.shape[0] / (statistics.mean(
                        timed(lambda: lut.calc_range_many(gq, out=gout), 3, 1)) * 1e-3)}
    lut.close()
    del lut_out

    # the Bresenham baseline (Section II's BL) on the same 10 M sweep and on
    # the tracking filter's rays (every particle x beam as a query), against
    # the CDDT's plain ray cast of the same rays
    bl_out = torch.empty(sw.shape[0], dtype=torch.float32, device=dev)
    ms_bl = timed(lambda: d.cast_bresenham(sw, out=bl_out), 3, 1)
    fr = torch.cat([parts_d[:, :2].repeat_interleave(B, 0),
                    (parts_d[:, 2:3] + bo_d[None, :]).reshape(-1, 1)], 1).contiguous()
    fr_out = torch.empty(fr.shape[0], dtype=torch.float32, device=dev)
    ms_blf = timed(lambda: d.cast_bresenham(fr, out=fr_out), 3, 1)
    ms_cf = timed(lambda: d.calc_range_many(fr, out=fr_out), 3, 1)
    ms_blg = timed(lambda: d.cast_bresenham(gq, out=gout), 3, 1)
    extra["bresenham"] = {"sweep_rays_per_s": sw.shape[0] / (statistics.mean(ms_bl) * 1e-3),
                          "grid_sweep_rays_per_s": gq.shape[0] / (statistics.mean(ms_blg) * 1e-3),
                          "filter_rays_per_s": fr.shape[0] / (statistics.mean(ms_blf) * 1e-3),
                          "cddt_filter_rays_per_s": fr.shape[0] / (statistics.mean(ms_cf) * 1e-3)}

    # the ray marching baseline (Section II's RM): its distance transform's
    # build, the same sweep and filter rays, and the distance reads per ray
    # of the sweep (the long tail the paper describes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rm = G.RayMarch(d)
    torch.cuda.synchronize()
    rm_build_ms = (time.perf_counter() - t0) * 1e3
    ms_rm = timed(lambda: rm.calc_range_many(sw, out=bl_out), 3, 1)
    ms_rmf = timed(lambda: rm.calc_range_many(fr, out=fr_out), 3, 1)
    ms_rmg = timed(lambda: rm.calc_range_many(gq, out=gout), 3, 1)
    rm_steps = torch.empty(sw.shape[0], dtype=torch.int32, device=dev)
    rm.calc_range_many(sw, out=bl_out, steps=rm_steps)
    st_f = rm_steps.float()
    extra["raymarch"] = {"sweep_rays_per_s": sw.shape[0] / (statistics.mean(ms_rm) * 1e-3),
                         "grid_sweep_rays_per_s": gq.shape[0] / (statistics.mean(ms_rmg) * 1e-3),
                         "filter_rays_per_s": fr.shape[0] / (statistics.mean(ms_rmf) * 1e-3),
                         "build_ms": rm_build_ms, "transform_bytes": 4 * grid.shape[0] * grid.shape[1],
                         "sweep_reads_mean": float(st_f.mean()),
                         "sweep_reads_p99": float(torch.quantile(st_f[:1 << 20], 0.99)),
                         "sweep_reads_max": int(rm_steps.max())}
    rm.close()
    del bl_out, fr, fr_out, rm_steps, st_f



    # the 16-bit zero-point store (Section IV-C's compression; reading S7):
    # half the key bytes, ranges quantised to 1/Q of a cell
    du = G.CDDT(grid, w["theta_disc"], mr, u16=True)
    stu = du.stats()
    plan_u = G.Plan(filters_for(du))
    shape_u = plan_u.autotune()
    ms_u = timed(plan_u.run, k2, 2)
    ms_uu = timed(lambda: du.calc_range_many(sw, out=out), 5, 2)
    ms_ug = timed(lambda: du.calc_range_many(gq, out=gout), 3, 1)
    # uniform particles (global localization) on the 16-bit store: there the
    # gathers reach DRAM, and the store is half the size
    plan_uq = G.Plan(filters_for(du, upart_d))
    shape_uq = plan_uq.autotune()
    ms_uq = timed(plan_uq.run, k2, 2)
    plan_uq.close()
    extra["u16"] = {"rays_per_s": rays_per_step / (statistics.mean(ms_u) * 1e-3),
                    "uniform_particles_rays_per_s": rays_per_step / (statistics.mean(ms_uq) * 1e-3),
                    "uniform_particles_shape": shape_uq,
                    "sweep_rays_per_s": sw.shape[0] / (statistics.mean(ms_uu) * 1e-3),
                    "grid_sweep_rays_per_s": gq.shape[0] / (statistics.mean(ms_ug) * 1e-3),
                    "store_bytes": stu["store_bytes"], "f32_store_bytes": st0["store_bytes"],
                    "build_ms": stu["build_ms"], "shape": shape_u}
    plan_u.close()
    du.close()

    dp = G.CDDT(grid, w["theta_disc"], mr)
    dp.prune()
    stp = dp.stats()
    plan_p = G.Plan(filters_for(dp))
    plan_p.set_shape(**shape)
    ms_p = timed(plan_p.run, k2, 2)
    extra["pruned_rays_per_s"] = rays_per_step / (statistics.mean(ms_p) * 1e-3)
    extra["prune_ms"] = stp["prune_ms"]
    extra["pruned_zero_points"] = stp["n_zero_points"]
    ms_pu = timed(lambda: dp.calc_range_many(sw, out=out), 5, 2)
    extra["pruned_sweep_rays_per_s"] = sw.shape[0] / (statistics.mean(ms_pu) * 1e-3)
    ms_pg = timed(lambda: dp.calc_range_many(gq, out=gout), 3, 1)
    extra["pruned_grid_sweep_rays_per_s"] = gq.shape[0] / (statistics.mean(ms_pg) * 1e-3)
    # the paper's comparison of methods (Section V): ray casts/s on the random
    # and the grid samples, the CDDT against its variants and the baselines
    extra["methods"] = {
        "cddt": {"random": extra["sweep_rays_per_s"], "grid": extra["grid_sweep_rays_per_s"]},
        "pcddt": {"random": extra["pruned_sweep_rays_per_s"], "grid": extra["pruned_grid_sweep_rays_per_s"]},
        "cddt_u16": {"random": extra["u16"]["sweep_rays_per_s"], "grid": extra["u16"]["grid_sweep_rays_per_s"]},
        "lut": {"random": extra["lut"]["sweep_rays_per_s"], "grid": extra["lut"]["grid_sweep_rays_per_s"]},
        "ray_marching": {"random": extra["raymarch"]["sweep_rays_per_s"],
                         "grid": extra["raymarch"]["grid_sweep_rays_per_s"]},
        "bresenham": {"random": extra["bresenham"]["sweep_rays_per_s"],
                      "grid": extra["bresenham"]["grid_sweep_rays_per_s"]}}
    del gq, gout
    plan_p.close()

    # end to end through the public API from pinned host buffers
    parts_h = torch.from_numpy(w["parts"].reshape(-1, 3)).pin_memory()
    obs_h = torch.from_numpy(obs).pin_memory()
    logw_h = torch.empty(S * P, dtype=torch.float32).pin_memory()

    def e2e_copy():
        parts_d.copy_(parts_h, non_blocking=True)
        obs_d.copy_(obs_h, non_blocking=True)
        plan.run()
        logw_h.copy_(logw_d, non_blocking=True)
    ms_c = timed(e2e_copy, k2, 2)
    copy_ms = max_over_ranks(world, statistics.mean(ms_c))
    # the same step on a plan whose particles, scans and log-weights are the
    # page-locked host buffers: the kernel reads the inputs and writes the
    # results across the host link itself (no copy-engine transfers)
    plan_h = G.Plan([dict(map=d, particles=parts_h[t * P:(t + 1) * P], beam_off=bo_d, obs=obs_h[t], model=m,
                          logw=logw_h[t * P:(t + 1) * P], pair_offset=D) for t in range(S)])
    plan_h.set_shape(**shape)
    ms_e = timed(plan_h.run, k2, 2)
    e2e_ms = max_over_ranks(world, statistics.mean(ms_e))
    plan_h.close()

    # the limit that binds the tracking workload: the L1 data pipe, one
    # wavefront per cycle per SM (global and shared wavefronts counted by ncu
    # on this kernel source), at the SM clock sampled in the timed region
    rec = recorded("batched_kernel")
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    wf_peak = nsm * sm_mhz * 1e6 / 1e9  # G wavefronts/s
    if rec and rec.get("l1_wavefronts_per_unit"):
        wf = rec["l1_wavefronts_per_unit"] * S * P
        binding = {"limit": "l1_data_pipe", "achieved": wf / (ms_step * 1e-3) / 1e9, "peak": wf_peak,
                   "unit": "G wavefronts/s", "frac": wf / (ms_step * 1e-3) / 1e9 / wf_peak,
                   "wavefronts_per_particle": rec["l1_wavefronts_per_unit"], "sms": nsm, "sm_mhz": sm_mhz,
                   "source": "ncu l1tex__data_pipe_lsu_wavefronts_mem_lg + _mem_shared per launch, this kernel source"}
    else:
        binding = {"limit": "l1_data_pipe", "achieved": None, "peak": wf_peak, "unit": "G wavefronts/s",
                   "frac": None, "sms": nsm, "sm_mhz": sm_mhz,
                   "source": "no ncu wavefront count recorded for this kernel source"}
    configs = {}
    if not args.no_configs:
        for name, fn in MEASURES.items():
            configs[name] = fn(G, torch, dev, world, rank, args.config_steps, 3)
    line = base_line(args, world, value, ms_step, "corridor2000",
                     {"launch": f"persistent batched, autotuned {shape}", "zero_points": st0["n_zero_points"],
                      "store_bytes": st0["store_bytes"], "occupancy": round(synth.occupancy(w["grid"]), 4)})
    line.update({
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic("batched_kernel", S * P), "peak_kind": peak_kind,
                     "kernel": "batched_kernel", "algorithmic_bytes_per_launch": alg, "work": work,
                     "sector_bytes_per_launch": sec, "sector_gbs": sec / (ms_step * 1e-3) / 1e9,
                     "gather_gbs_measured": gbw,
                     "sector_frac_of_hbm_gather": sec / (ms_step * 1e-3) / 1e9 / gbw["hbm"],
                     "binding": binding,
                     "limiter": ("on-chip: the L1 data pipe (wavefronts, binding.frac) and instruction issue (ncu "
                                 "capture of batched_kernel on this workload); the tracking filter's gathers are "
                                 "cache resident, DRAM traffic ~1 % of the algorithmic bytes")},
        "e2e": {"value": world * rays_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(parts_h.numel() * 4 + obs_h.numel() * 4),
                "d2h_bytes_per_step": int(logw_h.numel() * 4),
                "path": "plan on page-locked host buffers (kernel reads and writes them across the host link)",
                "copy_engine_value": world * rays_per_step / (copy_ms * 1e-3)},
        "gpu_launches": args.steps, "clocks": clocks,
        "build_ms": st0["build_ms"], "build_wall_s": build_wall, **extra, "configs": configs})
    if not args.no_cpu and rank == 0 and world == 1:
        from oracle import oracle as O
        cores = os.cpu_count() or 1
        o = O.OracleCDDT(w["grid"], w["theta_disc"], mr)
        sample = 40
        dt, n = cpu_oracle_run(o, w["parts"], bo, obs, sample, cores, mr)
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{sample} of {S} filter steps ({n} ray casts), oracle sensor weights, "
                                          f"OpenMP over particles"}
        dt1, n1 = cpu_oracle_run(o, w["parts"], bo, obs, 4, 1, mr)
        line["cpu_one_thread"] = {"value": n1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"4 of {S} filter steps ({n1} ray casts)"}
        line["cpu_host"] = host_cpu()
    plan.close()
    return line


# ------------------------------------------------------------------ the other configurations
#
# Each measure_* function times one configuration and returns a compact dict
# (rays/s and the figures the configuration is about); the default line
# carries all four under "configs", and `--workload NAME` prints one as its
# own line.

def measure_rects(G, torch, dev, world, rank, steps, warmup):
    """rects256: one 1000-particle filter, one cddt_sensor_weights call per
    step (host call + launch), and the same as a one-filter plan under a CUDA
    graph."""
    w = WL.rects256()
    bo, D, mr = w["beam_off"], w["D"], w["max_range"]
    d = G.CDDT(torch.from_numpy(w["grid"]).to(dev), w["theta_disc"], mr)
    r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], bo)).to(dev)).cpu().numpy()
    obs = torch.from_numpy(np.clip(r + w["noise"][0], 0, mr).astype(np.float32)).to(dev)
    parts = torch.from_numpy(w["parts"][0]).to(dev)
    bo_d = torch.from_numpy(bo).to(dev)
    logw = torch.empty(parts.shape[0], device=dev)
    m = G.beam_model(mr)
    timed = Timer(world, dev)
    with ClockSampler(dev.index) as clk:
        ms = timed(lambda: d.sensor_weights(parts, bo_d, obs, m, D, logw=logw), steps, warmup)
    ms_step = max_over_ranks(world, statistics.mean(ms))
    rays = parts.shape[0] * bo.size
    plan = G.Plan([dict(map=d, particles=parts, beam_off=bo_d, obs=obs, model=m, logw=logw, pair_offset=D)])
    plan.autotune()
    ms_g = timed(plan.launch_graph, steps, 2)
    st = d.stats()
    plan.close()
    d.close()
    return {"rays_per_s": world * rays / (ms_step * 1e-3), "ms_per_step": ms_step, "rays_per_step": rays,
            "graph_rays_per_s": rays / (statistics.mean(ms_g) * 1e-3), "build_ms": st["build_ms"],
            "zero_points": st["n_zero_points"], "clocks": clk.summary(timed.window),
            "launch": "cddt_sensor_weights, one call per step"}


def measure_batched64(G, torch, dev, world, rank, steps, warmup):
    """batched64: 64 maps and filters in one persistent launch under a CUDA
    graph, against the same filters as 64 per-filter launches."""
    w = WL.batched64(seed_offset=RK.seed_offset(rank))
    bo = torch.from_numpy(w["beam_off"]).to(dev)
    D = w["D"]
    filters, build_ms = [], []
    for mp in w["maps"]:
        d = G.CDDT(torch.from_numpy(mp["grid"]).to(dev), mp["theta_disc"], mp["max_range"])
        build_ms.append(d.stats()["build_ms"])
        r = d.calc_range_many(torch.from_numpy(WL.gt_queries(mp["gt"], w["beam_off"])).to(dev)).cpu().numpy()
        obs = torch.from_numpy(np.clip(r + mp["noise"][0], 0, mp["max_range"]).astype(np.float32)).to(dev)
        parts = torch.from_numpy(mp["parts"][0]).to(dev)
        filters.append(dict(map=d, particles=parts, beam_off=bo, obs=obs, model=G.beam_model(mp["max_range"]),
                            logw=torch.empty(parts.shape[0], device=dev), pair_offset=D))
    plan = G.Plan(filters)
    shape = plan.autotune()
    timed = Timer(world, dev)
    rays = sum(f["particles"].shape[0] for f in filters) * bo.numel()
    with ClockSampler(dev.index) as clk:
        ms = timed(plan.launch_graph, steps, warmup)
    clocks = clk.summary(timed.window)
    ms_step = max_over_ranks(world, statistics.mean(ms))

    def sequential():
        for f in filters:
            f["map"].sensor_weights(f["particles"], bo, f["obs"], f["model"], D, logw=f["logw"])
    ms_s = timed(sequential, max(3, steps // 2), 2)
    plan.close()
    for f in filters:
        f["map"].close()
    return {"rays_per_s": world * rays / (ms_step * 1e-3), "ms_per_step": ms_step, "rays_per_step": rays,
            "particles": rays // bo.numel(), "sequential_rays_per_s": rays / (statistics.mean(ms_s) * 1e-3),
            "batched_speedup_vs_sequential": statistics.mean(ms_s) / statistics.mean(ms),
            "build_ms_total": sum(build_ms), "shape": shape, "clocks": clocks,
            "launch": "persistent batched under a CUDA graph vs 64 cddt_sensor_weights launches"}


def measure_diff(G, torch, dev, world, rank, steps, warmup):
    """diff2000: forward + adjoint of 4096 x 61 and 1024 x 1081 beams with 10
    gradient refinement steps x += eta g / |g| (11 evaluations): in one
    launch (cddt_plan_refine), and as the step-by-step loop of
    cddt_sensor_weights_fwd_bwd calls and torch updates, eager and captured
    in a CUDA graph; the forward pass alone beside them."""
    w = WL.diff2000(seed_offset=RK.seed_offset(rank))
    mr = w["max_range"]
    d = G.CDDT(torch.from_numpy(w["grid"]).to(dev), w["theta_disc"], mr)
    m = G.beam_model(mr)
    scans, filters = [], []
    for sc in w["scans"]:
        r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], sc["beam_off"])).to(dev)).cpu().numpy()
        obs = torch.from_numpy(np.clip(r + sc["noise"], 0, mr).astype(np.float32)).to(dev)
        p0, bo = torch.from_numpy(sc["parts"]).to(dev), torch.from_numpy(sc["beam_off"]).to(dev)
        P = p0.shape[0]
        scans.append((p0, bo, obs, sc["D"]))
        filters.append(dict(map=d, particles=p0, beam_off=bo, obs=obs, model=m, logw=torch.empty(P, device=dev),
                            pair_offset=sc["D"], grad_xy=torch.empty((P, 2), device=dev),
                            particles_out=torch.empty((P, 3), device=dev)))
    n_eval = w["refine_steps"] + 1
    rays_eval = sum(p.shape[0] * bo.numel() for p, bo, _, _ in scans)
    rays = rays_eval * n_eval
    plan = G.Plan(filters)
    timed = Timer(world, dev)
    with ClockSampler(dev.index) as clk:
        ms = timed(lambda: plan.refine(w["refine_steps"], w["eta"]), steps, warmup)
    clocks = clk.summary(timed.window)
    ms_step = max_over_ranks(world, statistics.mean(ms))

    def loop():  # forward + adjoint, then the update, n_eval times per scan
        for p0, bo, obs, D in scans:
            x = p0.clone()
            for _ in range(n_eval):
                lw, g = d.sensor_weights_fwd_bwd(x, bo, obs, m, D)
                n = torch.linalg.norm(g, dim=1, keepdim=True).clamp_min(1e-12)
                x[:, :2] += w["eta"] * g / n
    ms_e = timed(loop, max(3, steps // 2), 2)
    graph_rays = None
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            loop()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            loop()
        graph_rays = rays / (statistics.mean(timed(graph.replay, max(3, steps // 2), 2)) * 1e-3)
    except RuntimeError as e:
        print(f"graph capture of the refinement loop failed: {e}", file=sys.stderr)
    fwd = timed(lambda: [d.sensor_weights(p, bo, obs, m, D) for p, bo, obs, D in scans], max(3, steps // 2), 2)
    plan.close()
    d.close()
    return {"rays_per_s": world * rays / (ms_step * 1e-3), "ms_per_step": ms_step, "rays_per_step": rays,
            "launch": "cddt_plan_refine: 10 refinement steps + final evaluation, one launch (value counts "
                      "forward+adjoint ray casts)",
            "loop_rays_per_s": rays / (statistics.mean(ms_e) * 1e-3), "loop_graph_rays_per_s": graph_rays,
            "forward_only_rays_per_s": rays_eval / (statistics.mean(fwd) * 1e-3), "clocks": clocks}


def measure_update(G, torch, dev, world, rank, steps, warmup):
    """update4000: 10^4 cell writes (5000 inserts, 5000 removes) through
    cddt_update_cells on a 4000 x 4000 map (theta_disc 360), then 100,000
    particles x 61 beams; full build and prune (on a separate handle) times;
    and a 10 M-query uniform sweep of the fresh map, unsorted and
    slice-sorted."""
    w = WL.update4000(steps=steps + warmup, seed_offset=RK.seed_offset(rank))
    mr = w["max_range"]
    grid = torch.from_numpy(w["grid"]).to(dev)
    d = G.CDDT(grid, w["theta_disc"], mr)
    st = d.stats()
    # a 10 M uniform sweep of the 2 GB store, unsorted and slice-sorted: with
    # the store 16x the L2, each unsorted search misses at every level, and
    # the sort's slice-by-slice order reads each slice's nodes about once
    sw = torch.from_numpy(synth.uniform_queries(w["grid"], 10_000_000, seed=synth.SEED_PARTICLES + 4007)).to(dev)
    sw_out = torch.empty(sw.shape[0], device=dev)
    timed = Timer(world, dev)
    ms_sw = timed(lambda: d.calc_range_many(sw, out=sw_out), 5, 2)
    ms_so = timed(lambda: d.calc_range_many(sw, sort_by_slice=True, out=sw_out), 5, 2)
    sweep = {"sweep_rays_per_s": sw.shape[0] / (statistics.mean(ms_sw) * 1e-3),
             "sweep_sorted_rays_per_s": sw.shape[0] / (statistics.mean(ms_so) * 1e-3)}
    del sw, sw_out
    dp = G.CDDT(grid, w["theta_disc"], mr)
    dp.prune()
    prune_ms = dp.stats()["prune_ms"]
    dp.close()
    bo = torch.from_numpy(w["beam_off"]).to(dev)
    r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], w["beam_off"])).to(dev)).cpu().numpy()
    obs = torch.from_numpy(np.clip(r + w["noise"][0], 0, mr).astype(np.float32)).to(dev)
    parts = torch.from_numpy(w["parts"]).to(dev)
    m = G.beam_model(mr)
    logw = torch.empty(parts.shape[0], device=dev)
    writes = iter([(torch.from_numpy(xy).to(dev), torch.from_numpy(occ).to(dev)) for xy, occ in w["writes"]])
    upd_ms = []

    def step():
        xy, occ = next(writes)
        d.update_cells(xy, occ)
        upd_ms.append(d.stats()["update_ms"])
        d.sensor_weights(parts, bo, obs, m, w["D"], logw=logw)
    with ClockSampler(dev.index) as clk:
        ms = timed(step, steps, warmup)
    clocks = clk.summary(timed.window)
    ms_step = max_over_ranks(world, statistics.mean(ms))
    qms = timed(lambda: d.sensor_weights(parts, bo, obs, m, w["D"], logw=logw), steps, 2)
    rays = parts.shape[0] * bo.numel()
    st2 = d.stats()
    d.close()
    return {"rays_per_s": world * rays / (ms_step * 1e-3), "ms_per_step": ms_step, "rays_per_step": rays,
            "writes_per_step": int(w["writes"][0][0].shape[0]),
            "update_ms_per_1e4_writes": statistics.mean(upd_ms[warmup:] or upd_ms),
            "query_only_rays_per_s": rays / (statistics.mean(qms) * 1e-3), "build_ms": st["build_ms"],
            "prune_ms": prune_ms, "zero_points": st2["n_zero_points"], "store_bytes": st2["store_bytes"],
            **sweep, "clocks": clocks,
            "launch": "cddt_update_cells (10^4 writes) then cddt_sensor_weights (100,000 x 61) per step"}


MEASURES = {"rects256": measure_rects, "batched64": measure_batched64, "diff2000": measure_diff,
            "update4000": measure_update}


def bench_other(name):
    def run(args, G, torch, dev, world, rank):
        r = MEASURES[name](G, torch, dev, world, rank, args.steps, args.warmup)
        line = base_line(args, world, r.pop("rays_per_s"), r.pop("ms_per_step"), name,
                         {"launch": r.pop("launch", "")})
        line.update({"gpu_launches": args.steps, **r})
        return line
    return run


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    from paper_1705_01167_gb300 import cddt as G
    G.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fn = bench_corridor if args.workload == "corridor2000" else bench_other(args.workload)
    line = fn(args, G, torch, dev, world, rank)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_update(args):
    """A short run for ncu: build the 4000 x 4000 corridor CDDT, then apply
    warmup + steps batches of 10^4 cell writes (the update4000 writes); with
    --profile-case update2000 the 2000 x 2000 corridor CDDT (theta_disc 200)
    and batches of 2,800 writes (1,400 set, 1,400 cleared), the same number
    of changes per bin on a store that an ncu capture handles in seconds."""
    import torch
    from paper_1705_01167_gb300 import cddt as G
    if args.profile_case == "update2000":
        g = synth.corridor_map(2000, 2000)
        cur, writes = g.copy(), []
        for t in range(args.warmup + args.steps):
            xy, occ = synth.cell_toggles(cur, 1400, 1400, seed=synth.SEED_UPDATES + t)
            writes.append((xy, occ))
            cur = synth.apply_writes(cur, xy, occ)
        w = dict(grid=g, theta_disc=200, max_range=1000.0, writes=writes)
    else:
        w = WL.update4000(steps=args.warmup + args.steps)
    dev = torch.device("cuda", 0)
    d = G.CDDT(torch.from_numpy(w["grid"]).to(dev), w["theta_disc"], w["max_range"])
    ms = []
    for xy, occ in w["writes"]:
        d.update_cells(torch.from_numpy(xy).to(dev), torch.from_numpy(occ).to(dev))
        ms.append(round(d.stats()["update_ms"], 3))
    torch.cuda.synchronize()
    print(json.dumps({"profile": "update", "update_ms": ms, "status": d.status(),
                      "zero_points": d.stats()["n_zero_points"]}))
    return 0


def run_profile_prune(args):
    """A short run for ncu: build the 2000 x 2000 corridor CDDT (theta_disc
    200) and prune it, warmup + steps times (a fresh handle each time)."""
    import torch
    from paper_1705_01167_gb300 import cddt as G
    dev = torch.device("cuda", 0)
    grid = torch.from_numpy(synth.corridor_map(2000, 2000)).to(dev)
    ms = []
    for _ in range(args.warmup + args.steps):
        d = G.CDDT(grid, 200, 1000.0)
        d.prune()
        st = d.stats()
        ms.append(round(st["prune_ms"], 3))
        d.close()
    torch.cuda.synchronize()
    print(json.dumps({"profile": "prune", "prune_ms": ms, "zero_points": st["n_zero_points"]}))
    return 0


def run_profile_refine(args):
    """A short run for ncu: warmup + steps one-launch refinements of the
    diff2000 workload (10 steps each)."""
    import torch
    from paper_1705_01167_gb300 import cddt as G
    w = WL.diff2000()
    dev = torch.device("cuda", 0)
    d = G.CDDT(torch.from_numpy(w["grid"]).to(dev), w["theta_disc"], w["max_range"])
    m = G.beam_model(w["max_range"])
    filters = []
    for sc in w["scans"]:
        r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], sc["beam_off"])).to(dev)).cpu().numpy()
        obs = torch.from_numpy(np.clip(r + sc["noise"], 0, w["max_range"]).astype(np.float32)).to(dev)
        P = sc["parts"].shape[0]
        filters.append(dict(map=d, particles=torch.from_numpy(sc["parts"]).to(dev),
                            beam_off=torch.from_numpy(sc["beam_off"]).to(dev), obs=obs, model=m,
                            logw=torch.empty(P, device=dev), pair_offset=sc["D"],
                            grad_xy=torch.empty((P, 2), device=dev), particles_out=torch.empty((P, 3), device=dev)))
    plan = G.Plan(filters)
    for _ in range(args.warmup + args.steps):
        plan.refine(w["refine_steps"], w["eta"])
    torch.cuda.synchronize()
    print(json.dumps({"profile": "refine", "logw0": float(filters[0]["logw"][0])}))
    return 0


def run_profile_sweep4000(args):
    """A short run for ncu: one unsorted and one slice-sorted 10 M uniform
    sweep of the 4000 x 4000 map (theta_disc 360, 2 GB store), after
    `warmup` of each."""
    import torch
    from paper_1705_01167_gb300 import cddt as G
    g = synth.corridor_map(4000, 4000)
    dev = torch.device("cuda", 0)
    d = G.CDDT(torch.from_numpy(g).to(dev), 360, 1000.0)
    sw = torch.from_numpy(synth.uniform_queries(g, 10_000_000, seed=synth.SEED_PARTICLES + 4007)).to(dev)
    out = torch.empty(sw.shape[0], device=dev)
    for _ in range(args.warmup + 1):
        d.calc_range_many(sw, out=out)
        d.calc_range_many(sw, sort_by_slice=True, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "sweep4000", "store_bytes": d.stats()["store_bytes"]}))
    return 0


def run_profile(args):
    """A short run for ncu: the batched launch (fixed shape), one per-filter
    pass and one sweep launch, a few launches each."""
    if args.profile_case in ("update", "update2000"):
        return run_profile_update(args)
    if args.profile_case == "prune":
        return run_profile_prune(args)
    if args.profile_case == "sweep4000":
        return run_profile_sweep4000(args)
    if args.profile_case == "refine":
        return run_profile_refine(args)
    import torch
    from paper_1705_01167_gb300 import cddt as G
    w = WL.corridor2000()
    dev = torch.device("cuda", 0)
    d = G.CDDT(torch.from_numpy(w["grid"]).to(dev), w["theta_disc"], w["max_range"],
               u16=args.profile_case == "u16")
    bo, D = w["beam_off"], w["D"]
    S, P = w["parts"].shape[:2]
    r = d.calc_range_many(torch.from_numpy(WL.gt_queries(w["gt"], bo)).to(dev)).cpu().numpy()
    obs = np.clip(r.reshape(S, bo.size) + w["noise"], 0, w["max_range"]).astype(np.float32)
    parts = w["parts"]
    if args.profile_case == "uniform":  # global localization: particles over the whole free space
        parts = np.stack([synth.uniform_particles(w["grid"], P, seed=synth.SEED_PARTICLES + 5000 + t)
                          for t in range(S)])
    parts_d = torch.from_numpy(parts.reshape(-1, 3)).to(dev).contiguous()
    bo_d = torch.from_numpy(bo).to(dev)
    obs_d = torch.from_numpy(obs).to(dev).contiguous()
    logw_d = torch.empty(S * P, dtype=torch.float32, device=dev)
    m = G.beam_model(w["max_range"])
    plan = G.Plan([dict(map=d, particles=parts_d[t * P:(t + 1) * P], beam_off=bo_d, obs=obs_d[t], model=m,
                        logw=logw_d[t * P:(t + 1) * P], pair_offset=D) for t in range(S)])
    plan.set_shape(args.shape_tpp, args.shape_ppi, args.shape_block, args.shape_regcap)
    for _ in range(args.warmup + args.steps):
        plan.run()
    for t in range(S):
        d.sensor_weights(parts_d[t * P:(t + 1) * P], bo_d, obs_d[t], m, D, logw=logw_d[t * P:(t + 1) * P])
    sw = torch.from_numpy(w["sweep"]).to(dev)
    d.calc_range_many(sw)
    d.calc_range_many(sw, sort_by_slice=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "ok", "logw0": float(logw_d[0]), "zero_points": d.stats()["n_zero_points"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cddt", choices=["cddt", "reference"])
    ap.add_argument("--workload", default="corridor2000", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = every rank runs the whole workload (rank-seeded inputs); strong = the "
                         "200 filters are split across ranks (ranks.partition)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the other configurations' compact measurements")
    ap.add_argument("--config-steps", type=int, default=10, help="timed steps of each other configuration")
    ap.add_argument("--profile", action="store_true", help="short fixed-shape run for ncu")
    ap.add_argument("--profile-case", default="corridor", choices=["corridor", "u16", "uniform", "update", "update2000", "prune", "refine",
                             "sweep4000"],
                    help="--profile workload: the corridor plan (u16: on the 16-bit store; uniform: uniform "
                         "particles), 10^4-write updates on the 4000^2 map (update2000: 2,800-write updates on the "
                         "2000^2 map), pruning the 2000^2 map, the diff2000 refinement launch, "
                         "or a 10 M sweep of the 4000^2 map, unsorted and slice-sorted")
    ap.add_argument("--shape-tpp", type=int, default=1)
    ap.add_argument("--shape-ppi", type=int, default=512)
    ap.add_argument("--shape-block", type=int, default=512)
    ap.add_argument("--shape-regcap", type=int, default=1)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
