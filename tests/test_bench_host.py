"""The benchmark's host-side arithmetic and bookkeeping, on the CPU: the
roofline byte counts, the recorded-traffic gate on the kernel's source, the
measured-peak lookup, the clock-sample summary over the timed region, and the
fields of the JSON line."""
import argparse
import datetime
import json
import os
import time

import pytest

import bench


def test_algorithmic_and_sector_bytes():
    # 8 B of offsets per search, 4 B per probe, 4 B per paired reverse beam,
    # 17 B per particle; 32 B per sorted-CSR sector plus 17 B per particle
    work = {"traversals": 10, "probes": 30, "paired": 4, "sectors": 5}
    assert bench.algorithmic_bytes(work, 2) == 8 * 10 + 4 * 30 + 4 * 4 + 17 * 2
    assert bench.sector_bytes(work, 2) == 32 * 5 + 17 * 2
    acc = {}
    bench.add_work(acc, work)
    bench.add_work(acc, work)
    assert acc["traversals"] == 20 and acc["sectors"] == 10


def test_recorded_traffic_follows_the_kernel_source(monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["batched_kernel"]
    got = bench.recorded_traffic("batched_kernel", 1000)
    if d["source_sha"] == bench.kernel_source_sha("batched_kernel"):
        assert got == pytest.approx(d["dram_bytes_per_unit"] * 1000)
    else:
        assert got is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda k: "0" * 16)
    assert bench.recorded_traffic("batched_kernel", 1000) is None


def test_measured_peaks():
    peak, kind = bench.measured_peaks()
    assert peak > 1000.0 and kind in ("measured", "fallback")
    if not os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert (peak, kind) == (6800.0, "fallback")


def _write_samples(path, t0, rows):
    def ts(t):
        return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    with open(path, "w") as f:
        for dt, mhz, cap in rows:
            f.write(f"{ts(t0 + dt)}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, "
                    f"{'Active' if cap else 'Not Active'}\n")


def test_clock_summary_over_the_timed_region(tmp_path, monkeypatch):
    monkeypatch.setenv("CDDT_CLOCKS_DIR", str(tmp_path))
    c = bench.ClockSampler(0)
    c.proc = object()  # as if nvidia-smi had been started
    now = time.time()
    _write_samples(c.path, now, [(-0.5, 1200, False), (0.1, 2070, True), (0.3, 2040, False), (0.9, 900, False)])
    s = c.summary((now, now + 0.5))
    assert s["basis"] == "samples inside the timed region" and s["samples"] == 2
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    s = c.summary((now + 0.4, now + 0.45))
    assert s["basis"].startswith("nearest samples") and s["samples"] == 2 and s["sm_mhz"] == (2040 + 900) / 2
    s = c.summary()
    assert s["basis"] == "all samples" and s["samples"] == 4
    c.proc = None
    assert c.summary((now, now + 1))["reasons"] == ["unavailable"]


def test_json_line_fields():
    args = argparse.Namespace(steps=7, warmup=3)
    line = bench.base_line(args, 2, 1.5e9, 0.25, "corridor2000", {"extra": 1})
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["n_gpus"] == 2 and line["steps"] == 7 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["config"]["workload"] and line["config"]["extra"] == 1
    json.dumps(line)  # serialisable
    h = bench.host_cpu()
    assert h["nproc"] >= 1


def test_recorded_counts_of_other_launches_follow_their_kernel_source(monkeypatch):
    # the uniform-particle launch of batched_kernel is gated on that kernel's
    # sources too, and carries its L1 wavefronts and DRAM bytes per particle
    rec = bench.recorded("batched_kernel_uniform")
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    if d["batched_kernel_uniform"]["source_sha"] == bench.kernel_source_sha("batched_kernel"):
        assert rec["l1_wavefronts_per_unit"] > 0 and rec["dram_bytes_per_unit"] > 0
    else:
        assert rec is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda k: "0" * 16)
    assert bench.recorded("batched_kernel_uniform") is None
    assert bench.recorded("batched_kernel") is None


def test_every_configuration_states_its_launch():
    # each measure_* result names its launch (the standalone --workload line
    # carries it in config.launch)
    import inspect
    for name, fn in bench.MEASURES.items():
        src = inspect.getsource(fn)
        assert '"launch":' in src, name
