"""The CUDA-event call trace on the GPU: per-entry-point call counts and
device times, nothing recorded while tracing is off or while a stream is
being captured into a graph, and results unchanged by tracing."""
import numpy as np
import pytest
import torch

from paper_1705_01167_gb300 import synth
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01167_gb300 import cddt
    cddt.load()
    return cddt


def test_trace_counts_and_times_calls(G):
    g = synth.rect_map(256, 256)
    d = G.CDDT(torch.from_numpy(g).cuda(), 108, 300.0)
    q = torch.from_numpy(gc.random_queries(256, 256, 1 << 20, 601)).cuda()
    ref = d.calc_range_many(q)
    G.trace_report()  # drop anything earlier
    G.trace_enable(True)
    try:
        outs = [d.calc_range_many(q) for _ in range(3)]
        parts = torch.from_numpy(synth.uniform_particles(g, 1000, seed=602)).cuda()
        bo = torch.from_numpy(synth.beam_offsets(61)).cuda()
        obs = torch.full((61,), 50.0, device="cuda")
        d.sensor_weights(parts, bo, obs, G.beam_model(300.0), synth.pair_offset(61))
        rep = {r["entry"]: r for r in G.trace_report()}
        assert rep["cddt_calc_range_many"]["calls"] == 3
        assert rep["cddt_sensor_weights"]["calls"] == 1
        r = rep["cddt_calc_range_many"]
        assert 0 < r["min_ms"] <= r["mean_ms"] <= r["max_ms"] and r["total_ms"] > 0
        for o in outs:
            assert torch.equal(o, ref)
        assert G.trace_report() == []  # the report cleared it
        # nothing is recorded for calls captured into a graph
        out = torch.empty_like(ref)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            d.calc_range_many(q, out=out, stream=s)  # warm-up outside capture
        torch.cuda.synchronize()
        G.trace_report()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            d.calc_range_many(q, out=out, stream=s)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert G.trace_report() == []
    finally:
        G.trace_enable(False)
    d.calc_range_many(q)
    assert G.trace_report() == []
