"""The GPU lookup table (the paper's main comparison) against the oracle's
16-bit table of O4 ranges."""
import numpy as np
import pytest
import torch

from paper_1705_01167_gb300 import synth, workloads as WL
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01167_gb300 import cddt
    cddt.load()
    return cddt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("u16", [False, True])
def test_lut_matches_oracle(G, oracle, u16):
    from oracle import oracle as O
    g = synth.rect_map(96, 80, n_rects=12, seed=111)
    N, mr = 36, 150.0
    d = G.CDDT(dev(g), N, mr, u16=u16)
    o = oracle.OracleCDDT(g, N, mr, u16=u16)
    lut = G.Lut(d)
    info = lut.info()
    assert info["bytes"] == 2 * 96 * 80 * N and info["scale"] == O.lut_scale(mr)
    tab = O.lut_table(o.params, g, mr) if not u16 else None
    # every state of the table, read back by lookups at the states
    q = WL.grid_states(96, 80, 1, N)
    got = lut.calc_range_many(dev(q)).cpu().numpy()
    if not u16:
        want = (tab.astype(np.float32) / np.float32(info["scale"])).reshape(-1)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    else:  # a 16-bit CDDT's table codes its own (quantised) ranges
        r = d.calc_range_many(dev(q)).cpu().numpy()
        code = np.clip(np.floor(r * np.float32(info["scale"]) + np.float32(0.5)), 0, 65535)
        assert np.array_equal(got, (code / info["scale"]).astype(np.float32))
    if not u16:
        rq = gc.random_queries(96, 80, 20000, 112)
        rq[:3] = [[-1.0, 5.0, 0.2], [95.6, 79.4, 1.0], [10.0, 10.0, np.inf]]
        got = lut.calc_range_many(dev(rq)).cpu().numpy()
        want = O.lut_lookup(o.params, tab, mr, rq)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        # the fused sensor model over table reads, three filters
        sizes = [200, 1, 317]
        seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        gts = synth.uniform_particles(g, 3, seed=113)
        parts = np.concatenate([synth.tracking_particles(gts[f].astype(np.float64), n, seed=114 + f)
                                for f, n in enumerate(sizes)])
        bo = synth.beam_offsets(61)
        obs = np.stack([gc.observations(o, gts[f], bo, mr, seed=120 + f) for f in range(3)]).astype(np.float32)
        lw = lut.sensor_weights(dev(parts), dev(seg), dev(bo), dev(obs), G.beam_model(mr)).cpu().numpy()
        want = np.concatenate([O.lut_sensor_weights(o.params, tab, mr, parts[seg[f]:seg[f + 1]], bo, obs[f],
                                                    oracle.beam_model(mr)) for f in range(3)])
        assert (np.abs(lw - want) <= 1e-5 * np.maximum(1.0, np.abs(want))).all()
    lut.close()


def test_lut_full_size_sampled(G, oracle):
    """The 2000 x 2000 corridor map at theta_disc 200 (the bench's table,
    1.6 GB): sampled states read back exactly as the oracle's coded cast of
    that state, and continuous queries read their nearest state's entry."""
    from oracle import oracle as O
    g = synth.corridor_map(2000, 2000)
    N, mr = 200, 1000.0
    d = G.CDDT(dev(g), N, mr)
    lut = G.Lut(d)
    o = oracle.OracleCDDT(g, N, mr)
    sc = np.float32(O.lut_scale(mr))

    def coded(r):
        code = np.clip(np.floor(r * sc + np.float32(0.5)), 0, 65535).astype(np.float32)
        return (code / sc).astype(np.float32)

    rs = synth.Stream(131)
    n = 20000
    i = rs.integers(n, 0, 1999)
    j = rs.integers(n, 0, 1999)
    k = rs.integers(n, 0, N - 1)
    th = np.array([np.float32(2.0 * np.pi * kk / N) for kk in k], np.float32)
    st = np.stack([i, j, th], 1).astype(np.float32)
    got = lut.calc_range_many(dev(st)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), coded(o.calc_range(st)).view(np.uint32))
    q = synth.uniform_queries(g, 20000, seed=132)
    ks = np.array([o.params.query_k(float(t)) for t in q[:, 2]])
    snap = np.stack([np.floor(q[:, 0] + np.float32(0.5)), np.floor(q[:, 1] + np.float32(0.5)),
                     np.array([np.float32(2.0 * np.pi * kk / N) for kk in ks], np.float32)], 1).astype(np.float32)
    got = lut.calc_range_many(dev(q)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), coded(o.calc_range(snap)).view(np.uint32))
