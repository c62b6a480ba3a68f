"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Zero-point lists and ranges are compared bit for bit; log-weights within
1e-5 relative of the float64 oracle, gradients within 1e-5 of the float64
oracle relative to the sum of the per-beam term magnitudes (the scale of a
float32 summation's rounding error) and, on samples whose terms cancel by
less than a factor 10, within 1e-5 relative to the gradient itself."""
import math

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_bits_equal(got, want, what=""):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape, what
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}"


def check_csr(G, oracle, g, N, mr, u16=False):
    d = G.CDDT(dev(g), N, mr, u16=u16)
    o = oracle.OracleCDDT(g, N, mr, u16=u16)
    sb, bs, zp = d.export()
    obs_, ozp = o.export()
    np.testing.assert_array_equal(sb, o.params.sbase)
    np.testing.assert_array_equal(bs, obs_)
    assert_bits_equal(zp, ozp, "zero points")
    gg, ee = d.export_grid()
    og, oe = o.grid_edge()
    np.testing.assert_array_equal(gg, og)
    np.testing.assert_array_equal(ee, oe)
    st = d.stats()
    assert st["n_zero_points"] == o.total_zp
    assert st["total_bins"] == o.params.total_bins
    return d, o


# ------------------------------------------------------------------ build

@pytest.mark.parametrize("u16", [False, True])
def test_build_tiny_maps(G, oracle, u16):
    for g in gc.tiny_maps():
        for N in (2, 4, 8, 12, 16):
            check_csr(G, oracle, g, N, 37.5, u16)


@pytest.mark.parametrize("u16", [False, True])
def test_build_rect_map_config1(G, oracle, u16):
    """256 x 256 rectangles map, N = 108 (the small configuration)."""
    g = synth.rect_map(256, 256)
    check_csr(G, oracle, g, 108, 300.0, u16)


def test_build_empty_and_full(G, oracle):
    check_csr(G, oracle, np.zeros((17, 23), np.uint8), 8, 50.0)
    check_csr(G, oracle, np.ones((17, 23), np.uint8), 8, 50.0)
    check_csr(G, oracle, np.ones((1, 1), np.uint8), 2, 5.0)
    check_csr(G, oracle, np.zeros((1, 1), np.uint8), 2, 5.0)


def test_build_large_bins(G, oracle):
    """Every size class of the per-bin sort: a striped 20000 x 12 map gives
    rows of 20000 zero points at theta = 0 (larger than shared memory) and
    bins of a few hundred to a few thousand at the other angles."""
    g = np.zeros((12, 20000), np.uint8)
    g[::2, :] = 1
    g[1, ::7] = 1
    d, o = check_csr(G, oracle, g, 16, 30000.0)
    assert d.stats()["max_bin"] >= 20000
    q = gc.random_queries(20000, 12, 20000, 77)
    assert_bits_equal(d.calc_range_many(dev(q)).cpu().numpy(), o.calc_range(q))


# ------------------------------------------------------------------ ranges

@pytest.mark.parametrize("u16", [False, True])
@pytest.mark.parametrize("search", [0, 1])
@pytest.mark.parametrize("sort", [False, True])
def test_calc_range_tiny_maps(G, oracle, u16, search, sort):
    for mi, g in enumerate(gc.tiny_maps()):
        H, W = g.shape
        for N in (4, 8, 16):
            d = G.CDDT(dev(g), N, 37.5, u16=u16)
            d.set_search(search)
            o = oracle.OracleCDDT(g, N, 37.5, u16=u16)
            q = np.concatenate([gc.grid_states(W, H, N), gc.random_queries(W, H, 3000, 100 + mi),
                                gc.special_queries(W, H)])
            got = d.calc_range_many(dev(q), sort_by_slice=sort).cpu().numpy()
            assert_bits_equal(got, o.calc_range(q), f"map {mi} N {N}")


@pytest.mark.parametrize("u16", [False, True])
@pytest.mark.parametrize("search", [0, 1])
def test_calc_range_config1(G, oracle, u16, search):
    g = synth.rect_map(256, 256)
    d = G.CDDT(dev(g), 108, 300.0, u16=u16)
    d.set_search(search)
    o = oracle.OracleCDDT(g, 108, 300.0, u16=u16)
    q = np.concatenate([gc.grid_states(256, 256, 108, stride=7), gc.random_queries(256, 256, 200001, 5),
                        synth.uniform_queries(g, 100003, seed=6), gc.special_queries(256, 256)])
    want = o.calc_range(q, nthreads=8)
    for sort in (False, True):
        got = d.calc_range_many(dev(q), sort_by_slice=sort).cpu().numpy()
        assert_bits_equal(got, want, f"sort={sort}")


def test_calc_range_empty_batch(G):
    g = synth.rect_map(64, 64, n_rects=5)
    d = G.CDDT(dev(g), 16, 100.0)
    out = d.calc_range_many(torch.empty((0, 3), dtype=torch.float32, device="cuda"))
    assert out.numel() == 0
    out = d.calc_range_many(torch.empty((0, 3), dtype=torch.float32, device="cuda"), sort_by_slice=True)
    assert out.numel() == 0


# ------------------------------------------------------------------ sensor model

def _scan(B):
    bo = synth.beam_offsets(B)
    return bo, synth.pair_offset(B)


def _logw_close(got, want, rtol=1e-5):
    got = np.asarray(got, np.float64)
    err = np.abs(got - want)
    lim = rtol * np.maximum(1.0, np.abs(want))
    bad = np.flatnonzero(err > lim)
    assert bad.size == 0, f"{bad.size} log-weights off: {got[bad[:5]]} vs {want[bad[:5]]}"


@pytest.mark.parametrize("u16", [False, True])
@pytest.mark.parametrize("B", [61, 1, 2, 7, 1081])
def test_sensor_weights_config1(G, oracle, u16, B):
    g = synth.rect_map(256, 256)
    mr = 300.0
    d = G.CDDT(dev(g), 108, mr, u16=u16)
    o = oracle.OracleCDDT(g, 108, mr, u16=u16)
    bo, D = _scan(B)
    gt = synth.uniform_particles(g, 1, seed=1700)[0]
    obs = gc.observations(o, gt, bo, mr)
    P = 1000 if B < 200 else 97
    parts = synth.uniform_particles(g, P, seed=1706)
    # a few particles off the map, in walls and with odd headings
    parts[:3] = [[-3.0, 5.0, 0.1], [1.0e4, 2.0, 1.0], [0.0, 0.0, 2.0]]
    parts[3, 2] = float("nan")
    m = G.beam_model(mr)
    om = oracle.beam_model(mr)
    logw, ranges = d.sensor_weights(dev(parts), dev(bo), dev(obs), m, D, want_ranges=True)
    want_logw, want_ranges = o.sensor_weights(parts, bo, obs, om, nthreads=8, want_ranges=True)
    assert_bits_equal(ranges.cpu().numpy(), want_ranges, "ranges")
    _logw_close(logw.cpu().numpy(), want_logw)
    # the pairing hint never changes a range
    logw0, ranges0 = d.sensor_weights(dev(parts), dev(bo), dev(obs), m, 0, want_ranges=True)
    assert_bits_equal(ranges0.cpu().numpy(), want_ranges, "ranges without pairing")
    _logw_close(logw0.cpu().numpy(), want_logw)
    # tree and binary search agree
    d.set_search(G.SEARCH_BINARY)
    logw1, ranges1 = d.sensor_weights(dev(parts), dev(bo), dev(obs), m, D, want_ranges=True)
    assert_bits_equal(ranges1.cpu().numpy(), want_ranges, "ranges (binary search)")


def test_sensor_truncnorm(G, oracle):
    g = synth.rect_map(128, 128, n_rects=15, seed=3)
    mr = 200.0
    d = G.CDDT(dev(g), 72, mr)
    o = oracle.OracleCDDT(g, 72, mr)
    bo, D = _scan(61)
    gt = synth.uniform_particles(g, 1, seed=4)[0]
    obs = gc.observations(o, gt, bo, mr)
    parts = synth.tracking_particles(gt.astype(np.float64), 500, seed=5)
    m = G.beam_model(mr, hit_truncnorm=1)
    om = oracle.beam_model(mr, hit_truncnorm=1)
    logw = d.sensor_weights(dev(parts), dev(bo), dev(obs), m, D).cpu().numpy()
    _logw_close(logw, o.sensor_weights(parts, bo, obs, om))
    g_gpu = d.sensor_weights_backward(dev(parts), dev(bo), dev(obs), m,
                                      torch.ones(500, device="cuda"), D).cpu().numpy()
    g_ref, scale = o.sensor_grad(parts, bo, obs, om)
    _grad_close(g_gpu, g_ref, scale)


def _grad_close(got, want, scale, rtol=1e-5):
    """Every gradient within rtol of the float64 oracle relative to the sum of
    its per-beam term magnitudes (the scale of a float32 sum's rounding, which
    bounds the error whatever the cancellation); and, where the terms cancel
    by less than a factor 10 (that sum <= 10 |g|), within rtol of |g| itself."""
    err = np.linalg.norm(np.asarray(got, np.float64) - want, axis=1)
    lim = rtol * np.maximum(np.linalg.norm(scale, axis=1), 1e-6)
    bad = np.flatnonzero(err > lim)
    assert bad.size == 0, f"{bad.size} gradients off: {got[bad[:3]]} vs {want[bad[:3]]}"
    gn = np.linalg.norm(want, axis=1)
    mild = (gn > 0) & (np.linalg.norm(scale, axis=1) <= 10 * gn)
    rel = err[mild] / gn[mild]
    assert mild.sum() >= len(gn) // 2, "too few samples without heavy cancellation to bound |g|-relative errors"
    assert rel.max() <= rtol, f"|g|-relative error {rel.max():.3g} on {mild.sum()} uncancelled samples"


@pytest.mark.parametrize("B", [61, 1081])
def test_adjoint(G, oracle, B):
    g = synth.rect_map(256, 256)
    mr = 300.0
    d = G.CDDT(dev(g), 108, mr)
    o = oracle.OracleCDDT(g, 108, mr)
    bo, D = _scan(B)
    gt = synth.uniform_particles(g, 1, seed=1800)[0]
    obs = gc.observations(o, gt, bo, mr)
    P = 777 if B == 61 else 64
    parts = synth.tracking_particles(gt.astype(np.float64), P, seed=1801)
    gl = synth.Stream(1802).uniform(P, -2.0, 2.0).astype(np.float32)
    m = G.beam_model(mr)
    om = oracle.beam_model(mr)
    got = d.sensor_weights_backward(dev(parts), dev(bo), dev(obs), m, dev(gl), D).cpu().numpy()
    want, scale = o.sensor_grad(parts, bo, obs, om, grad_logw=gl.astype(np.float64), nthreads=8)
    _grad_close(got, want, scale)
    logw, gxy = d.sensor_weights_fwd_bwd(dev(parts), dev(bo), dev(obs), m, D)
    want1, scale1 = o.sensor_grad(parts, bo, obs, om, nthreads=8)
    _grad_close(gxy.cpu().numpy(), want1, scale1)
    _logw_close(logw.cpu().numpy(), o.sensor_weights(parts, bo, obs, om, nthreads=8))


def test_autograd_function(G, oracle):
    g = synth.rect_map(128, 128, n_rects=20, seed=9)
    mr = 300.0
    d = G.CDDT(dev(g), 108, mr)
    o = oracle.OracleCDDT(g, 108, mr)
    bo, D = _scan(61)
    gt = synth.uniform_particles(g, 1, seed=10)[0]
    obs = gc.observations(o, gt, bo, mr)
    parts = dev(synth.tracking_particles(gt.astype(np.float64), 300, seed=11)).requires_grad_(True)
    m = G.beam_model(mr)
    logw = G.SensorWeights.apply(parts, d, dev(bo), dev(obs), m, D)
    w = torch.randn(300, device="cuda")
    (logw * w).sum().backward()
    direct = d.sensor_weights_backward(parts.detach(), dev(bo), dev(obs), m, w.contiguous(), D)
    torch.testing.assert_close(parts.grad[:, :2], direct, rtol=0, atol=0)
    assert torch.all(parts.grad[:, 2] == 0)


# ------------------------------------------------------------------ work figures

def test_work_counts_match_oracle(G, oracle):
    """The per-launch work figures used for the roofline equal the counts
    derived from the oracle's instrumented casts."""
    g = synth.rect_map(256, 256)
    mr = 300.0
    d = G.CDDT(dev(g), 108, mr)
    o = oracle.OracleCDDT(g, 108, mr)
    bo, D = _scan(61)
    parts = synth.uniform_particles(g, 2000, seed=21)
    parts[:2] = [[-3.0, 5.0, 0.1], [1.0, 1.0, float("inf")]]
    w = d.sensor_work(dev(parts), dev(bo), D)
    B = bo.size
    ths = (parts[:, 2:3] + bo[None, :]).astype(np.float32)
    q = np.concatenate([np.repeat(parts[:, :2], B, 0), ths.reshape(-1, 1)], 1)
    _, kb, _, _, _ = o.calc_range_info(q)
    kb = kb.reshape(-1, B)
    ks = np.array([[o.params.query_k(t) for t in row] for row in ths])
    N = 108
    paired = np.zeros_like(kb, dtype=bool)
    for i in range(B - D):
        j = i + D
        ok = (ks[:, i] >= 0) & (ks[:, j] >= 0) & (ks[:, j] == (ks[:, i] + N // 2) % N) & (kb[:, j] >= 0)
        paired[:, j] = ok
    looked = kb >= 0
    trav = looked & ~paired
    lg = np.ceil(np.log2(np.maximum(kb, 0).astype(np.float64) + 1))
    assert w["beams"] == int(looked.sum())
    assert w["paired"] == int(paired.sum())
    assert w["traversals"] == int(trav.sum())
    assert w["nonempty"] == int((trav & (kb > 0)).sum())
    assert w["probes"] == int(lg[trav].sum())
    assert w["sectors"] == int(oracle.sorted_search_sectors(kb[trav], 8).sum())
    gx = np.floor(parts[:, 0] + np.float32(0.5))
    gy = np.floor(parts[:, 1] + np.float32(0.5))
    inmap = (gx >= 0) & (gx < 256) & (gy >= 0) & (gy < 256)
    free = np.zeros(parts.shape[0], bool)
    free[inmap] = g[gy[inmap].astype(int), gx[inmap].astype(int)] == 0
    assert w["passed"] == int(free.sum())


def test_grid_states_and_warp_latency(G, oracle):
    """The grid benchmark's states (integer cell centres, headings on exact
    multiples of 2 pi / N, occupied and border cells included) cast exactly as
    the oracle; the latency-instrumented cast returns the same ranges and one
    positive cycle count per warp."""
    from paper_1705_01167_gb300 import workloads as WL
    g = synth.rect_map(256, 256)
    d = G.CDDT(dev(g), 108, 300.0)
    o = oracle.OracleCDDT(g, 108, 300.0)
    q = WL.grid_states(256, 256, 3, 108)
    got = d.calc_range_many(dev(q)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), o.calc_range(q).view(np.uint32))
    r, cyc = d.calc_range_timed(dev(q))
    assert np.array_equal(r.cpu().numpy().view(np.uint32), got.view(np.uint32))
    c = cyc.cpu().numpy()
    assert c.shape == ((q.shape[0] + 31) // 32,) and (c > 0).all()


def test_bresenham_baseline_matches_oracle(G, oracle):
    """The GPU Bresenham baseline caster walks the same digital lines as the
    oracle's (float32 end points by the direction rule, integer stepping)."""
    g = synth.rect_map(256, 256)
    d = G.CDDT(dev(g), 108, 300.0)
    q = gc.random_queries(256, 256, 20000, 31)
    q[:4] = [[-2.0, 10.0, 0.5], [10.0, 10.0, np.nan], [100.2, 50.7, 0.0], [255.4, 255.4, 0.785398]]
    got = d.cast_bresenham(dev(q)).cpu().numpy()
    want = oracle.cast_bresenham(g, q, 300.0)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_bresenham_full_size(G, oracle):
    """The Bresenham baseline on the bench's 2000 x 2000 corridor map (max
    range 1000): uniform queries and edge cases walked one by one by the
    oracle."""
    g = synth.corridor_map(2000, 2000)
    d = G.CDDT(dev(g), 200, 1000.0)
    q = np.concatenate([gc.special_queries(2000, 2000), synth.uniform_queries(g, 30000, seed=33)])
    got = d.cast_bresenham(dev(q)).cpu().numpy()
    want = oracle.cast_bresenham(g, q, 1000.0)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
