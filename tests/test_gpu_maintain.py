"""GPU pruning (Section IV-C) and incremental update (Section IV-D) against
the CPU oracle: pruned zero-point lists bit-exact with the oracle's prune and
answers unchanged; updated zero-point lists bit-exact with a build of the
updated grid."""
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


def bits_equal(a, b):
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def same_store(d, o):
    sb, bs, zp = d.export()
    obs_, ozp = o.export()
    assert np.array_equal(bs, obs_), "bin sizes differ"
    assert bits_equal(zp, ozp), "zero points differ"


# ------------------------------------------------------------------ prune

@pytest.mark.parametrize("u16", [False, True])
def test_prune_tiny_maps(G, oracle, u16):
    for mi, g in enumerate(gc.tiny_maps()):
        H, W = g.shape
        for N in (4, 8, 16):
            d = G.CDDT(dev(g), N, 37.5, u16=u16)
            o = oracle.OracleCDDT(g, N, 37.5, u16=u16)
            before = d.calc_range_many(dev(gc.random_queries(W, H, 2000, mi))).cpu().numpy()
            d.prune()
            o.prune()
            same_store(d, o)
            q = gc.random_queries(W, H, 2000, mi)
            after = d.calc_range_many(dev(q)).cpu().numpy()
            free = _free_mask(g, q)
            assert bits_equal(after[free], before[free])
            assert bits_equal(after, o.calc_range(q))


@pytest.mark.parametrize("u16", [False, True])
def test_prune_degenerate_maps(G, oracle, u16):
    """Single cells, single rows and columns, all-free and all-occupied maps
    (the prune's strips of one line or one cell), against the oracle's prune."""
    rs = synth.Stream(91)
    maps = [np.zeros((1, 1), np.uint8), np.ones((1, 1), np.uint8), np.zeros((4, 5), np.uint8),
            np.ones((3, 4), np.uint8), (rs.uniform(9) < 0.4).astype(np.uint8).reshape(1, 9),
            (rs.uniform(9) < 0.4).astype(np.uint8).reshape(9, 1),
            (rs.uniform(6) < 0.5).astype(np.uint8).reshape(2, 3)]
    for mi, g in enumerate(maps):
        H, W = g.shape
        for N in (4, 8, 36):
            d = G.CDDT(dev(g), N, 20.0, u16=u16)
            o = oracle.OracleCDDT(g, N, 20.0, u16=u16)
            d.prune()
            o.prune()
            same_store(d, o)
            q = gc.random_queries(W, H, 500, 100 + mi)
            assert bits_equal(d.calc_range_many(dev(q)).cpu().numpy(), o.calc_range(q)), (mi, N)


def _free_mask(g, q):
    H, W = g.shape
    fx = np.floor(q[:, 0] + np.float32(0.5))
    fy = np.floor(q[:, 1] + np.float32(0.5))
    ok = (fx >= 0) & (fx < W) & (fy >= 0) & (fy < H)
    free = np.zeros(q.shape[0], bool)
    free[ok] = g[fy[ok].astype(int), fx[ok].astype(int)] == 0
    return free


@pytest.mark.parametrize("u16", [False, True])
def test_prune_corridor_map(G, oracle, u16):
    g = synth.corridor_map(400, 300, seed=77, r_min=48)
    d = G.CDDT(dev(g), 120, 500.0, u16=u16)
    o = oracle.OracleCDDT(g, 120, 500.0, u16=u16)
    n0 = d.stats()["n_zero_points"]
    q = np.concatenate([synth.uniform_queries(g, 200000, seed=78), gc.grid_states(400, 300, 120, stride=13)])
    before = d.calc_range_many(dev(q)).cpu().numpy()
    d.prune()
    o.prune()
    st = d.stats()
    assert st["pruned"] == 1 and st["n_zero_points"] < n0 and st["prune_ms"] > 0
    same_store(d, o)
    after = d.calc_range_many(dev(q)).cpu().numpy()
    free = _free_mask(g, q)
    assert bits_equal(after[free], before[free])
    with pytest.raises(G.CDDTError) as e:
        d.prune()
    assert e.value.status == G.CDDT_ERR_PRUNED
    with pytest.raises(G.CDDTError) as e:
        d.update_cells(dev(np.array([[3, 3]], np.int32)), dev(np.array([1], np.uint8)))
    assert e.value.status == G.CDDT_ERR_PRUNED


# ------------------------------------------------------------------ update

@pytest.mark.parametrize("u16", [False, True])
def test_update_sequence_equals_rebuild(G, oracle, u16):
    g = synth.rect_map(96, 80, n_rects=14, seed=101)
    N, mr = 36, 150.0
    d = G.CDDT(dev(g), N, mr, u16=u16)
    o = oracle.OracleCDDT(g, N, mr, u16=u16)
    rs = synth.Stream(102)
    cur = g.copy()
    for step in range(6):
        n = int(rs.integers(1, 1, 400)[0])
        xy = np.stack([rs.integers(n, 0, 95), rs.integers(n, 0, 79)], 1).astype(np.int32)
        occ = (rs.uniform(n) < 0.5).astype(np.uint8)
        if step == 2:  # a solid block written, then partly cleared below
            blk = np.array([(x, y) for y in range(20, 30) for x in range(40, 52)], np.int32)
            xy = np.concatenate([xy, blk])
            occ = np.concatenate([occ, np.ones(len(blk), np.uint8)])
        if step == 3:
            blk = np.array([(x, y) for y in range(22, 28) for x in range(42, 50)], np.int32)
            xy = np.concatenate([xy, blk])
            occ = np.concatenate([occ, np.zeros(len(blk), np.uint8)])
        d.update_cells(dev(xy), dev(occ))
        assert d.status() == G.CDDT_OK
        assert o.update(xy, occ) == 0
        for (x, y), v in zip(xy, occ):
            cur[y, x] = v
        same_store(d, o)
        ref = oracle.OracleCDDT(cur, N, mr, u16=u16)
        same_store(d, ref)
        gg, ee = d.export_grid()
        assert np.array_equal(gg, cur)
        assert np.array_equal(ee, oracle.edge_map(cur))
    q = gc.random_queries(96, 80, 20000, 5)
    assert bits_equal(d.calc_range_many(dev(q)).cpu().numpy(), o.calc_range(q))
    assert d.stats()["update_ms"] > 0


@pytest.mark.parametrize("u16", [False, True])
def test_update_bin_with_many_deltas(G, oracle, u16):
    """A wall of 300 cells written along one row, then half of it cleared:
    the row's bins get hundreds of inserts and deletes (the merge's sorted
    path), while other bins get a handful (its unsorted path)."""
    g = np.zeros((64, 512), np.uint8)
    g[0, :] = g[-1, :] = 1
    g[:, 0] = g[:, -1] = 1
    N, mr = 40, 600.0
    d = G.CDDT(dev(g), N, mr, u16=u16)
    cur = g.copy()
    wall = np.array([(x, 30) for x in range(100, 400)], np.int32)
    for xy, occ in ((wall, np.ones(len(wall), np.uint8)), (wall[::2], np.zeros(len(wall[::2]), np.uint8)),
                    (np.array([[5, 5], [6, 5], [7, 9]], np.int32), np.ones(3, np.uint8))):
        d.update_cells(dev(xy), dev(occ))
        assert d.status() == G.CDDT_OK
        for (x, y), v in zip(xy, occ):
            cur[y, x] = v
        same_store(d, oracle.OracleCDDT(cur, N, mr, u16=u16))
    q = gc.random_queries(512, 64, 20000, 6)
    ref = oracle.OracleCDDT(cur, N, mr, u16=u16)
    assert bits_equal(d.calc_range_many(dev(q)).cpu().numpy(), ref.calc_range(q))


@pytest.mark.parametrize("u16", [False, True])
def test_update_light_heavy_boundary(G, oracle, u16):
    """Bins at the edge between the two merges: a one-cell wall of 32 cells
    along a row gives that row's slice-0 bin exactly 32 inserts (the light
    merge's limit), one of 33 cells 33 (the sorted merge); then one update
    clears the 32-cell wall and draws another 32 cells in the same row (32
    deletes and 32 inserts in one bin), and the 33-cell wall is cleared."""
    g = np.zeros((64, 512), np.uint8)
    g[0, :] = g[-1, :] = 1
    g[:, 0] = g[:, -1] = 1
    N, mr = 40, 600.0
    d = G.CDDT(dev(g), N, mr, u16=u16)
    cur = g.copy()
    a = np.array([(x, 20) for x in range(100, 132)], np.int32)
    b = np.array([(x, 40) for x in range(200, 233)], np.int32)
    c = np.array([(x, 20) for x in range(300, 332)], np.int32)
    steps = ((np.concatenate([a, b]), np.ones(len(a) + len(b), np.uint8)),
             (np.concatenate([a, c, b]), np.concatenate([np.zeros(len(a), np.uint8), np.ones(len(c), np.uint8),
                                                         np.zeros(len(b), np.uint8)])))
    for xy, occ in steps:
        d.update_cells(dev(xy), dev(occ))
        assert d.status() == G.CDDT_OK
        for (x, y), v in zip(xy, occ):
            cur[y, x] = v
        same_store(d, oracle.OracleCDDT(cur, N, mr, u16=u16))
    q = gc.random_queries(512, 64, 20000, 7)
    ref = oracle.OracleCDDT(cur, N, mr, u16=u16)
    assert bits_equal(d.calc_range_many(dev(q)).cpu().numpy(), ref.calc_range(q))


def test_update_repeated_cells_last_write_wins(G, oracle):
    g = synth.rect_map(64, 64, n_rects=6, seed=5)
    d = G.CDDT(dev(g), 24, 100.0)
    xy = np.array([[10, 10], [10, 10], [10, 10], [20, 20], [20, 20]], np.int32)
    occ = np.array([1, 0, 1, 1, 0], np.uint8)
    d.update_cells(dev(xy), dev(occ))
    cur = g.copy()
    cur[10, 10] = 1
    cur[20, 20] = 0
    same_store(d, oracle.OracleCDDT(cur, 24, 100.0))
    # writing the current state is a no-op
    before = d.export()
    d.update_cells(dev(xy[:1]), dev(occ[:1]))
    after = d.export()
    assert np.array_equal(before[1], after[1]) and bits_equal(before[2], after[2])


def test_update_out_of_map_flags_status(G, oracle):
    g = synth.rect_map(48, 48, n_rects=5, seed=6)
    d = G.CDDT(dev(g), 16, 80.0)
    xy = np.array([[5, 5], [-1, 3], [48, 2], [7, 7]], np.int32)
    occ = np.array([1, 1, 1, 1], np.uint8)
    d.update_cells(dev(xy), dev(occ))
    assert d.status() == G.CDDT_ERR_DEVICE
    assert d.status() == G.CDDT_OK  # reading clears it
    cur = g.copy()
    cur[5, 5] = 1
    cur[7, 7] = 1
    same_store(d, oracle.OracleCDDT(cur, 16, 80.0))


def test_update_large_map_sampled(G, oracle):
    """A 1024 x 1024 corridor map with 2000 toggles: whole-store equality
    with a CPU build of the updated grid, and sensor weights on it."""
    g = synth.corridor_map(1024, 1024, seed=31, r_min=64)
    N, mr = 96, 800.0
    d = G.CDDT(dev(g), N, mr)
    xy, occ = synth.cell_toggles(g, 1000, 1000, seed=32)
    d.update_cells(dev(xy), dev(occ))
    assert d.status() == G.CDDT_OK
    cur = g.copy()
    for (x, y), v in zip(xy, occ):
        cur[y, x] = v
    o = oracle.OracleCDDT(cur, N, mr)
    same_store(d, o)
    bo = synth.beam_offsets(61)
    parts = synth.uniform_particles(cur, 3000, seed=33)
    gt = synth.uniform_particles(cur, 1, seed=34)[0]
    obs = gc.observations(o, gt, bo, mr)
    m = G.beam_model(mr)
    _, ranges = d.sensor_weights(dev(parts), dev(bo), dev(obs), m, 40, want_ranges=True)
    _, want = o.sensor_weights(parts, bo, obs, oracle.beam_model(mr), nthreads=8, want_ranges=True)
    assert bits_equal(ranges.cpu().numpy(), want)


def test_update_empty_batch(G):
    g = synth.rect_map(32, 32, n_rects=3, seed=7)
    d = G.CDDT(dev(g), 8, 50.0)
    d.update_cells(torch.empty((0, 2), dtype=torch.int32, device="cuda"),
                   torch.empty(0, dtype=torch.uint8, device="cuda"))
    assert d.status() == G.CDDT_OK


# ------------------------------------------------------------------ import

@pytest.mark.parametrize("u16", [False, True])
def test_import_round_trip(G, oracle, u16):
    """cddt_import of an exported store answers exactly as the original,
    before and after the same update, and restores a pruned store."""
    g = synth.corridor_map(300, 260, seed=61, r_min=48)
    N, mr = 72, 400.0
    d = G.CDDT(dev(g), N, mr, u16=u16)
    sb, bs, zp = d.export()
    d2 = G.CDDT.from_export(dev(g), N, mr, bs, zp, u16=u16)
    sb2, bs2, zp2 = d2.export()
    assert np.array_equal(bs, bs2) and np.array_equal(zp.view(np.uint32), zp2.view(np.uint32))
    assert d2.stats()["n_zero_points"] == d.stats()["n_zero_points"]
    q = gc.random_queries(300, 260, 20000, 62)
    assert bits_equal(d2.calc_range_many(dev(q)).cpu().numpy(), d.calc_range_many(dev(q)).cpu().numpy())
    xy, occ = synth.cell_toggles(g, 300, 300, seed=63)
    d.update_cells(dev(xy), dev(occ))
    d2.update_cells(dev(xy), dev(occ))
    assert d2.status() == G.CDDT_OK
    same = d.export()
    assert np.array_equal(same[1], d2.export()[1])
    assert bits_equal(d2.calc_range_many(dev(q)).cpu().numpy(), d.calc_range_many(dev(q)).cpu().numpy())
    # a pruned store comes back pruned (updates refused)
    d.prune()
    _, bsp, zpp = d.export()
    d3 = G.CDDT.from_export(dev(synth.apply_writes(g, xy, occ)), N, mr, bsp, zpp, u16=u16, pruned=True)
    assert d3.stats()["pruned"] == 1
    assert bits_equal(d3.calc_range_many(dev(q)).cpu().numpy(), d.calc_range_many(dev(q)).cpu().numpy())
    with pytest.raises(G.CDDTError):
        d3.update_cells(dev(xy[:1]), dev(occ[:1]))


def test_import_rejects_mismatched_csr(G):
    g = synth.rect_map(128, 96, seed=64)
    d = G.CDDT(dev(g), 40, 200.0)
    _, bs, zp = d.export()
    with pytest.raises(G.CDDTError):  # other theta_disc: another bin count
        G.CDDT.from_export(dev(g), 44, 200.0, bs, zp)
    bad = zp.copy()
    i = int(np.argmax(np.diff(bs) > 2))
    a = bs[i]
    bad[a], bad[a + 1] = bad[a + 1] + 1.0, bad[a]  # an unsorted bin
    with pytest.raises(G.CDDTError):
        G.CDDT.from_export(dev(g), 40, 200.0, bs, bad)


def test_injected_faults_leave_handles_usable(G, oracle, monkeypatch):
    """Host-injected failures (CDDT_FAULT) surface as errors of the named
    call; the handle and plan keep working once the variable is cleared."""
    g = synth.rect_map(96, 80, seed=71)
    d = G.CDDT(dev(g), 36, 150.0)
    o = oracle.OracleCDDT(g, 36, 150.0)
    q = dev(gc.random_queries(96, 80, 5000, 72))
    before = d.export()
    monkeypatch.setenv("CDDT_FAULT", "launch:cddt_calc_range_many")
    with pytest.raises(G.CDDTError) as e:
        d.calc_range_many(q)
    assert e.value.status == G.CDDT_ERR_CUDA
    monkeypatch.setenv("CDDT_FAULT", "oom:cddt_update_cells")
    xy, occ = synth.cell_toggles(g, 50, 50, seed=73)
    with pytest.raises(G.CDDTError) as e:
        d.update_cells(dev(xy), dev(occ))
    assert e.value.status == G.CDDT_ERR_OOM
    after = d.export()
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[2], after[2])
    bo = dev(synth.beam_offsets(61))
    obs = dev(gc.observations(o, synth.uniform_particles(g, 1, seed=74)[0], synth.beam_offsets(61), 150.0))
    parts = dev(synth.uniform_particles(g, 300, seed=75))
    logw = torch.empty(300, device="cuda")
    plan = G.Plan([dict(map=d, particles=parts, beam_off=bo, obs=obs, model=G.beam_model(150.0), logw=logw,
                        pair_offset=synth.pair_offset(61))])
    monkeypatch.setenv("CDDT_FAULT", "timeout:cddt_plan_run")
    with pytest.raises(G.CDDTError) as e:
        plan.run()
    assert e.value.status == G.CDDT_ERR_TIMEOUT
    monkeypatch.delenv("CDDT_FAULT")
    plan.run()
    want = d.sensor_weights(parts, bo, obs, G.beam_model(150.0), synth.pair_offset(61))
    assert torch.allclose(logw, want, rtol=1e-5, atol=1e-5)
    assert bits_equal(d.calc_range_many(q).cpu().numpy(), o.calc_range(q.cpu().numpy()))
    plan.close()
