"""The seeded input generators against their stated recipe: SplitMix64's
published output sequence, determinism, the maps' structure and occupancy,
particles in free cells, the 61-beam 270-degree scan and its pairing, and
the cell-write batches.  (Generators only; they hold none of the method's
arithmetic.)"""
import math

import numpy as np

from paper_1705_01167_gb300 import synth, workloads as WL


def test_splitmix64_published_sequence():
    """SplitMix64 (Steele, Lea & Flood; Vigna's reference code) from state
    1234567 yields 6457827717110365317, 3203168211198807973,
    9817491932198370423: the stream's mixer and increment reproduce it."""
    with np.errstate(over="ignore"):
        st = np.uint64(1234567)
        out = [int(synth._mix64(np.array([st + np.uint64(i) * synth.GAMMA], np.uint64))[0]) for i in (1, 2, 3)]
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_streams_are_deterministic_and_in_range():
    a, b = synth.Stream(5), synth.Stream(5)
    assert np.array_equal(a.u64(100), b.u64(100))
    assert not np.array_equal(synth.Stream(6).u64(100), synth.Stream(5).u64(100))
    u = synth.Stream(7).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    k = synth.Stream(8).integers(100000, 3, 9)
    assert k.min() == 3 and k.max() == 9 and set(np.unique(k)) == set(range(3, 10))
    z = synth.Stream(9).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_maps_follow_the_recipe():
    g = synth.rect_map(256, 256)
    assert g.dtype == np.uint8 and g.shape == (256, 256)
    assert g[0].all() and g[-1].all() and g[:, 0].all() and g[:, -1].all()
    assert math.isclose(synth.occupancy(g), 0.16827, abs_tol=1e-4)  # the value the design notes report
    assert np.array_equal(g, synth.rect_map(256, 256))
    c = synth.corridor_map(2000, 2000)
    assert c[0].all() and c[-1].all() and c[:, 0].all() and c[:, -1].all()
    assert math.isclose(synth.occupancy(c), 0.0797, abs_tol=2e-4)
    assert not np.array_equal(c, synth.corridor_map(2000, 2000, seed=synth.SEED_MAP + 1))
    # every interior wall run across a row or column is 1..3 cells thick:
    # no 4 x 4 block of the corridor map is fully occupied
    inner = c[1:-1, 1:-1].astype(np.int32)
    s = np.pad(inner, ((1, 0), (1, 0))).cumsum(0).cumsum(1)
    blocks = s[4:, 4:] - s[:-4, 4:] - s[4:, :-4] + s[:-4, :-4]
    assert blocks.max() < 16


def test_particles_queries_and_scan():
    g = synth.corridor_map(500, 500, r_min=48)
    p = synth.uniform_particles(g, 5000, seed=3)
    ix = np.floor(p[:, 0] + 0.5).astype(int)
    iy = np.floor(p[:, 1] + 0.5).astype(int)
    assert (g[iy, ix] == 0).all()
    assert (p[:, 2] >= 0).all() and (p[:, 2] < 2 * np.pi).all()
    q = synth.uniform_queries(g, 5000, seed=4)
    assert (g[np.floor(q[:, 1] + 0.5).astype(int), np.floor(q[:, 0] + 0.5).astype(int)] == 0).all()
    gt = synth.random_free_pose(g, synth.Stream(5))
    tp = synth.tracking_particles(gt.astype(np.float64), 20000, seed=6)
    assert np.allclose(tp[:, :2].mean(0), gt[:2], atol=0.2)
    assert np.allclose(tp[:, :2].std(0), 5.0, rtol=0.05)
    # 61 beams over 270 degrees, 4.5 degrees apart; beam i + 40 is opposite beam i
    bo = synth.beam_offsets(61)
    assert bo.dtype == np.float32 and bo.size == 61
    assert np.isclose(bo[0], -0.75 * np.pi) and np.isclose(bo[-1], 0.75 * np.pi)
    assert np.allclose(np.diff(bo.astype(np.float64)), np.deg2rad(4.5), atol=1e-6)
    D = synth.pair_offset(61)
    assert D == 40 and np.allclose(bo[D:].astype(np.float64) - bo[:61 - D], np.pi, atol=1e-6)
    assert synth.pair_offset(1081) == 720
    n = synth.noise(100000, 2.0, seed=7)
    assert abs(n.mean()) < 0.03 and abs(n.std() - 2.0) < 0.03


def test_cell_writes_and_workloads():
    g = synth.rect_map(128, 96, n_rects=10, seed=9)
    xy, occ = synth.cell_toggles(g, 300, 200, seed=10)
    assert xy.dtype == np.int32 and occ.dtype == np.uint8 and xy.shape == (500, 2)
    assert occ.sum() == 300
    ins, rem = xy[occ == 1], xy[occ == 0]
    assert (g[ins[:, 1], ins[:, 0]] == 0).all() and (g[rem[:, 1], rem[:, 0]] == 1).all()
    g2 = synth.apply_writes(g, xy, occ)
    assert (g2[ins[:, 1], ins[:, 0]] == 1).all()
    st = WL.grid_states(8, 6, 2, 4)
    assert st.shape == (4 * 3 * 4, 3) and st[:4, 2].tolist() == [0.0, 0.0, 0.0, 0.0]
    w = WL.corridor2000(steps=3, particles=64, sweep=10)
    assert w["parts"].shape == (3, 64, 3) and w["theta_disc"] == 200 and w["max_range"] == 1000.0
