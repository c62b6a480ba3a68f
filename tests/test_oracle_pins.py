"""Pins of the CPU oracle against facts fixed outside it: the paper's worked
example (Fig. 4), axis-aligned geometry, library routines, brute force on tiny
maps, closed forms and invariants stated in the paper."""
import math
import os

import numpy as np
import pytest

from paper_1705_01167_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig4():
    grid, lut, cur = [], [], None
    with open(os.path.join(GOLDEN, "fig4_theta0.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("grid", "lut_theta0"):
                cur = grid if line == "grid" else lut
                continue
            cur.append(line.split())
    g = np.array([[int(v) for v in r] for r in grid], np.uint8)
    return g, lut


def _tiny_maps(n_maps=6, seed=11):
    rs = synth.Stream(seed)
    out = []
    for m in range(n_maps):
        W = int(rs.integers(1, 5, 20)[0])
        H = int(rs.integers(1, 5, 20)[0])
        dens = rs.uniform(1, 0.05, 0.45)[0]
        g = (rs.uniform(W * H) < dens).astype(np.uint8).reshape(H, W)
        out.append(g)
    # a map with a solid 3x3 block (interior cell that is not an edge)
    g = np.zeros((9, 11), np.uint8)
    g[3:6, 4:7] = 1
    out.append(g)
    return out


def _grid_states(W, H, N):
    th = np.array([np.float32(2.0 * math.pi * k / N) for k in range(N)], np.float32)
    jj, ii, kk = np.meshgrid(np.arange(H), np.arange(W), np.arange(N), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel(), th[kk.ravel()]], 1).astype(np.float32)


def _random_queries(W, H, n, seed):
    rs = synth.Stream(seed)
    x = rs.uniform(n, -0.7, W - 0.3)
    y = rs.uniform(n, -0.7, H - 0.3)
    th = rs.uniform(n, -7.0, 14.0)
    return np.stack([x, y, th], 1).astype(np.float32)


# ------------------------------------------------------------------ Fig. 4

def test_fig4_worked_example(oracle):
    """Fig. 4: the theta = 0 LUT slice of the 4x4 example, cast at cell centres."""
    g, lut = _read_fig4()
    max_range = 100.0
    d = oracle.OracleCDDT(g, 8, max_range)
    poses = np.array([[i, j, 0.0] for j in range(4) for i in range(4)], np.float32)
    want = np.array([[max_range if v == "-" else float(v) for v in row] for row in lut], np.float32)
    np.testing.assert_array_equal(d.calc_range(poses).reshape(4, 4), want)
    np.testing.assert_array_equal(d.params.calc_range_brute(g, poses).reshape(4, 4), want)
    # the same slice from the 16-bit variant: the zero points are integers
    d16 = oracle.OracleCDDT(g, 8, max_range, u16=True)
    np.testing.assert_array_equal(d16.calc_range(poses).reshape(4, 4), want)


# ------------------------------------------------------------------ edge map

def test_edge_map_is_map_minus_erosion(oracle):
    """Section IV-A: edge_map = map - erosion(map), 3x3 structuring element,
    off-map cells count as free (scipy's binary erosion, border_value=0)."""
    from scipy import ndimage
    rs = synth.Stream(5)
    for _ in range(5):
        g = (rs.uniform(40 * 33) < 0.6).astype(np.uint8).reshape(33, 40)
        er = ndimage.binary_erosion(g.astype(bool), structure=np.ones((3, 3), bool), border_value=0)
        want = (g.astype(bool) & ~er).astype(np.uint8)
        np.testing.assert_array_equal(oracle.edge_map(g), want)


# ------------------------------------------------------------------ O1 == O2

@pytest.mark.parametrize("u16", [False, True])
def test_plain_cddt_equals_brute_force(oracle, u16):
    """The stored, sorted, binary-searched CDDT (O2) answers every grid state
    and random continuous queries exactly as the definition scanned over all
    edge cells (O1)."""
    for mi, g in enumerate(_tiny_maps()):
        H, W = g.shape
        for N in (4, 8, 12, 16):
            d = oracle.OracleCDDT(g, N, 37.5, u16=u16)
            q = np.concatenate([_grid_states(W, H, N), _random_queries(W, H, 800, 100 + mi)])
            np.testing.assert_array_equal(d.calc_range(q), d.params.calc_range_brute(g, q))


def test_lut_equals_cddt_at_grid_states(oracle):
    """O4 (a lookup table of every discrete state, Section II) read at each
    state equals the CDDT cast from that state."""
    g = _tiny_maps()[2]
    H, W = g.shape
    N = 12
    d = oracle.OracleCDDT(g, N, 50.0)
    lut = d.params.lut(g)
    assert lut.shape == (N, H, W)
    q = _grid_states(W, H, N)  # ordered (j, i, k)
    got = d.calc_range(q).reshape(H, W, N).transpose(2, 0, 1)
    np.testing.assert_array_equal(got, lut)


def test_lut_memory_closed_forms():
    """Reading S1 (N directions span the full circle) reproduces the paper's
    lookup-table sizes at 16 bits per entry: 1000^2 x 108 x 2 B = 216 MB
    (Table I) and 2000^2 x 200 x 2 B > 1.5 GB (Section I)."""
    assert 1000 * 1000 * 108 * 2 == 216_000_000
    assert 2000 * 2000 * 200 * 2 > 1.5e9
    assert 4000 * 4000 * 200 * 2 > 6e9


# ------------------------------------------------------------------ axis-aligned

def _walk(g, i, j, di, dj):
    """First occupied cell from (i, j) stepping by (di, dj), or None."""
    H, W = g.shape
    while True:
        i += di
        j += dj
        if not (0 <= i < W and 0 <= j < H):
            return None
        if g[j, i]:
            return i, j


@pytest.mark.parametrize("N", [8, 108, 200])
def test_axis_aligned_rays_are_exact(oracle, N):
    """At theta = 0, pi/2, pi, 3pi/2 a CDDT range is exactly the distance from
    the query to the centre of the first occupied cell along the axis
    (Section III's d_ray with the cell centre as the collision point), and a
    query in an occupied cell returns 0 (Section IV-C pre-check)."""
    g = synth.rect_map(64, 48, n_rects=12, seed=21)
    H, W = g.shape
    mr = 300.0
    d = oracle.OracleCDDT(g, N, mr)
    rs = synth.Stream(22)
    n = 3000
    ci = rs.integers(n, 0, W - 1)
    cj = rs.integers(n, 0, H - 1)
    fx = rs.uniform(n, -0.499, 0.499)
    fy = rs.uniform(n, -0.499, 0.499)
    dirs = [(0.0, 1, 0), (math.pi / 2, 0, 1), (math.pi, -1, 0), (3 * math.pi / 2, 0, -1)]
    for th, di, dj in dirs:
        q = np.stack([ci + fx, cj + fy, np.full(n, th)], 1).astype(np.float32)
        got = d.calc_range(q)
        for t in range(n):
            x, y = q[t, 0], q[t, 1]
            i, j = int(ci[t]), int(cj[t])
            if g[j, i]:
                assert got[t] == 0.0
                continue
            hit = _walk(g, i, j, di, dj)
            if hit is None:
                want = np.float32(mr)
            elif di:
                want = np.float32(hit[0]) - x if di > 0 else x - np.float32(hit[0])
            else:
                want = np.float32(hit[1]) - y if dj > 0 else y - np.float32(hit[1])
            assert got[t] == min(want, np.float32(mr)), (th, x, y, got[t], want)


def test_max_range_clamp(oracle):
    """Ranges are clamped to max_range (Section III's ray cast up to the sensor
    limit): with a short limit every axis-aligned range equals
    min(distance to the first wall centre, max_range)."""
    g = synth.rect_map(64, 64, n_rects=6, seed=23)
    mr = 6.0
    d = oracle.OracleCDDT(g, 16, mr)
    q = np.array([[i, j, 0.0] for j in range(64) for i in range(64) if not g[j, i]], np.float32)
    r = d.calc_range(q)
    assert np.all(r <= np.float32(mr))
    for t in range(q.shape[0]):
        i, j = int(q[t, 0]), int(q[t, 1])
        hit = _walk(g, i, j, 1, 0)
        want = mr if hit is None else min(float(hit[0] - i), mr)
        assert r[t] == np.float32(want)
    assert np.mean(r == np.float32(mr)) > 0.2


def test_sawtooth_rows(oracle):
    """Section IV: along a row of the theta = 0 slice the distance grows by
    exactly one per cell and drops to zero at an obstacle (Fig. 5)."""
    g = synth.rect_map(80, 60, n_rects=15, seed=31)
    H, W = g.shape
    d = oracle.OracleCDDT(g, 108, 1000.0)
    q = np.array([[i, j, 0.0] for j in range(H) for i in range(W)], np.float32)
    r = d.calc_range(q).reshape(H, W)
    for j in range(H):
        for i in range(W - 1):
            if g[j, i]:
                assert r[j, i] == 0
            elif g[j, i + 1]:
                assert r[j, i] == 1
            else:
                assert r[j, i] == r[j, i + 1] + 1


def test_empty_map_and_occupied_cells(oracle):
    """An empty map has no zero points: every in-map query returns max_range.
    A query inside an occupied cell, or off the map, returns 0."""
    g = np.zeros((30, 40), np.uint8)
    for u16 in (False, True):
        d = oracle.OracleCDDT(g, 36, 123.0, u16=u16)
        assert d.total_zp == 0
        q = _random_queries(40, 30, 2000, 3)
        inside = (np.floor(q[:, 0] + np.float32(0.5)) >= 0) & (np.floor(q[:, 0] + np.float32(0.5)) < 40) \
            & (np.floor(q[:, 1] + np.float32(0.5)) >= 0) & (np.floor(q[:, 1] + np.float32(0.5)) < 30)
        r = d.calc_range(q)
        assert np.all(r[inside] == np.float32(123.0))
        assert np.all(r[~inside] == 0.0)
    g = synth.rect_map(50, 50, n_rects=8, seed=4)
    d = oracle.OracleCDDT(g, 24, 80.0)
    jj, ii = np.nonzero(g)
    th = synth.Stream(6).uniform(ii.size, 0, 2 * math.pi)
    q = np.stack([ii + 0.3, jj - 0.2, th], 1).astype(np.float32)
    assert np.all(d.calc_range(q) == 0.0)


def test_theta_wraps(oracle):
    """theta and theta + 2 pi m name the same discrete direction."""
    g = synth.rect_map(60, 60, n_rects=10, seed=8)
    d = oracle.OracleCDDT(g, 60, 200.0)
    N = 60
    ks = np.arange(N)
    th = np.array([np.float32(2 * math.pi * k / N) for k in ks], np.float32)
    assert [d.params.query_k(t) for t in th] == list(ks)
    # a direction just below / above the half-way point between two slices
    step = 2 * math.pi / N
    assert d.params.query_k(np.float32(0.49 * step)) == 0
    assert d.params.query_k(np.float32(0.51 * step)) == 1
    assert d.params.query_k(np.float32(-0.49 * step)) == 0
    assert d.params.query_k(np.float32(-0.51 * step)) == N - 1
    rs = synth.Stream(9)
    n = 2000
    q = _random_queries(60, 60, n, 10)
    q[:, 2] = rs.uniform(n, 0.001, 2 * math.pi - 0.001)
    # keep directions away from the rounding boundary so the float32 shift
    # by 2 pi cannot move them across it
    frac = (q[:, 2] * N / (2 * math.pi)) % 1.0
    q = q[np.abs(frac - 0.5) > 1e-3]
    q2 = q.copy()
    q2[:, 2] = q[:, 2] + np.float32(2 * math.pi)
    q3 = q.copy()
    q3[:, 2] = q[:, 2] - np.float32(2 * math.pi)
    r = d.calc_range(q)
    np.testing.assert_array_equal(r, d.calc_range(q2))
    np.testing.assert_array_equal(r, d.calc_range(q3))


# ------------------------------------------------------------------ symmetry, pairing

def test_half_storage_matches_full_circle(oracle):
    """Section IV-C: one set of zero points answers theta and theta + pi; the
    half-storage CDDT with a backward search equals a CDDT that stores all N
    directions, on every query not within 1e-4 of a bin edge."""
    g = synth.rect_map(70, 50, n_rects=14, seed=41)
    H, W = g.shape
    N = 36
    half = oracle.OracleCDDT(g, N, 150.0)
    full = oracle.OracleCDDT(g, N, 150.0, full=True)
    ph, pf = half.params, full.params
    # the stored tables of directions s and s + N/2 are exact negations
    S = N // 2
    exact = np.array([pf.c[s + S] == -ph.c[s] and pf.s[s + S] == -ph.s[s] for s in range(S)])
    q = _random_queries(W, H, 20000, 42)
    k = np.array([ph.query_k(t) for t in q[:, 2]])
    s = k % S
    yr = q[:, 1] * ph.c[s] - q[:, 0] * ph.s[s]
    away = np.abs((yr % 1.0) - 0.5) > 1e-4
    sel = away & exact[s]
    assert sel.sum() > 10000
    np.testing.assert_array_equal(half.calc_range(q[sel]), full.calc_range(q[sel]))


def test_radial_pairing(oracle):
    """Section IV-C and VI: with a 270-degree, 61-beam scan, beams i and i + 40
    point opposite ways; when their slices coincide the backward answer sits at
    index i - 1 of the forward search, and 21 pairs leave 40 traversals,
    'a third' fewer than 61."""
    B = 61
    bo = synth.beam_offsets(B, 270.0)
    D = synth.pair_offset(B, 270.0)
    assert D == 40
    assert abs((float(bo[D]) - float(bo[0])) - math.pi) < 1e-6
    g = synth.rect_map(128, 128, n_rects=20, seed=51)
    d = oracle.OracleCDDT(g, 108, 300.0)
    parts = synth.uniform_particles(g, 400, seed=52)
    trav = np.array([d.params.traversals(t, bo, D) for t in parts[:, 2]])
    assert trav.min() >= 40 and trav.max() <= B
    assert np.mean(trav == 40) > 0.6
    assert abs(1.0 - np.mean(trav) / B - 1.0 / 3.0) < 0.03
    # index relation of Section IV-C on every valid pair
    ths = (parts[:, 2:3] + bo[None, :]).astype(np.float32)
    q = np.concatenate([np.repeat(parts[:, :2], B, 0), ths.reshape(-1, 1)], 1)
    r, kb, zi, sl, b = d.calc_range_info(q)
    r, kb, zi, sl = (a.reshape(-1, B) for a in (r, kb, zi, sl))
    checked = 0
    for p in range(parts.shape[0]):
        for i in range(B - D):
            ki = d.params.query_k(ths[p, i])
            kj = d.params.query_k(ths[p, i + D])
            if kj != (ki + 54) % 108 or kb[p, i] < 0:
                continue
            f, r_ = (i, i + D) if ki < 54 else (i + D, i)
            ub = zi[p, f] if zi[p, f] >= 0 else kb[p, f]
            assert zi[p, r_] == ub - 1
            checked += 1
    assert checked > 4000


# ------------------------------------------------------------------ approximation

def test_exact_caster_closed_forms(oracle):
    """The exact voxel-traversal caster (O3, Amanatides & Woo) on rays whose
    answers are known by hand.  Mode 0 returns the distance along the ray to
    the projection of the first crossed occupied cell's centre, mode 1 the
    distance to the ray's entry point into that cell.
    (a) Axis rays in a box with 1-cell border walls from a fractional start:
    +x hits column W-1 (mode 0: W-1-x, mode 1: W-1.5-x), -x column 0 (x and
    x - 0.5), and likewise in y; a pillar in the way is hit first.
    (b) The start cell is the nearest cell centre: from x = 3.49 the pillar at
    column 4 is one cell away, from x = 3.51 the start is the pillar (range 0).
    A wall entered within max_range whose centre projects beyond it returns
    max_range in mode 0.
    (c) Rays from a cell centre just either side of 45 degrees pass next to
    cell corners: with only the cells just above the diagonal occupied, a ray
    a hair above 45 degrees crosses the y face first, into (i, i + 1) at
    t = 0.5 / sin(theta) (mode 1; mode 0: its centre projects to sin(theta)),
    while one a hair below crosses x faces first all the way and meets
    nothing (max_range).  Through a checkerboard of occupied (i + j odd)
    cells a 45-degree ray from (i + 0.1, j - 0.2) leaves through the x face
    first, into cell (i + 1, j) at t = 0.4 / cos 45 (mode 1), whose centre
    projects to 1.1 cos 45 (mode 0).
    (d) A sloped ray to a vertical wall at column 20 enters it through the
    wall's left face at t = (19.5 - x) / cos(theta) (mode 1); mode 0 is the
    projection of the centre of the wall cell in the row the ray is in
    there."""
    W, H = 30, 20
    box = np.zeros((H, W), np.uint8)
    box[0, :] = box[-1, :] = box[:, 0] = box[:, -1] = 1
    x, y, mr = 7.3, 11.6, 100.0
    rays = [(0.0, W - 1 - x, W - 1.5 - x), (math.pi, x, x - 0.5), (math.pi / 2, H - 1 - y, H - 1.5 - y),
            (1.5 * math.pi, y, y - 0.5)]
    for th, want0, want1 in rays:
        q = np.array([[x, y, th]])
        assert oracle.cast_exact(box, q, mr, 0)[0] == pytest.approx(want0, abs=1e-9), th
        assert oracle.cast_exact(box, q, mr, 1)[0] == pytest.approx(want1, abs=1e-9), th
    pillar = box.copy()
    pillar[12, 4] = 1  # column 4, row 12 (the row of y = 11.6)
    q = np.array([[1.2, 11.6, 0.0], [3.49, 11.6, 0.0], [3.51, 11.6, 0.0]])
    assert np.allclose(oracle.cast_exact(pillar, q, mr, 0), [4 - 1.2, 4 - 3.49, 0.0], atol=1e-9)
    assert np.allclose(oracle.cast_exact(pillar, q, mr, 1), [3.5 - 1.2, 3.5 - 3.49, 0.0], atol=1e-9)
    # the short ray ends at max_range; a wall entered within max_range whose
    # centre projects beyond it is clamped to max_range (mode 0)
    assert oracle.cast_exact(box, np.array([[x, y, 0.0]]), 5.0, 1)[0] == 5.0
    assert oracle.cast_exact(box, np.array([[x, y, 0.0]]), W - 1.4 - x, 0)[0] == pytest.approx(W - 1.4 - x)
    assert oracle.cast_exact(box, np.array([[x, y, 0.0]]), W - 1.4 - x, 1)[0] == pytest.approx(W - 1.5 - x)
    # (c) the diagonal's corners, then a checkerboard
    ii, jj = np.meshgrid(np.arange(16), np.arange(16))
    stair = (jj == ii + 1).astype(np.uint8)
    up, down = math.pi / 4 + 1e-6, math.pi / 4 - 1e-6
    q = np.array([[5.0, 5.0, up], [5.0, 5.0, down]])
    assert np.allclose(oracle.cast_exact(stair, q, mr, 1), [0.5 / math.sin(up), mr], atol=1e-9)
    assert np.allclose(oracle.cast_exact(stair, q, mr, 0), [math.sin(up), mr], atol=1e-9)
    cb = ((ii + jj) % 2).astype(np.uint8)
    c45 = math.cos(math.pi / 4)
    i0, j0 = 6, 8  # i + j even: free
    q = np.array([[i0 + 0.1, j0 - 0.2, math.pi / 4]])
    assert oracle.cast_exact(cb, q, mr, 1)[0] == pytest.approx(0.4 / c45, abs=1e-9)
    assert oracle.cast_exact(cb, q, mr, 0)[0] == pytest.approx(1.1 * c45, abs=1e-9)
    # (d) sloped ray to a vertical wall
    wall = np.zeros((40, 40), np.uint8)
    wall[:, 20] = 1
    for (x0, y0, th) in ((2.3, 4.6, math.atan2(1, 3)), (5.7, 30.2, -0.4), (11.0, 19.5, 0.05)):
        t1 = (19.5 - x0) / math.cos(th)
        row = math.floor(y0 + t1 * math.sin(th) + 0.5)
        t0 = (20 - x0) * math.cos(th) + (row - y0) * math.sin(th)
        q = np.array([[x0, y0, th]])
        assert oracle.cast_exact(wall, q, mr, 1)[0] == pytest.approx(t1, abs=1e-9), (x0, y0, th)
        assert oracle.cast_exact(wall, q, mr, 0)[0] == pytest.approx(t0, abs=1e-9), (x0, y0, th)


def test_against_exact_caster(oracle):
    """The CDDT is an approximation (Section II, III).  At a discrete direction
    a cell counts as hit when its rotated square meets the query's bin, a
    superset of the cells the exact ray crosses, so (a) no ray leaks: the CDDT
    range never exceeds the exact cast to the first crossed cell's centre by
    more than half a cell (the centre-ordering slack), and (b) no hit is
    invented: the reported collision point lies within 1 + h of the centre of
    an occupied cell, h = (|cos| + |sin|)/2 the half-extent of a rotated cell."""
    g = synth.rect_map(128, 128, n_rects=25, seed=61)
    H, W = g.shape
    N, mr = 108, 500.0
    d = oracle.OracleCDDT(g, N, mr)
    parts = synth.uniform_particles(g, 5000, seed=62)
    ks = synth.Stream(63).integers(parts.shape[0], 0, N - 1)
    th = np.array([np.float32(2 * math.pi * k / N) for k in ks], np.float32)
    q = parts.copy()
    q[:, 2] = th
    r = d.calc_range(q).astype(np.float64)
    ang = 2 * math.pi * ks / N
    ex = oracle.cast_exact(g, np.stack([q[:, 0], q[:, 1], ang], 1), mr, 0)
    assert np.all(r <= ex + 0.5 + 1e-4)
    assert np.mean(np.abs(r - ex) < 1e-3) > 0.3
    occ = np.argwhere(g)  # (row, col)
    h = 0.5 * (np.abs(np.cos(ang)) + np.abs(np.sin(ang)))
    hit = r < mr
    assert hit.mean() > 0.99
    px = q[:, 0] + r * np.cos(ang)
    py = q[:, 1] + r * np.sin(ang)
    for t in np.flatnonzero(hit):
        dd = np.min(np.hypot(occ[:, 1] - px[t], occ[:, 0] - py[t]))
        assert dd < 1.0 + h[t] + 1e-3, (t, dd)


# ------------------------------------------------------------------ 16-bit

def test_u16_quantisation(oracle):
    """Reading S7: 16-bit zero points change a range by at most 1/(2Q) when the
    same obstacle is hit; Q is the largest power of two with
    (diag + 4) Q <= 65535."""
    g = synth.rect_map(256, 256, n_rects=40, seed=71)
    d32 = oracle.OracleCDDT(g, 108, 300.0)
    d16 = oracle.OracleCDDT(g, 108, 300.0, u16=True)
    diag = math.hypot(256, 256)
    Q = d16.params.Q
    assert Q == 2 ** math.floor(math.log2(65535 / (diag + 4)))
    assert (diag + 4) * Q <= 65535 < (diag + 4) * 2 * Q
    q = synth.uniform_particles(g, 20000, seed=72)
    r32, kb32, zi32, _, _ = d32.calc_range_info(q)
    r16, kb16, zi16, _, _ = d16.calc_range_info(q)
    same = (zi32 == zi16) & (kb32 == kb16) & (zi32 >= 0) & (r32 < 300.0)
    assert same.mean() > 0.95
    assert np.max(np.abs(r32[same] - r16[same])) <= 0.5 / Q + 1e-4
    assert d16.total_zp == d32.total_zp


# ------------------------------------------------------------------ prune

def test_prune_changes_no_answer(oracle):
    """Section IV-C pruning (reading S8) removes zero points without changing
    the answer of any query from a free cell: every grid state and random
    continuous free-space queries."""
    for seed, (W, H, N) in [(81, (40, 30, 16)), (82, (64, 64, 36))]:
        g = synth.rect_map(W, H, n_rects=10, seed=seed)
        full = oracle.OracleCDDT(g, N, 200.0)
        pr = oracle.OracleCDDT(g, N, 200.0)
        removed = pr.prune()
        assert removed > 0
        assert pr.total_zp == full.total_zp - removed
        q = np.concatenate([_grid_states(W, H, N), _random_queries(W, H, 100000, seed + 1)])
        np.testing.assert_array_equal(pr.calc_range(q), full.calc_range(q))
        assert pr.prune() == -1


def test_prune_interior_of_straight_wall(oracle):
    """Section IV-C's example: in the theta = 0 slice the middle cells of a
    line of obstacles along x are never hit, only its two ends."""
    g = np.zeros((11, 21), np.uint8)
    g[5, 3:18] = 1
    d = oracle.OracleCDDT(g, 8, 100.0)
    bs0, zp0 = d.export()
    b = 5 + int(d.params.T[0])  # row 5 of slice 0
    assert bs0[b + 1] - bs0[b] == 15
    d.prune()
    bs, zp = d.export()
    np.testing.assert_array_equal(zp[bs[b]:bs[b + 1]], np.array([3.0, 17.0], np.float32))


def test_prune_single_bin_agrees(oracle):
    """The per-bin form of the pruning rule (all free cells scanned for one
    bin) agrees with the whole-map pass."""
    g = synth.rect_map(48, 40, n_rects=9, seed=91)
    d = oracle.OracleCDDT(g, 20, 100.0)
    bs, zp = d.export()
    eps = oracle.prune_eps(48, 40)
    keep_ref = []
    sb = d.params.sbase
    rs = synth.Stream(92)
    picks = rs.integers(40, 0, d.params.total_bins - 1)
    for gb in picks:
        sl = int(np.searchsorted(sb, gb, side="right") - 1)
        b = int(gb - sb[sl])
        keep_ref.append((gb, d.params.prune_bin(g, sl, b, zp[bs[gb]:bs[gb + 1]], eps)))
    d.prune(eps)
    bs2, zp2 = d.export()
    for gb, keep in keep_ref:
        np.testing.assert_array_equal(zp2[bs2[gb]:bs2[gb + 1]], zp[bs[gb]:bs[gb + 1]][keep])


# ------------------------------------------------------------------ update

@pytest.mark.parametrize("u16", [False, True])
def test_update_equals_rebuild(oracle, u16):
    """Section IV-D: after any sequence of cell writes the incrementally updated
    CDDT holds exactly the zero points of a CDDT built from the final map,
    including obstacles revealed or hidden by the erosion."""
    g = synth.rect_map(48, 36, n_rects=10, seed=101)
    d = oracle.OracleCDDT(g, 24, 100.0, u16=u16)
    rs = synth.Stream(102)
    cur = g.copy()
    for step in range(4):
        n = 60
        xy = np.stack([rs.integers(n, 0, 47), rs.integers(n, 0, 35)], 1).astype(np.int32)
        occ = (rs.uniform(n) < 0.5).astype(np.uint8)
        # a block write and clear exercises neighbour reveal
        if step == 1:
            blk = np.array([(x, y) for y in range(10, 15) for x in range(20, 26)], np.int32)
            xy = np.concatenate([xy, blk])
            occ = np.concatenate([occ, np.ones(len(blk), np.uint8)])
        if step == 2:
            blk = np.array([(x, y) for y in range(11, 14) for x in range(21, 25)], np.int32)
            xy = np.concatenate([xy, blk])
            occ = np.concatenate([occ, np.zeros(len(blk), np.uint8)])
        assert d.update(xy, occ) == 0
        for (x, y), o in zip(xy, occ):
            cur[y, x] = o
        ref = oracle.OracleCDDT(cur, 24, 100.0, u16=u16)
        bs, zp = d.export()
        bs_r, zp_r = ref.export()
        np.testing.assert_array_equal(bs, bs_r)
        np.testing.assert_array_equal(zp, zp_r)
        gg, ee = d.grid_edge()
        np.testing.assert_array_equal(gg, cur)
        np.testing.assert_array_equal(ee, oracle.edge_map(cur))
    d.prune()
    assert d.update(np.zeros((1, 2), np.int32), np.ones(1, np.uint8)) == -1


# ------------------------------------------------------------------ beam model

def _model(oracle, mr=300.0, **kw):
    base = dict(z_hit=0.0, z_short=0.0, z_max=0.0, z_rand=0.0, sigma_hit=8.0,
                lambda_short=0.01, hit_truncnorm=0)
    base.update(kw)
    return oracle.beam_model(mr, **base)


def test_beam_model_components(oracle):
    """Beam model (Probabilistic Robotics): p_hit is the normal density
    N(z; z*, sigma^2) (scipy), its truncated form integrates to 1 on
    [0, z_max], p_short integrates to 1 on [0, z*], p_rand to 1 on
    [0, z_max), p_max is a point mass at z_max, and the mixture is the
    weighted sum with the weights unnormalised (they sum to 0.95)."""
    from scipy import integrate, stats
    mr = 300.0
    zs_list = [0.0, 0.5, 3.0, 40.0, 150.0, 299.0]
    z = np.linspace(0, mr, 30001)
    for zs in zs_list:
        p, _ = oracle.beam_eval(_model(oracle, z_hit=1.0), z, np.full_like(z, zs))
        np.testing.assert_allclose(p, stats.norm.pdf(z, loc=zs, scale=8.0), rtol=1e-12, atol=1e-300)
        p, _ = oracle.beam_eval(_model(oracle, z_hit=1.0, hit_truncnorm=1), z, np.full_like(z, zs))
        assert abs(integrate.trapezoid(p, z) - 1.0) < 1e-6
        if zs > 0:
            zz = np.linspace(0, zs, 20001)
            p, _ = oracle.beam_eval(_model(oracle, z_short=1.0), zz, np.full_like(zz, zs))
            assert abs(integrate.trapezoid(p, zz) - 1.0) < 1e-6
            p, _ = oracle.beam_eval(_model(oracle, z_short=1.0), np.array([zs + 0.1]), np.array([zs]))
            assert p[0] == 0.0
    p, _ = oracle.beam_eval(_model(oracle, z_rand=1.0), z[:-1], np.full(z.size - 1, 10.0))
    assert abs(integrate.trapezoid(p, z[:-1]) - 1.0) < 1e-3
    p, _ = oracle.beam_eval(_model(oracle, z_max=1.0), np.array([mr, mr + 5, mr - 1e-3, 0.0]), np.full(4, 10.0))
    np.testing.assert_array_equal(p, [1.0, 1.0, 0.0, 0.0])
    # the mixture is linear in the weights
    full = oracle.beam_model(mr)
    zz = np.linspace(0, mr, 777)
    zs = np.full_like(zz, 37.0)
    parts = [oracle.beam_eval(_model(oracle, **{k: 1.0}), zz, zs)[0]
             for k in ("z_hit", "z_short", "z_max", "z_rand")]
    want = 0.75 * parts[0] + 0.01 * parts[1] + 0.07 * parts[2] + 0.12 * parts[3]
    np.testing.assert_allclose(oracle.beam_eval(full, zz, zs)[0], want, rtol=1e-6)
    assert abs((0.75 + 0.01 + 0.07 + 0.12) - 0.95) < 1e-12


@pytest.mark.parametrize("trunc", [0, 1])
def test_beam_model_derivative(oracle, trunc):
    """The analytic dp/dz* equals a central difference of p in z*."""
    m = oracle.beam_model(300.0, hit_truncnorm=trunc)
    rs = synth.Stream(111)
    zs = rs.uniform(4000, 0.5, 299.0)
    z = rs.uniform(4000, 0.0, 300.0)
    keep = np.abs(z - zs) > 1e-2
    zs, z = zs[keep], z[keep]
    h = 1e-5
    p1, _ = oracle.beam_eval(m, z, zs + h)
    p0, _ = oracle.beam_eval(m, z, zs - h)
    _, dp = oracle.beam_eval(m, z, zs)
    fd = (p1 - p0) / (2 * h)
    np.testing.assert_allclose(dp, fd, rtol=1e-5, atol=1e-12)


def test_logw_is_sum_of_log_beams(oracle):
    """log w of a particle is the sum over its beams of log p(z_i | z*_i)."""
    g = synth.rect_map(96, 96, n_rects=15, seed=121)
    d = oracle.OracleCDDT(g, 108, 300.0)
    bo = synth.beam_offsets(61)
    parts = synth.uniform_particles(g, 50, seed=122)
    obs = np.clip(synth.Stream(123).uniform(61, 0.0, 320.0), 0, 300).astype(np.float32)
    m = oracle.beam_model(300.0)
    logw, ranges = d.sensor_weights(parts, bo, obs, m, want_ranges=True)
    for p in range(parts.shape[0]):
        pv, _ = oracle.beam_eval(m, obs.astype(np.float64), ranges[p].astype(np.float64))
        assert abs(np.sum(np.log(pv)) - logw[p]) < 1e-9 * max(1.0, abs(logw[p]))
        q = np.stack([np.full(61, parts[p, 0]), np.full(61, parts[p, 1]),
                      (parts[p, 2] + bo).astype(np.float32)], 1)
        np.testing.assert_array_equal(d.calc_range(q), ranges[p])


# ------------------------------------------------------------------ gradient

def test_gradient_matches_finite_differences(oracle):
    """d log w / d(x, y): the analytic float64 gradient equals a central finite
    difference (delta = 1e-3 cell) of the float64 piecewise-linear log-weight,
    within 1e-3 relative.  Per particle, a sample counts when no discrete
    choice (cell, slice, bin, zero point, clamp, short-range indicator)
    changes inside the stencil and no expected range lies in (0, 0.1) cell,
    where the short-range density ~ 1/z* curves too fast for delta = 1e-3;
    per beam, additionally when the beam's query point lies at least 0.25 cell
    from a bin edge."""
    g = synth.rect_map(128, 128, n_rects=20, seed=131)
    N, mr = 108, 300.0
    d = oracle.OracleCDDT(g, N, mr)
    bo = synth.beam_offsets(61)
    m = oracle.beam_model(mr)
    gt = synth.uniform_particles(g, 1, seed=132)[0]
    q = np.stack([np.full(61, gt[0]), np.full(61, gt[1]), (gt[2] + bo).astype(np.float32)], 1)
    obs = np.clip(d.calc_range(q) + synth.noise(61, 2.0, seed=133), 0, mr).astype(np.float32)
    parts = synth.tracking_particles(gt.astype(np.float64), 300, seed=134)
    grad_main, _ = d.sensor_grad(parts, bo, obs, m)
    delta = 1e-3
    p = d.params

    def fd_check(x, y, th, bo_, obs_):
        qq = np.stack([np.full(bo_.size, x), np.full(bo_.size, y), (np.float32(th) + bo_)], 1)
        zs = d.calc_range(qq)
        if np.any((zs > 0) & (zs < 0.1)):
            return None
        v0, s0, g0 = d.logw_piecewise(x, y, th, bo_, obs_, m)
        vals = []
        for dx, dy in ((delta, 0), (-delta, 0), (0, delta), (0, -delta)):
            v, s_, _ = d.logw_piecewise(x + dx, y + dy, th, bo_, obs_, m)
            if s_ != s0:
                return None
            vals.append(v)
        fd = np.array([(vals[0] - vals[1]) / (2 * delta), (vals[2] - vals[3]) / (2 * delta)])
        return fd, g0

    n_part = n_beam = nonzero = 0
    for t in range(parts.shape[0]):
        x, y, th = float(parts[t, 0]), float(parts[t, 1]), parts[t, 2]
        r = fd_check(x, y, th, bo, obs)
        if r is not None:
            fd, g0 = r
            scale = max(np.linalg.norm(g0), 1e-9)
            assert np.linalg.norm(fd - g0) <= 1e-3 * scale + 1e-9, (t, fd, g0)
            # the oracle's gradient on float32 ranges agrees with it
            assert np.linalg.norm(grad_main[t] - g0) <= 1e-3 * scale + 1e-9
            n_part += 1
            nonzero += np.linalg.norm(g0) > 0
        ths = (np.float32(th) + bo).astype(np.float32)
        ks = np.array([p.query_k(a) for a in ths]) % (N // 2)
        yr = np.float32(y) * p.c[ks] - np.float32(x) * p.s[ks]
        for i in np.flatnonzero(np.abs((yr % 1.0) - 0.5) >= 0.25)[:6]:
            r = fd_check(x, y, th, bo[i:i + 1], obs[i:i + 1])
            if r is None:
                continue
            fd, g0 = r
            scale = max(np.linalg.norm(g0), 1e-9)
            assert np.linalg.norm(fd - g0) <= 1e-3 * scale + 1e-9, (t, i, fd, g0)
            n_beam += 1
    assert n_part > 100 and nonzero > 50 and n_beam > 500


def test_sorted_search_sectors_pins():
    """The sector count of a sorted-CSR binary search on hand-checked sizes:
    an empty bin touches only its offsets; up to 8 keys fit one sector; 9 to
    16 keys take one halving, 17 to 32 two."""
    from oracle import oracle as O
    got = O.sorted_search_sectors([0, 1, 8, 9, 16, 17, 32, 33, 1000], 8)
    assert list(got) == [1, 2, 2, 3, 3, 4, 4, 5, 9]
    assert list(O.sorted_search_sectors([16, 17], 16)) == [2, 3]


def test_motion_model_pins():
    """The motion model on closed forms: no motion is the identity; a step
    forward along theta = 0 moves +x, sideways (dy) moves +y; a turn past
    2 pi wraps by one turn; noise adds to the odometry."""
    from oracle import oracle as O
    p = np.array([[10.0, 20.0, 0.0], [5.0, 5.0, 1.0], [7.0, 3.0, 6.2]], np.float32)
    seg = np.array([0, 3])
    z = np.zeros((3, 3), np.float32)
    assert np.array_equal(O.motion(p, seg, np.zeros((1, 3), np.float32), z), p)
    out = O.motion(p[:1], [0, 1], np.array([[1.0, 0.0, 0.0]], np.float32), z[:1])
    assert np.allclose(out, [[11.0, 20.0, 0.0]])
    out = O.motion(p[:1], [0, 1], np.array([[0.0, 2.0, 0.0]], np.float32), z[:1])
    assert np.allclose(out, [[10.0, 22.0, 0.0]])
    out = O.motion(p[2:], [0, 1], np.array([[0.0, 0.0, 0.2]], np.float32), z[:1])
    assert np.isclose(out[0, 2], np.float32(6.2) + np.float32(0.2) - 2 * np.pi, atol=1e-6)
    nz = np.array([[0.5, -0.25, 0.1]], np.float32)
    a = O.motion(p[1:2], [0, 1], np.array([[1.0, 1.0, 0.3]], np.float32), nz)
    b = O.motion(p[1:2], [0, 1], np.array([[1.5, 0.75, 0.4]], np.float32), z[:1])
    assert np.allclose(a, b, atol=1e-6)
    th = np.float64(np.float32(1.0))
    assert np.isclose(a[0, 0], 5.0 + 1.5 * np.cos(th) - 0.75 * np.sin(th), atol=1e-5)
    # a turn below 0 wraps up by one turn
    out = O.motion(np.array([[1.0, 1.0, 0.1]], np.float32), [0, 1], np.array([[0.0, 0.0, -0.3]], np.float32), z[:1])
    assert np.isclose(out[0, 2], np.float32(0.1) - np.float32(0.3) + 2 * np.pi, atol=1e-6)
    # each filter segment (one of them empty) moves by its own odometry
    q = np.array([[0.0, 0.0, 0.0]] * 5, np.float32)
    out = O.motion(q, [0, 2, 2, 5], np.array([[1.0, 0, 0], [9.0, 0, 0], [3.0, 0, 0]], np.float32),
                   np.zeros((5, 3), np.float32))
    assert list(out[:, 0]) == [1.0, 1.0, 3.0, 3.0, 3.0]


def test_resampling_of_undefined_weights():
    """Reading R1 where exp(logw - max) is undefined: a filter whose every
    log-weight is -inf (or NaN) has no weighted particle, so all weigh the
    same and systematic resampling keeps each once, in order; a NaN among
    finite log-weights is never drawn; +inf log-weights share every draw."""
    from oracle import oracle as O
    n = 40
    for lw in (np.full(n, -np.inf, np.float32), np.full(n, np.nan, np.float32)):
        idx, _ = O.resample_indices(lw, [0, n], np.array([0.6], np.float32))
        assert np.array_equal(idx, np.arange(n))
    lw = np.random.default_rng(7).normal(-30.0, 2.0, n).astype(np.float32)
    lw[::3] = np.nan
    idx, _ = O.resample_indices(lw, [0, n], np.array([0.2], np.float32))
    assert not np.isnan(lw[idx]).any()
    lw = np.full(n, -10.0, np.float32)
    lw[[5, 21]] = np.inf
    idx, _ = O.resample_indices(lw, [0, n], np.array([0.3], np.float32))
    assert set(idx.tolist()) == {5, 21} and (idx == 5).sum() == n // 2


def test_resampling_pins():
    """Systematic resampling: equal weights keep every particle once in
    order; one finite weight takes every draw; for any weights each particle
    is drawn floor or ceil of n times its normalised weight, in index order."""
    from oracle import oracle as O
    n = 50
    idx, _ = O.resample_indices(np.full(n, -3.0, np.float32), [0, n], np.array([0.37], np.float32))
    assert np.array_equal(idx, np.arange(n))
    # offset 0 and n a power of two: every target (m / n of the total) equals
    # a running sum exactly, and the first sum above it is particle m's own
    idx, _ = O.resample_indices(np.full(64, -3.0, np.float32), [0, 64], np.array([0.0], np.float32))
    assert np.array_equal(idx, np.arange(64))
    lw = np.full(n, -np.inf, np.float32)
    lw[17] = -5.0
    idx, _ = O.resample_indices(lw, [0, n], np.array([0.9], np.float32))
    assert (idx == 17).all()
    rs = np.random.default_rng(5)
    lw = rs.normal(-40.0, 3.0, 400).astype(np.float32)
    seg = np.array([0, 150, 150, 400])
    u = np.array([0.1, 0.5, 0.99], np.float32)
    idx, _ = O.resample_indices(lw, seg, u)
    for f in (0, 2):
        a, b = seg[f], seg[f + 1]
        k = idx[a:b]
        assert (np.diff(k) >= 0).all()
        w = np.exp(lw[a:b].astype(np.float64) - lw[a:b].max())
        expect = (b - a) * w / w.sum()
        cnt = np.bincount(k, minlength=b - a)
        assert (np.abs(cnt - expect) < 1.0 + 1e-9).all()
    # only relative weights matter: a common shift of every log-weight, even
    # one far beyond exp's range, draws the same particles
    idx2, _ = O.resample_indices(lw + np.float32(1000.0), seg, u)
    assert np.array_equal(idx2, idx)


def test_lookup_table_pins(oracle):
    """The 16-bit table: its scale is the largest power of two that fits
    max_range in 16 bits; entries code the O4 ranges exactly up to half a
    step; a lookup at a cell centre in a table direction returns that
    entry, and snaps any pose inside the cell to it."""
    from oracle import oracle as O
    assert O.lut_scale(1000.0) == 64.0 and O.lut_scale(300.0) == 128.0 and O.lut_scale(65535.0) == 1.0
    g = synth.rect_map(48, 40, n_rects=5, seed=9)
    N, mr = 24, 80.0
    d = oracle.OracleCDDT(g, N, mr)
    tab = O.lut_table(d.params, g, mr)
    ref = d.params.lut(g)
    sc = O.lut_scale(mr)
    assert np.all(np.abs(tab / sc - ref) <= 0.5 / sc + 1e-6)
    k, j, i = 5, 17, 23
    th = np.float32(2.0 * np.pi * k / N)
    poses = np.array([[i, j, th], [i + 0.3, j - 0.45, th], [-3.0, 2.0, th]], np.float32)
    got = O.lut_lookup(d.params, tab, mr, poses)
    assert got[0] == np.float32(tab[k, j, i]) / np.float32(sc) == got[1]
    assert got[2] == 0.0
    # any pose inside a cell reads its state: the O1 brute-force cast from
    # the cell centre in direction theta_k, coded
    rs = synth.Stream(19)
    m = 300
    ii, jj, kk = rs.integers(m, 0, 47), rs.integers(m, 0, 39), rs.integers(m, 0, N - 1)
    ths = np.array([np.float32(2.0 * np.pi * t / N) for t in kk], np.float32)
    centre = np.stack([ii, jj, ths], 1).astype(np.float32)
    jit = (rs.uniform(2 * m, -0.45, 0.45).reshape(m, 2)).astype(np.float32)
    q = centre.copy()
    q[:, :2] += jit
    want = np.clip(np.floor(d.params.calc_range_brute(g, centre) * np.float32(sc) + np.float32(0.5)), 0, 65535)
    got = O.lut_lookup(d.params, tab, mr, q)
    assert np.array_equal(got, (want / np.float32(sc)).astype(np.float32))


# ------------------------------------------------------------------ baselines

def test_direction_rule_pins():
    """The baseline casters' float32 cos / sin of a heading (reading D1) lie
    within 2 ulp and 1.2e-7 of the exact values (float64 library sin and cos
    of the same float heading; beyond 2^16 rad, of its exact remainder by the
    float 2 pi), and the axis headings give the exact values' float
    roundings."""
    from oracle import oracle as O
    rs = synth.Stream(93)
    for lo, hi in ((-7.0, 14.0), (-65536.0, 65536.0)):
        th = rs.uniform(40000, lo, hi).astype(np.float32)
        s, c = O.dir_sincos(th)
        for got, want in ((s, np.sin(th.astype(np.float64))), (c, np.cos(th.astype(np.float64)))):
            err = np.abs(got.astype(np.float64) - want)
            assert err.max() < 1.2e-7
            assert np.all(err <= 2 * np.spacing(np.abs(want).astype(np.float32)))
    th = np.concatenate([np.array([1e5, -2.5e6, 1e7, 3e38], np.float32),
                         rs.uniform(40, 7e4, 1e8).astype(np.float32)])
    s, c = O.dir_sincos(th)
    red = np.fmod(th.astype(np.float64), np.float64(np.float32(2 * np.pi)))
    assert np.abs(s - np.sin(red)).max() < 1.2e-7 and np.abs(c - np.cos(red)).max() < 1.2e-7
    axes = np.array([0.0, np.pi / 2, np.pi, -np.pi / 2, 2 * np.pi], np.float32)
    s, c = O.dir_sincos(axes)
    assert np.array_equal(s, np.sin(axes.astype(np.float64)).astype(np.float32))
    assert np.array_equal(c, np.cos(axes.astype(np.float64)).astype(np.float32))


def _box(W, H):
    g = np.zeros((H, W), np.uint8)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 1
    return g


def test_bresenham_closed_forms(oracle):
    """The Bresenham caster (Section II) walks the textbook digital line: in
    a shallow octant the cell of column x is the nearest integer to the ideal
    line's y there.  One occupied cell on that line is hit at its centre's
    distance; the same cell one row off the line is never met (the walk
    leaves the map).  Axis rays in a box end at the wall cell's centre;
    degenerate queries return 0."""
    from oracle import oracle as O
    rs = synth.Stream(91)
    W, H = 80, 60
    checked = 0
    for trial in range(200):
        x0, y0 = int(rs.integers(1, 2, 20)[0]), int(rs.integers(1, 2, 20)[0])
        dx, dy = int(rs.integers(1, 20, 55)[0]), int(rs.integers(1, 0, 30)[0])
        if dy > dx:
            continue
        sx = int(rs.integers(1, 0, 1)[0]) * 2 - 1  # mirror in x about the start
        xs0 = x0 if sx > 0 else W - 1 - x0
        th = math.atan2(dy, sx * dx)
        R = math.hypot(dx, dy)
        # end cell = (xs0 + sx dx, y0 + dy) exactly when R (cos, sin) lands there
        if round(xs0 + R * math.cos(th)) != xs0 + sx * dx or round(y0 + R * math.sin(th)) != y0 + dy:
            continue
        k = int(rs.integers(1, 1, dx)[0])
        num = k * dy  # y offset of column k is num / dx
        if 2 * (num % dx) == dx:
            continue  # a tie: either neighbour is a valid digital line
        yk = y0 + (num + dx // 2) // dx
        cell = (xs0 + sx * k, yk)
        pose = np.array([[xs0, y0, th]], np.float64)
        g = np.zeros((H, W), np.uint8)
        g[cell[1], cell[0]] = 1
        r = O.cast_bresenham(g, pose, R)[0]
        assert r == np.float32(math.hypot(cell[0] - xs0, cell[1] - y0)), (trial, cell)
        g[:] = 0
        g[cell[1] + 1, cell[0]] = 1
        assert O.cast_bresenham(g, pose, R)[0] == np.float32(R)
        checked += 1
    assert checked > 40
    g = _box(12, 9)
    poses = np.array([[2, 4, 0.0], [5, 2, math.pi / 2], [7, 3, math.pi], [4, 6, -math.pi / 2],
                      [0, 4, 0.0], [-3, 4, 0.0], [3, 3, float("nan")]], np.float64)
    r = O.cast_bresenham(g, poses, 100.0)
    assert list(r) == [9.0, 6.0, 7.0, 6.0, 0.0, 0.0, 0.0]
    # the start cell is the nearest cell centre: (0.6, 4.2) starts in the free
    # cell (1, 4), not the wall cell (0, 4), and meets the wall at (11, 4)
    r = O.cast_bresenham(g, np.array([[0.6, 4.2, 0.0]], np.float32), 100.0)[0]
    dx, dy = np.float32(11) - np.float32(0.6), np.float32(4) - np.float32(4.2)
    assert r == np.sqrt(dx * dx + dy * dy)
    # a tie of the error term, traced by hand through the textbook all-octant
    # stepping (err = dx - |dy|; step x when 2 err >= -|dy|, y when 2 err <=
    # dx): (5, 5) -> (9, 7) visits (6, 6), (7, 6), (8, 7), (9, 7)
    R = math.hypot(4, 2)
    pose = np.array([[5, 5, math.atan2(2, 4)]], np.float32)
    for cell, want in (((6, 6), math.sqrt(2)), ((7, 6), math.sqrt(5)), ((8, 7), math.sqrt(13))):
        g = np.zeros((12, 12), np.uint8)
        g[cell[1], cell[0]] = 1
        assert O.cast_bresenham(g, pose, R)[0] == np.float32(want), cell
    for cell in ((6, 5), (7, 7)):
        g = np.zeros((12, 12), np.uint8)
        g[cell[1], cell[0]] = 1
        assert O.cast_bresenham(g, pose, R)[0] == np.float32(R), cell


def _edt_brute(g):
    occ = np.argwhere(g != 0)  # (row, col)
    H, W = g.shape
    if occ.size == 0:
        return np.full((H, W), np.float32(W + H), np.float32)
    jj, ii = np.mgrid[0:H, 0:W]
    d2 = ((jj.reshape(-1, 1) - occ[None, :, 0]) ** 2 + (ii.reshape(-1, 1) - occ[None, :, 1]) ** 2).min(1)
    return np.sqrt(d2.astype(np.float64)).astype(np.float32).reshape(H, W)


def test_distance_transform_pins():
    """The ray marcher's Euclidean distance transform (Section II) equals the
    definition -- the least centre-to-centre distance to an occupied cell --
    computed by brute force, on tiny maps of every density, a free map and a
    fully occupied one."""
    from oracle import oracle as O
    maps = _tiny_maps(8, seed=23) + [np.zeros((7, 13), np.uint8), np.ones((5, 4), np.uint8), _box(12, 9)]
    rs = synth.Stream(24)
    for dens in (0.01, 0.2, 0.7):
        maps.append((rs.uniform(37 * 29) < dens).astype(np.uint8).reshape(29, 37))
    for g in maps:
        assert np.array_equal(O.edt(g), _edt_brute(g)), g.shape


def test_raymarch_closed_forms():
    """Ray marching (Section II) steps by the distance to the nearest
    obstacle.  In a box an axis ray's steps stay on cell centres and end
    exactly on the wall cell (the hand-traced case from (2, 4) along +x in a
    12 x 9 box reads distances 2, 4, 3, 0: range 9, 4 reads).  With a single
    occupied cell at (x0 + 3k, y0 + 4k) the first distance is 5k and the ray
    at atan2(4, 3) lands on it: range 5k, 2 reads (the ray at atan2(3, 4)
    misses it).  Degenerate queries give 0; leaving the map or reaching
    max_range gives max_range."""
    from oracle import oracle as O
    g = _box(12, 9)
    E = O.edt(g)
    r, s = O.raymarch(E, np.array([[2, 4, 0.0]], np.float32), 100.0)
    assert r[0] == 9.0 and s[0] == 4
    poses = np.array([[5, 2, np.pi / 2], [7, 3, np.pi], [4, 6, -np.pi / 2], [1, 1, 0.0]], np.float32)
    r, _ = O.raymarch(E, poses, 100.0)
    assert list(r) == [6.0, 7.0, 6.0, 10.0]
    for k in (1, 3, 7):
        g = np.zeros((60, 50), np.uint8)
        x0, y0 = 4, 5
        g[y0 + 4 * k, x0 + 3 * k] = 1
        E = O.edt(g)
        r, s = O.raymarch(E, np.array([[x0, y0, math.atan2(4, 3)]], np.float32), 500.0)
        assert r[0] == np.float32(5 * k) and s[0] == 2, (k, r, s)
        r, _ = O.raymarch(E, np.array([[x0, y0, math.atan2(3, 4)]], np.float32), 500.0)
        assert r[0] == 500.0
    g = _box(12, 9)
    E = O.edt(g)
    poses = np.array([[0, 4, 0.0], [-3, 4, 0.0], [3, 3, np.nan], [np.inf, 3, 0.0], [2, 4, 0.0]], np.float32)
    r, s = O.raymarch(E, poses, 5.0)
    assert list(r) == [0.0, 0.0, 0.0, 0.0, 5.0] and list(s[:4]) == [1, 0, 0, 0]
    E = O.edt(np.zeros((9, 12), np.uint8))
    r, _ = O.raymarch(E, np.array([[2, 4, 0.0]], np.float32), 1000.0)
    assert r[0] == 1000.0


def test_raymarch_against_exact_caster(oracle):
    """A marched ray stops only on a sample inside an occupied cell, so its
    range is never short of the exact cast's entry into the first occupied
    cell on the ray; it matches that entry to within a cell for nearly every
    ray (a ray that grazes a corner can step past it, the method's own
    error)."""
    from oracle import oracle as O
    g = synth.rect_map(128, 128, n_rects=25, seed=61)
    mr = 500.0
    E = O.edt(g)
    q = synth.uniform_queries(g, 4000, seed=64)
    r, s = O.raymarch(E, q, mr)
    ex = oracle.cast_exact(g, q.astype(np.float64), mr, 1)
    assert np.all(r.astype(np.float64) >= ex - 1e-3)
    assert np.mean(r - ex < 1.5) > 0.97
    assert s.min() >= 1
    occ = g != 0
    hit = r < mr
    px = q[hit, 0] + r[hit].astype(np.float64) * np.cos(q[hit, 2].astype(np.float64))
    py = q[hit, 1] + r[hit].astype(np.float64) * np.sin(q[hit, 2].astype(np.float64))
    ok = np.zeros(px.size, bool)
    for ex_ in (-1e-3, 0.0, 1e-3):
        for ey_ in (-1e-3, 0.0, 1e-3):
            ix = np.floor(px + ex_ + 0.5).astype(np.int64).clip(0, g.shape[1] - 1)
            iy = np.floor(py + ey_ + 0.5).astype(np.int64).clip(0, g.shape[0] - 1)
            ok |= occ[iy, ix]
    assert ok.all()


def test_approximation_error_falls_with_theta_disc(oracle):
    """The CDDT approximates the exact cast (Section II: discrete directions,
    cells as rotated squares): on a corridor map its error against the exact
    voxel-traversal caster (same query heading, distance to the first
    crossed cell's centre projection) falls as theta_disc grows, in median
    and at the 90th percentile, and at theta_disc >= 108 under 4 % of the
    rays are off by more than 10 cells (rays grazing a door jamb or corner,
    which the finer direction does not remove).  A report as much as a pin:
    the values are listed with the design notes."""
    g = synth.corridor_map(500, 500, r_min=48)
    mr = 500.0
    q = synth.uniform_queries(g, 20000, seed=71)
    ex = oracle.cast_exact(g, q.astype(np.float64), mr, 0)
    med, p90 = [], []
    for N in (16, 36, 108, 360):
        r = oracle.OracleCDDT(g, N, mr).calc_range(q).astype(np.float64)
        d = np.abs(r - ex)
        med.append(np.median(d))
        p90.append(np.percentile(d, 90))
        if N >= 108:
            assert np.mean(d > 10) < 0.04, N
    assert all(a > b for a, b in zip(med, med[1:])), med
    assert all(a > b for a, b in zip(p90, p90[1:])), p90
    assert med[-1] < 0.25 and p90[-1] < 1.5
