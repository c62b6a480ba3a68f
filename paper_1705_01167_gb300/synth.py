"""Seeded synthetic inputs: occupancy grids, particle sets, beam layouts, noise.

This module draws random numbers and lays out maps.  It holds none of the
CDDT arithmetic (no projection, no binning, no search, no beam model), so the
CPU oracle and the CUDA path can both consume its outputs without sharing any
of the method's code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output i
of a stream is the SplitMix64 finaliser applied to ``base + (i + 1) * GAMMA``.
That form vectorises in numpy and gives identical draws on every machine.

Workload shapes follow the paper's experiments: the rectangle map stands in
for the hand-drawn "Synthetic" map and the recursive-division corridor map for
the SLAM "Basement" map (Section VI); the 61-beam, 270-degree scan is the
Hokuyo UST-10LX layout of the particle-filter runs (Section VI).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Default seeds of the synthetic workloads.
SEED_MAP = 1705
SEED_PARTICLES = 1706
SEED_OBS = 1707
SEED_UPDATES = 1708


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (vectorised, wrapping uint64 arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based SplitMix64 stream keyed by an integer seed."""

    def __init__(self, seed: int):
        with np.errstate(over="ignore"):
            s = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
            self._base = _mix64(s + GAMMA)[0]
        self._ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + 1 + n, dtype=np.uint64)
        self._ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self._base + idx * GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """float64 uniform on [lo, hi) from the top 53 bits."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """int64 uniform on the closed range [lo, hi]."""
        span = hi - lo + 1
        return lo + np.floor(self.uniform(n) * span).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """Standard normal draws by the Box-Muller transform."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:n]


# ---------------------------------------------------------------- maps

def rect_map(W: int = 256, H: int = 256, n_rects: int = 40, side_lo: int = 4,
             side_hi: int = 30, seed: int = SEED_MAP) -> np.ndarray:
    """Border walls one cell thick plus ``n_rects`` filled axis-aligned rectangles.

    Sides are drawn independently per axis from U{side_lo..side_hi}; each
    rectangle lies fully inside the border.  Returns uint8 [H, W], 1 = occupied.
    """
    g = np.zeros((H, W), dtype=np.uint8)
    g[0, :] = 1
    g[-1, :] = 1
    g[:, 0] = 1
    g[:, -1] = 1
    rs = Stream(seed)
    for _ in range(n_rects):
        w = int(rs.integers(1, side_lo, side_hi)[0])
        h = int(rs.integers(1, side_lo, side_hi)[0])
        w = min(w, W - 2)
        h = min(h, H - 2)
        x0 = int(rs.integers(1, 1, W - 1 - w)[0])
        y0 = int(rs.integers(1, 1, H - 1 - h)[0])
        g[y0:y0 + h, x0:x0 + w] = 1
    return g


def corridor_map(W: int = 2000, H: int = 2000, seed: int = SEED_MAP, r_min: int = 64,
                 wall_lo: int = 1, wall_hi: int = 3, door_lo: int = 3,
                 door_hi: int = 20) -> np.ndarray:
    """Rooms and corridors by recursive division (a seeded stand-in for a SLAM map).

    A one-cell border encloses the map.  A room whose sides are both below
    ``r_min`` is left alone; otherwise it is split across its longer side by
    a wall ``wall_lo..wall_hi`` cells thick with one door ``door_lo..door_hi``
    cells wide.  Returns uint8 [H, W], 1 = occupied.
    """
    g = np.zeros((H, W), dtype=np.uint8)
    g[0, :] = 1
    g[-1, :] = 1
    g[:, 0] = 1
    g[:, -1] = 1
    rs = Stream(seed)
    stack = [(1, 1, W - 1, H - 1)]  # free interior [x0, x1) x [y0, y1)
    margin = door_hi + 4
    while stack:
        x0, y0, x1, y1 = stack.pop()
        w, h = x1 - x0, y1 - y0
        if w < r_min and h < r_min:
            continue
        split_x = w >= h
        extent = w if split_x else h
        t = int(rs.integers(1, wall_lo, wall_hi)[0])
        if extent < 2 * margin + t:
            continue
        lo0 = x0 if split_x else y0
        pos = int(rs.integers(1, lo0 + margin, lo0 + extent - margin - t)[0])
        span_lo, span_hi = (y0, y1) if split_x else (x0, x1)
        door = int(rs.integers(1, door_lo, door_hi)[0])
        door = min(door, span_hi - span_lo - 1)
        d0 = int(rs.integers(1, span_lo, span_hi - door)[0])
        if split_x:
            g[y0:y1, pos:pos + t] = 1
            g[d0:d0 + door, pos:pos + t] = 0
            stack.append((x0, y0, pos, y1))
            stack.append((pos + t, y0, x1, y1))
        else:
            g[pos:pos + t, x0:x1] = 1
            g[pos:pos + t, d0:d0 + door] = 0
            stack.append((x0, y0, x1, pos))
            stack.append((x0, pos + t, x1, y1))
    return g


def occupancy(grid: np.ndarray) -> float:
    return float(np.count_nonzero(grid)) / grid.size


# ---------------------------------------------------------------- poses

def _free_cells(grid: np.ndarray, n: int, rs: Stream) -> tuple[np.ndarray, np.ndarray]:
    H, W = grid.shape
    xs = np.empty(0, dtype=np.int64)
    ys = np.empty(0, dtype=np.int64)
    while xs.size < n:
        m = max(2 * (n - xs.size), 64)
        cx = rs.integers(m, 0, W - 1)
        cy = rs.integers(m, 0, H - 1)
        ok = grid[cy, cx] == 0
        xs = np.concatenate([xs, cx[ok]])
        ys = np.concatenate([ys, cy[ok]])
    return xs[:n], ys[:n]


def uniform_particles(grid: np.ndarray, P: int, seed: int = SEED_PARTICLES) -> np.ndarray:
    """P poses: a uniform free cell plus U[-1/2, 1/2)^2 jitter, theta ~ U[0, 2pi).

    Returns float32 [P, 3] as (x, y, theta) in cell units; cell (i, j) is
    centred on the integer point (i, j).
    """
    rs = Stream(seed)
    cx, cy = _free_cells(grid, P, rs)
    x = cx + rs.uniform(P, -0.5, 0.5)
    y = cy + rs.uniform(P, -0.5, 0.5)
    th = rs.uniform(P, 0.0, 2.0 * math.pi)
    return np.stack([x, y, th], axis=1).astype(np.float32)


def uniform_queries(grid: np.ndarray, n: int, seed: int = SEED_PARTICLES) -> np.ndarray:
    """n poses with (x, y) uniform over the map area, rejected unless the
    nearest cell is free, and theta ~ U[0, 2pi).  float32 [n, 3]."""
    H, W = grid.shape
    rs = Stream(seed)
    out = np.empty((0, 3), dtype=np.float32)
    while out.shape[0] < n:
        m = max(int(1.3 * (n - out.shape[0])), 64)
        x = rs.uniform(m, -0.5, W - 0.5).astype(np.float32)
        y = rs.uniform(m, -0.5, H - 0.5).astype(np.float32)
        th = rs.uniform(m, 0.0, 2.0 * math.pi).astype(np.float32)
        ix = np.floor(x + np.float32(0.5)).astype(np.int64)
        iy = np.floor(y + np.float32(0.5)).astype(np.int64)
        ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
        ok[ok] = grid[iy[ok], ix[ok]] == 0
        out = np.concatenate([out, np.stack([x[ok], y[ok], th[ok]], axis=1)])
    return np.ascontiguousarray(out[:n])


def random_free_pose(grid: np.ndarray, rs: Stream) -> np.ndarray:
    cx, cy = _free_cells(grid, 1, rs)
    return np.array([float(cx[0]), float(cy[0]), float(rs.uniform(1, 0.0, 2.0 * math.pi)[0])])


def gt_walk(grid: np.ndarray, steps: int, seed: int = SEED_PARTICLES) -> np.ndarray:
    """A ground-truth pose that random-walks one cell per step through free space.

    Each step turns by N(0, 0.3) rad and advances one cell; if the target cell
    is occupied or off the map, a fresh heading is drawn (up to 32 tries).
    Returns float64 [steps, 3].
    """
    H, W = grid.shape
    rs = Stream(seed)
    pose = random_free_pose(grid, rs)
    out = np.empty((steps, 3))
    for t in range(steps):
        out[t] = pose
        th = pose[2] + 0.3 * rs.normal(1)[0]
        for _ in range(32):
            nx = pose[0] + math.cos(th)
            ny = pose[1] + math.sin(th)
            ix, iy = int(math.floor(nx + 0.5)), int(math.floor(ny + 0.5))
            if 0 <= ix < W and 0 <= iy < H and grid[iy, ix] == 0:
                pose = np.array([nx, ny, th % (2.0 * math.pi)])
                break
            th = rs.uniform(1, 0.0, 2.0 * math.pi)[0]
    return out


def tracking_particles(gt: np.ndarray, P: int, sigma_xy: float = 5.0,
                       sigma_th: float = 0.05, seed: int = SEED_PARTICLES) -> np.ndarray:
    """P poses drawn around one ground-truth pose (a converged, tracking filter).

    Returns float32 [P, 3]; theta is wrapped into [0, 2pi).
    """
    rs = Stream(seed)
    x = gt[0] + sigma_xy * rs.normal(P)
    y = gt[1] + sigma_xy * rs.normal(P)
    th = np.mod(gt[2] + sigma_th * rs.normal(P), 2.0 * math.pi)
    return np.stack([x, y, th], axis=1).astype(np.float32)


# ---------------------------------------------------------------- scan layout

def beam_offsets(B: int = 61, fov_deg: float = 270.0) -> np.ndarray:
    """Beam angles relative to the particle heading, evenly over the field of
    view: phi_i = -fov/2 + i * fov / (B - 1), computed in double, stored f32."""
    if B == 1:
        return np.zeros(1, dtype=np.float32)
    i = np.arange(B, dtype=np.float64)
    phi = math.radians(-fov_deg / 2.0) + i * (math.radians(fov_deg) / (B - 1))
    return phi.astype(np.float32)


def pair_offset(B: int = 61, fov_deg: float = 270.0) -> int:
    """Index distance D between beam i and the beam pointing the opposite way
    (phi_{i+D} - phi_i = pi), or 0 when the layout has no such pairs.

    For 61 beams over 270 degrees D = 40, so beams 0..20 pair with 40..60.
    """
    if B < 2 or fov_deg < 180.0:
        return 0
    step = fov_deg / (B - 1)
    d = 180.0 / step
    D = int(round(d))
    if abs(d - D) > 1e-9 or D >= B or 2 * D < B:
        return 0
    return D


def noise(n: int, sigma: float, seed: int = SEED_OBS) -> np.ndarray:
    """Gaussian noise N(0, sigma^2), float64 [n]."""
    return sigma * Stream(seed).normal(n)


def cell_toggles(grid: np.ndarray, n_insert: int, n_remove: int,
                 seed: int = SEED_UPDATES) -> tuple[np.ndarray, np.ndarray]:
    """A batch of cell writes: ``n_insert`` random free cells set occupied and
    ``n_remove`` random occupied cells set free, interleaved at random.

    Returns (xy int32 [n, 2] as (x=column, y=row), occ uint8 [n]).  Cells may
    repeat; writes apply in order.
    """
    H, W = grid.shape
    rs = Stream(seed)
    fx, fy = _free_cells(grid, n_insert, rs)
    occ_idx = np.flatnonzero(grid.reshape(-1))
    if occ_idx.size == 0 or n_remove == 0:
        ox = oy = np.empty(0, dtype=np.int64)
    else:
        pick = occ_idx[rs.integers(n_remove, 0, occ_idx.size - 1)]
        ox, oy = pick % W, pick // W
    xy = np.concatenate([np.stack([fx, fy], 1), np.stack([ox, oy], 1)]).astype(np.int32)
    occ = np.concatenate([np.ones(fx.size, np.uint8), np.zeros(ox.size, np.uint8)])
    perm = np.argsort(rs.uniform(occ.size), kind="stable")
    return np.ascontiguousarray(xy[perm]), np.ascontiguousarray(occ[perm])


def apply_writes(grid: np.ndarray, xy: np.ndarray, occ: np.ndarray) -> np.ndarray:
    """The grid after cell writes applied in order (later writes to a cell
    win); writes outside the map are skipped.  Returns a new array."""
    g = grid.copy()
    H, W = g.shape
    for (x, y), v in zip(np.asarray(xy).tolist(), np.asarray(occ).tolist()):
        if 0 <= x < W and 0 <= y < H:
            g[y, x] = 1 if v else 0
    return g


# ---------------------------------------------------------------- workloads

BEAM_MODEL_DEFAULT = dict(z_hit=0.75, z_short=0.01, z_max=0.07, z_rand=0.12,
                          sigma_hit=8.0, lambda_short=0.01, hit_truncnorm=0)
