"""Seeded synthetic workloads shaped like the paper's experiments.

Each recipe returns host arrays only (maps, poses, scans, noise, cell
writes); it draws random numbers through ``synth`` and holds none of the
CDDT arithmetic.  Observed ranges are made by the caller from the ground
truth pose with whichever caster it trusts (the CPU oracle in tests, the GPU
in the benchmark), plus the recipe's noise.

  rects256       256 x 256 rectangles map (the hand-drawn "Synthetic" map of
                 Section VI), theta_disc 108, 1000 uniform particles x 61 beams
  corridor2000   2000 x 2000 corridor map (the SLAM "Basement" map), theta_disc
                 200, a 200-step tracking filter of 2500 particles x 61 beams,
                 and a 10 M-query uniform sweep
  batched64      64 corridor maps of uneven sizes 512^2 .. 4096^2, theta_disc
                 100 .. 360, one filter of 500 .. 10000 particles each
  diff2000       the 2000 x 2000 map with 4096 x 61 and 1024 x 1081 beams for
                 the adjoint and gradient refinement
  update4000     4000 x 4000 corridor map, theta_disc 360, 100,000 particles x
                 61 beams and 5000 inserts + 5000 removes per step
"""
from __future__ import annotations

import math

import numpy as np

from . import synth


def _scan(B: int):
    return synth.beam_offsets(B), synth.pair_offset(B)


def gt_queries(gt: np.ndarray, beam_off: np.ndarray) -> np.ndarray:
    """Poses (x, y, theta + phi_i) of every beam of every ground-truth pose:
    float32 [len(gt) * B, 3]."""
    gt = np.atleast_2d(gt)
    return np.concatenate([np.stack([np.full(beam_off.size, p[0]), np.full(beam_off.size, p[1]),
                                     (np.float32(p[2]) + beam_off)], 1) for p in gt]).astype(np.float32)


def grid_states(W: int, H: int, stride: int, n_theta: int) -> np.ndarray:
    """The "grid" benchmark's states (Section V): a uniformly spaced grid over
    (x, y, theta), every stride-th cell centre in x and y and n_theta headings
    2 pi k / n_theta; x varies fastest, then y, then theta.  float32 [n, 3]."""
    xs = np.arange(0, W, stride, dtype=np.float64)
    ys = np.arange(0, H, stride, dtype=np.float64)
    ts = 2.0 * np.pi * np.arange(n_theta, dtype=np.float64) / n_theta
    t, y, x = np.meshgrid(ts, ys, xs, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), t.ravel()], axis=1).astype(np.float32)


def rects256():
    g = synth.rect_map(256, 256)
    bo, D = _scan(61)
    rs = synth.Stream(synth.SEED_PARTICLES - 6)
    gt = synth.random_free_pose(g, rs)
    return dict(name="rects256", grid=g, theta_disc=108, max_range=300.0, beam_off=bo, D=D,
                gt=gt[None, :], parts=synth.uniform_particles(g, 1000)[None], noise=synth.noise(61, 2.0)[None])


def corridor2000(steps: int = 200, particles: int = 2500, sweep: int = 10_000_000, seed_offset: int = 0):
    g = synth.corridor_map(2000, 2000)
    gt = synth.gt_walk(g, steps, seed=synth.SEED_PARTICLES + seed_offset)
    parts = np.stack([synth.tracking_particles(gt[t], particles, seed=synth.SEED_PARTICLES + 1000 + t + 100000 * seed_offset)
                      for t in range(steps)]).astype(np.float32)
    bo, D = _scan(61)
    noise = np.stack([synth.noise(61, 2.0, seed=synth.SEED_OBS + t + 100000 * seed_offset) for t in range(steps)])
    sw = synth.uniform_queries(g, sweep, seed=synth.SEED_PARTICLES + 7 + seed_offset) if sweep else None
    return dict(name="corridor2000", grid=g, theta_disc=200, max_range=1000.0, beam_off=bo, D=D, gt=gt,
                parts=parts, noise=noise, sweep=sw)


def batched64(n_maps: int = 64, seed_offset: int = 0):
    """64 independent maps and filters: side uniform over multiples of 64 in
    [512, 4096], theta_disc over multiples of 4 in [100, 360], P over
    [500, 10000]; map m uses seed 1705 + 100 m."""
    rs = synth.Stream(4242 + seed_offset)
    maps = []
    for mi in range(n_maps):
        side = int(rs.integers(1, 512 // 64, 4096 // 64)[0]) * 64
        N = int(rs.integers(1, 100 // 4, 360 // 4)[0]) * 4
        P = int(rs.integers(1, 500, 10000)[0])
        g = synth.corridor_map(side, side, seed=synth.SEED_MAP + 100 * mi)
        mr = float(min(1000.0, side))
        rs2 = synth.Stream(synth.SEED_MAP + 100 * mi + 1 + seed_offset)
        gt = synth.random_free_pose(g, rs2)
        parts = synth.tracking_particles(gt, P, seed=synth.SEED_MAP + 100 * mi + 2 + seed_offset)
        maps.append(dict(grid=g, theta_disc=N, max_range=mr, gt=gt[None, :], parts=parts[None],
                         noise=synth.noise(61, 2.0, seed=synth.SEED_MAP + 100 * mi + 3)[None]))
    bo, D = _scan(61)
    return dict(name="batched64", maps=maps, beam_off=bo, D=D)


def diff2000(seed_offset: int = 0):
    g = synth.corridor_map(2000, 2000)
    gt = synth.gt_walk(g, 1, seed=synth.SEED_PARTICLES + 11 + seed_offset)[0]
    scans = []
    for P, B in ((4096, 61), (1024, 1081)):
        bo, D = _scan(B)
        scans.append(dict(P=P, B=B, beam_off=bo, D=D,
                          parts=synth.tracking_particles(gt, P, seed=synth.SEED_PARTICLES + 12 + B + seed_offset),
                          noise=synth.noise(B, 2.0, seed=synth.SEED_OBS + B)))
    return dict(name="diff2000", grid=g, theta_disc=200, max_range=1000.0, gt=gt[None, :], scans=scans,
                refine_steps=10, eta=0.1)


def update4000(steps: int = 3, particles: int = 100_000, inserts: int = 5000, removes: int = 5000,
               seed_offset: int = 0):
    g = synth.corridor_map(4000, 4000)
    bo, D = _scan(61)
    rs = synth.Stream(synth.SEED_UPDATES + 17 + seed_offset)
    gt = synth.random_free_pose(g, rs)
    parts = synth.uniform_particles(g, particles, seed=synth.SEED_PARTICLES + 21 + seed_offset)
    # each step's writes are drawn on the grid as it stands after the previous step
    cur = g.copy()
    writes = []
    for t in range(steps):
        xy, occ = synth.cell_toggles(cur, inserts, removes, seed=synth.SEED_UPDATES + t + 1000 * seed_offset)
        writes.append((xy, occ))
        cur = synth.apply_writes(cur, xy, occ)
    return dict(name="update4000", grid=g, theta_disc=360, max_range=1000.0, beam_off=bo, D=D,
                gt=gt[None, :], parts=parts, noise=synth.noise(61, 2.0, seed=synth.SEED_OBS + 9)[None],
                writes=writes, final_grid=cur)
