"""Shared seeded cases of the GPU parity tests (maps, particles, scans)."""
import math

import numpy as np

from paper_1705_01167_gb300 import synth


def tiny_maps(n_maps=5, seed=11):
    rs = synth.Stream(seed)
    out = []
    for _ in range(n_maps):
        W = int(rs.integers(1, 3, 40)[0])
        H = int(rs.integers(1, 3, 40)[0])
        dens = rs.uniform(1, 0.05, 0.5)[0]
        out.append((rs.uniform(W * H) < dens).astype(np.uint8).reshape(H, W))
    g = np.zeros((9, 11), np.uint8)
    g[3:6, 4:7] = 1
    out.append(g)
    return out


def grid_states(W, H, N, stride=1):
    th = np.array([np.float32(2.0 * math.pi * k / N) for k in range(N)], np.float32)
    jj, ii, kk = np.meshgrid(np.arange(0, H, stride), np.arange(0, W, stride), np.arange(N), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel(), th[kk.ravel()]], 1).astype(np.float32)


def random_queries(W, H, n, seed):
    rs = synth.Stream(seed)
    x = rs.uniform(n, -1.0, W)
    y = rs.uniform(n, -1.0, H)
    th = rs.uniform(n, -7.0, 14.0)
    return np.stack([x, y, th], 1).astype(np.float32)


def special_queries(W, H):
    """Edge cases: cell boundaries, map border, off-map, non-finite values."""
    nan, inf = float("nan"), float("inf")
    q = [
        [0.0, 0.0, 0.0], [W - 1.0, H - 1.0, 3.0], [-0.5, 0.0, 1.0], [W - 0.5, 0.0, 1.0],
        [0.5, 0.5, 0.5], [W * 0.5, H * 0.5, -1e7], [W * 0.5, H * 0.5, 1e9], [W * 0.5, H * 0.5, 3e38],
        [nan, 1.0, 0.0], [1.0, nan, 0.0], [1.0, 1.0, nan], [inf, 1.0, 0.0], [1.0, 1.0, inf],
        [1.0, 1.0, -inf], [-5.0, 2.0, 0.0], [2.0, H + 3.0, 0.0], [1.5, 1.5, math.pi],
        [1.49999, 2.50001, math.pi / 2],
    ]
    return np.array(q, np.float32)


def observations(oracle_cddt, gt, beam_off, max_range, sigma=2.0, seed=1707):
    q = np.stack([np.full(beam_off.size, gt[0]), np.full(beam_off.size, gt[1]),
                  (np.float32(gt[2]) + beam_off).astype(np.float32)], 1).astype(np.float32)
    r = oracle_cddt.calc_range(q).astype(np.float64)
    return np.clip(r + synth.noise(beam_off.size, sigma, seed=seed), 0, max_range).astype(np.float32)
