"""Host model of the bin-major prune's cell enumeration (CPU only).

The prune kernel visits, for each bin, the lines of the bin's strip of cells
and a few candidate cells per line, found with float32 arithmetic and a band
margin of 0.25; every candidate then takes the exact per-cell bin test of
reading S8.  Its marks equal the cell-by-cell rule's only if every (cell,
bin) pair that the exact test admits is among the candidates.  This test
evaluates the same float32 steps in NumPy (with and without the fused
multiply-adds the device compiler may form in the candidate arithmetic) and
checks that coverage on maps of several shapes, including single rows and
columns and theta_disc = 4 (a 90-degree slice with cos = 0).
"""
import math

import numpy as np
import pytest

f32 = np.float32


def _slices(W, H, N):
    out, base = [], 0
    cx = [-0.5, W - 0.5, -0.5, W - 0.5]
    cy = [-0.5, -0.5, H - 0.5, H - 0.5]
    for s in range(N // 2):
        ang = 2 * math.pi * s / N
        c, sn = f32(math.cos(ang)), f32(math.sin(ang))
        if s == 0:
            c, sn = f32(1), f32(0)
        if 4 * s == N:
            c, sn = f32(0), f32(1)
        ys = [cy[q] * float(c) - cx[q] * float(sn) for q in range(4)]
        T = int(math.ceil(-min(ys)) + 1)
        out.append((c, sn, T, int(math.ceil(max(ys) + T) + 2)))
        base += out[-1][3]
    return out


def _eps(W, H):
    e = math.ceil(math.log2(2 * math.sqrt(W * W + H * H) + 8))
    return f32(2.0 ** (e - 18))


def _mad(a, b, c, fma):
    """a * b + c in float32, rounded once (fma) or twice."""
    if fma:
        return f32(np.float64(a) * np.float64(b) + np.float64(c))
    return f32(f32(a * b) + c)


def _candidates(W, H, c, sn, T, b, eps, h, fma):
    bp = f32(b - T)
    ylo = f32(f32(f32(f32(bp - f32(0.5)) - h) - eps) - f32(0.25))
    yhi = f32(f32(f32(f32(bp + f32(0.5)) + h) + eps) + f32(0.25))
    cols = abs(c) >= sn
    L = W if cols else H
    k_lo, k_hi = 0.0, float(L - 1)
    if cols:
        if sn > 0:
            hc = f32(f32(H - 1) * c)
            if c > 0:
                k_lo, k_hi = f32(-yhi / sn), f32(f32(hc - ylo) / sn)
            else:
                k_lo, k_hi = f32(f32(hc - yhi) / sn), f32(-ylo / sn)
        elif yhi < 0 or ylo > H - 1:
            return set()
    else:
        ws = f32(f32(W - 1) * sn)
        if c > 0:
            k_lo, k_hi = f32(ylo / c), f32(f32(ws + yhi) / c)
        elif c < 0:
            k_lo, k_hi = f32(f32(ws + yhi) / c), f32(ylo / c)
        elif ylo > 0 or ws + yhi < 0:
            return set()
    l0 = max(0, int(math.floor(max(float(k_lo), -1.0))) - 1)
    l1 = min(L - 1, int(math.ceil(min(float(k_hi), float(L)))) + 1)
    inv = f32(f32(1) / (c if cols else sn))
    out = set()
    for k in range(l0, l1 + 1):
        if cols:
            p = f32(_mad(f32(k), sn, ylo, fma) * inv)
            q = f32(_mad(f32(k), sn, yhi, fma) * inv)
            a0, a1 = max(0, math.ceil(min(p, q))), min(H - 1, math.floor(max(p, q)))
            out.update((k, a) for a in range(a0, a1 + 1))
        else:
            p = f32(_mad(f32(k), c, -yhi, fma) * inv)
            q = f32(_mad(f32(k), c, -ylo, fma) * inv)
            a0, a1 = max(0, math.ceil(p)), min(W - 1, math.floor(q))
            out.update((a, k) for a in range(a0, a1 + 1))
    return out


@pytest.mark.parametrize("W,H,N", [(48, 40, 36), (25, 60, 20), (1, 7, 8), (30, 1, 36), (6, 6, 4), (11, 3, 8)])
@pytest.mark.parametrize("fma", [False, True])
def test_bin_major_candidates_cover_every_admitted_pair(W, H, N, fma):
    eps = _eps(W, H)
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    I, J = ii.ravel().astype(f32), jj.ravel().astype(f32)
    pairs = 0
    for s, (c, sn, T, nb) in enumerate(_slices(W, H, N)):
        h = f32(f32(0.5) * f32(abs(c) + abs(sn)))
        yr = (J * c).astype(f32) - (I * sn).astype(f32)  # the projection's y' (reading S3)
        if s == 0:
            b0 = jj.ravel() + T
            b1 = b0.copy()
        else:
            lo = ((yr - h).astype(f32) - eps).astype(f32)
            hi = ((yr + h).astype(f32) + eps).astype(f32)
            b0 = np.ceil((lo - f32(0.5)).astype(f32)).astype(np.int64) + T
            b1 = np.floor((hi + f32(0.5)).astype(f32)).astype(np.int64) + T
        b0, b1 = np.maximum(b0, 0), np.minimum(b1, nb - 1)
        cand = {b: _candidates(W, H, c, sn, T, b, eps, h, fma) for b in range(nb)}
        for idx in range(W * H):
            cell = (int(ii.ravel()[idx]), int(jj.ravel()[idx]))
            for b in range(int(b0[idx]), int(b1[idx]) + 1):
                pairs += 1
                assert cell in cand[b], (s, b, cell)
    assert pairs > 0
