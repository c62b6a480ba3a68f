"""ctypes front end of the CPU oracle (``cddt_oracle.c``).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this module.  The product path never does.

Beside the C oracle's O1-O5, prune and update, this module holds plain
NumPy forms of: the 16-bit lookup table's coding and lookups (reading L1),
the motion model and low-variance resampling (readings M1, R1, float64), the
sorted-CSR sector count of the roofline, the baseline casters' direction
rule (D1, through the C library) and the ray marcher's Euclidean distance
transform (scipy's exact transform as a library step, reading RM1).

Parity unpinned: the choices the paper leaves open (the beam-model constants
such as lambda_short = 0.01, the truncated-normal option, range 0 off the map,
the 16-bit Q and X_s); the functions themselves are pinned by the CPU tests.

The C library is built with ``-O2 -ffp-contract=off`` so that float32
expressions are evaluated one rounded operation at a time, exactly in the
order written, on every host (GCC contracts a*b+c into an FMA by default on
aarch64).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cddt_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcddt_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
          "-shared", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (a few seconds)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class BeamModel(C.Structure):
    _fields_ = [("z_hit", C.c_float), ("z_short", C.c_float), ("z_max", C.c_float),
                ("z_rand", C.c_float), ("sigma_hit", C.c_float), ("lambda_short", C.c_float),
                ("max_range", C.c_float), ("hit_truncnorm", C.c_int32)]


def beam_model(max_range: float, z_hit=0.75, z_short=0.01, z_max=0.07, z_rand=0.12,
               sigma_hit=8.0, lambda_short=0.01, hit_truncnorm=0) -> BeamModel:
    return BeamModel(z_hit, z_short, z_max, z_rand, sigma_hit, lambda_short, max_range,
                     hit_truncnorm)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i32, i64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double
            sig = {
                "oc_params_new": (vp, [i32, i32, i32, f32, i32, i32]),
                "oc_params_free": (None, [vp]),
                "oc_params_export": (None, [vp] + [vp] * 7),
                "oc_params_nsl": (i32, [vp]),
                "oc_params_total_bins": (i64, [vp]),
                "oc_edge_map": (None, [vp, i32, i32, vp]),
                "oc_build": (vp, [vp, i32, i32, i32, f32, i32, i32]),
                "oc_free": (None, [vp]),
                "oc_get_params": (vp, [vp]),
                "oc_total_zp": (i64, [vp]),
                "oc_export": (None, [vp, vp, vp]),
                "oc_export_grid": (None, [vp, vp, vp]),
                "oc_calc_range": (None, [vp, vp, i64, vp, i32]),
                "oc_calc_range_info": (None, [vp, vp, i64, vp, vp, vp, vp, vp]),
                "oc_calc_range_brute": (None, [vp, vp, vp, i64, vp, i32]),
                "oc_bin_brute": (i32, [vp, vp, i32, i32, vp, i32]),
                "oc_lut": (None, [vp, vp, vp]),
                "oc_cast_exact": (None, [vp, i32, i32, vp, i64, f64, i32, vp]),
                "oc_cast_bresenham": (None, [vp, i32, i32, vp, i64, f32, vp]),
                "oc_dir_sincos": (None, [f32, vp, vp]),
                "oc_raymarch": (None, [vp, i32, i32, vp, i64, f32, vp, vp]),
                "oc_beam_eval": (None, [vp, vp, vp, i64, vp, vp]),
                "oc_sensor_weights": (None, [vp, vp, i64, vp, vp, i32, vp, vp, vp, i32]),
                "oc_sensor_grad": (None, [vp, vp, i64, vp, vp, i32, vp, vp, vp, vp, i32]),
                "oc_logw_piecewise": (f64, [vp, f64, f64, f32, vp, vp, i32, vp, vp, vp]),
                "oc_traversals": (i32, [vp, f32, vp, i32, i32]),
                "oc_query_k": (i32, [vp, f32]),
                "oc_prune": (i64, [vp, f32]),
                "oc_prune_bin": (None, [vp, vp, i32, i32, vp, i32, f32, vp]),
                "oc_update": (i64, [vp, vp, vp, i64]),
                "oc_has_openmp": (i32, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def prune_eps(W: int, H: int) -> float:
    """Widening of the pruning test (reading S8): 32 units in the last place
    of the largest projected coordinate, 2^(ceil(log2(2 diag + 8)) - 18)."""
    import math
    diag = math.sqrt(W * W + H * H)
    e = math.ceil(math.log2(2.0 * diag + 8.0))
    return float(np.float32(2.0 ** (e - 18)))


class Params:
    """Slice tables of a W x H map with N directions (readings S1-S3, S7)."""

    def __init__(self, W, H, N, max_range, u16=False, full=False, _ptr=None):
        L = lib()
        self._own = _ptr is None
        self.ptr = _ptr if _ptr is not None else L.oc_params_new(W, H, N, max_range, int(u16), int(full))
        if not self.ptr:
            raise ValueError("invalid oracle parameters")
        self.W, self.H, self.N, self.max_range = W, H, N, max_range
        self.nsl = L.oc_params_nsl(self.ptr)
        self.total_bins = L.oc_params_total_bins(self.ptr)
        n = self.nsl
        self.c = np.empty(n, np.float32)
        self.s = np.empty(n, np.float32)
        self.T = np.empty(n, np.int32)
        self.X = np.empty(n, np.float32)
        self.nb = np.empty(n, np.int32)
        self.sbase = np.empty(n + 1, np.int64)
        Q = C.c_double()
        L.oc_params_export(self.ptr, _p(self.c), _p(self.s), _p(self.T), _p(self.X),
                           _p(self.nb), _p(self.sbase), C.byref(Q))
        self.Q = Q.value

    def __del__(self):
        if getattr(self, "_own", False) and self.ptr:
            lib().oc_params_free(self.ptr)
            self.ptr = None

    def query_k(self, theta: float) -> int:
        return lib().oc_query_k(self.ptr, float(theta))

    def calc_range_brute(self, grid, poses, nthreads: int = 1) -> np.ndarray:
        g = _u8(grid)
        q = _f32(poses).reshape(-1, 3)
        out = np.empty(q.shape[0], np.float32)
        lib().oc_calc_range_brute(self.ptr, _p(g), _p(q), q.shape[0], _p(out), nthreads)
        return out

    def bin_brute(self, grid, sl: int, b: int) -> np.ndarray:
        g = _u8(grid)
        cap = 1 << 16
        while True:
            out = np.empty(cap, np.float32)
            n = lib().oc_bin_brute(self.ptr, _p(g), sl, b, _p(out), cap)
            if n <= cap:
                return out[:n].copy()
            cap = n

    def lut(self, grid) -> np.ndarray:
        g = _u8(grid)
        out = np.empty((self.N, self.H, self.W), np.float32)
        lib().oc_lut(self.ptr, _p(g), _p(out))
        return out

    def traversals(self, theta: float, beam_off, D: int) -> int:
        bo = _f32(beam_off)
        return lib().oc_traversals(self.ptr, float(theta), _p(bo), bo.size, D)

    def prune_bin(self, grid, sl, b, zp, eps) -> np.ndarray:
        g = _u8(grid)
        a = _f32(zp)
        keep = np.zeros(max(a.size, 1), np.uint8)
        lib().oc_prune_bin(self.ptr, _p(g), sl, b, _p(a), a.size, eps, _p(keep))
        return keep[:a.size].astype(bool)


def sorted_search_sectors(kb, keys_per_sector: int = 8):
    """32-byte sectors a binary search of a sorted CSR bin of kb keys
    touches (the roofline's sector count): one for the bin's two offsets;
    for a non-empty bin, one per probe while the remaining range spans more
    than one sector (ceil(log2(kb / keys_per_sector)) halvings) and one for
    the last sector.  Array in, array out."""
    k = np.asarray(kb, np.int64)
    out = np.ones(k.shape, np.int64)
    for idx in np.ndindex(k.shape):
        r = int(k[idx])
        if r <= 0:
            continue
        c = 0
        while r > keys_per_sector:
            r = (r + 1) // 2
            c += 1
        out[idx] = 2 + c
    return out


def lut_scale(max_range: float) -> float:
    """The 16-bit table's scale (reading L1): the largest power of two s
    with max_range * s <= 65535, so code = round-half-up(range * s) fits and
    code / s is exact."""
    s = 1.0
    while max_range * s * 2.0 <= 65535.0:
        s *= 2.0
    while max_range * s > 65535.0:
        s /= 2.0
    return s


def lut_table(params, grid, max_range: float) -> np.ndarray:
    """The paper's three-dimensional lookup table (Section II, 16-bit entries,
    Table I): the O4 range of every discrete state (cell centre, theta_k),
    coded as round-half-up(range * scale) in float32, clamped to 65535."""
    r = params.lut(grid)
    sc = np.float32(lut_scale(max_range))
    code = np.floor(r * sc + np.float32(0.5))
    return np.clip(code, 0, 65535).astype(np.uint16)


def lut_lookup(params, table, max_range: float, poses) -> np.ndarray:
    """A query read from the table: its nearest cell centre (floor(x + 1/2),
    floor(y + 1/2) in float32; off the map gives 0) and its direction index
    (as the CDDT's query, S1), code / scale."""
    q = np.asarray(poses, np.float32).reshape(-1, 3)
    N, H, W = table.shape
    inv = np.float32(1.0 / lut_scale(max_range))
    out = np.zeros(q.shape[0], np.float32)
    for n in range(q.shape[0]):
        fx = np.floor(q[n, 0] + np.float32(0.5))
        fy = np.floor(q[n, 1] + np.float32(0.5))
        if not (0 <= fx < W and 0 <= fy < H):
            continue
        k = params.query_k(float(q[n, 2]))
        if k < 0:
            continue
        out[n] = np.float32(table[k, int(fy), int(fx)]) * inv
    return out


def lut_sensor_weights(params, table, max_range: float, particles, beam_off, obs, model) -> np.ndarray:
    """log w of each particle over table reads: the beam model (S9, float64)
    of every beam's looked-up range, summed."""
    q = np.asarray(particles, np.float32).reshape(-1, 3)
    bo = np.asarray(beam_off, np.float32)
    B = bo.size
    dirs = (q[:, 2:3] + bo[None, :]).astype(np.float32)
    poses = np.concatenate([np.repeat(q[:, :2], B, 0), dirs.reshape(-1, 1)], 1)
    r = lut_lookup(params, table, max_range, poses).astype(np.float64)
    z = np.tile(np.asarray(obs, np.float32).astype(np.float64), q.shape[0])
    p, _ = beam_eval(model, z, r)
    return np.log(p).reshape(-1, B).sum(1)


def motion(particles, seg_start, odom, noise) -> np.ndarray:
    """The odometry motion model around the sensor model (Section I names a
    movement model from odometry; the standard increment form is the reading
    used here): each particle moves by the robot's (dx, dy) in its own frame
    plus its noise sample and turns by dtheta plus noise, theta wrapped into
    [0, 2 pi) by one turn.  Evaluated in float64 from the float32 inputs and
    rounded to float32 once.  particles [P, 3], seg_start [F + 1], odom
    [F, 3], noise [P, 3]."""
    x = np.asarray(particles, np.float32).astype(np.float64)
    nz = np.asarray(noise, np.float32).astype(np.float64)
    od = np.asarray(odom, np.float32).astype(np.float64)
    seg = np.asarray(seg_start, np.int64)
    f = np.searchsorted(seg, np.arange(x.shape[0]), side="right") - 1
    a = od[f, 0] + nz[:, 0]
    b = od[f, 1] + nz[:, 1]
    th = x[:, 2]
    out = np.empty_like(x)
    out[:, 0] = x[:, 0] + a * np.cos(th) - b * np.sin(th)
    out[:, 1] = x[:, 1] + a * np.sin(th) + b * np.cos(th)
    t = th + od[f, 2] + nz[:, 2]
    two_pi = 2.0 * np.pi
    t = np.where(t >= two_pi, t - two_pi, np.where(t < 0.0, t + two_pi, t))
    out[:, 2] = t
    return out.astype(np.float32)


def resample_weights(lw):
    """Weights of one filter's log-weights (float64): exp(lw - max lw).  Where
    that is undefined (reading R1): if no log-weight is above -inf (all -inf
    or NaN, no particle has weight) every particle weighs 1; otherwise NaN
    weighs 0, and if the largest is +inf the +inf particles weigh 1 and the
    rest 0."""
    lw = np.asarray(lw, np.float64)
    num = lw[~np.isnan(lw)]
    top = num.max() if num.size else -np.inf
    if top == -np.inf:
        return np.ones(lw.shape[0])
    if top == np.inf:
        return (lw == np.inf).astype(np.float64)
    w = np.exp(lw - top)
    w[np.isnan(lw)] = 0.0
    return w


def resample_indices(logw, seg_start, u0):
    """Low-variance (systematic) resampling of every filter segment (Section
    I resamples by belief; the low-variance scheme is the reading used here):
    w_i = exp(logw_i - max logw) (resample_weights: also where that is
    undefined) and running sums C_i in float64, in index order; output m of a filter of n particles takes the first input i with
    C_i > (u0 + m) / n * C_{n-1} (the last one when none is).  Returns the
    within-filter indices [P] and, per output, the distance of its target
    from the nearest running sum relative to the total (a decision this
    close may round the other way in another summation order)."""
    lw = np.asarray(logw, np.float32).astype(np.float64)
    seg = np.asarray(seg_start, np.int64)
    u = np.asarray(u0, np.float32).astype(np.float64)
    idx = np.zeros(lw.shape[0], np.int64)
    margin = np.zeros(lw.shape[0], np.float64)
    for f in range(seg.size - 1):
        a, b = int(seg[f]), int(seg[f + 1])
        n = b - a
        if n <= 0:
            continue
        w = resample_weights(lw[a:b])
        C = np.cumsum(w)
        tot = C[-1]
        for m in range(n):
            t = (u[f] + m) / n * tot
            i = int(np.searchsorted(C, t, side="right"))
            idx[a + m] = min(i, n - 1)
            margin[a + m] = np.min(np.abs(C - t)) / tot
    return idx, margin


class OracleCDDT:
    """O2: the plain CDDT built on the CPU (Section IV-A), with query, prune,
    update, beam-model weights and gradient."""

    def __init__(self, grid, N: int, max_range: float, u16: bool = False, full: bool = False):
        L = lib()
        g = _u8(grid)
        self.H, self.W = g.shape
        self.N, self.max_range, self.u16, self.full = N, float(max_range), u16, full
        self.ptr = L.oc_build(_p(g), self.W, self.H, N, max_range, int(u16), int(full))
        if not self.ptr:
            raise ValueError("invalid oracle build arguments")
        self.params = Params(self.W, self.H, N, max_range, _ptr=L.oc_get_params(self.ptr))
        self.params._own = False

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().oc_free(self.ptr)
            self.ptr = None

    @property
    def total_zp(self) -> int:
        return lib().oc_total_zp(self.ptr)

    def export(self):
        """(bin_start int64 [total_bins + 1], zp float32 [total])."""
        bs = np.empty(self.params.total_bins + 1, np.int64)
        zp = np.empty(max(self.total_zp, 1), np.float32)
        lib().oc_export(self.ptr, _p(bs), _p(zp))
        return bs, zp[:bs[-1]].copy()

    def grid_edge(self):
        g = np.empty((self.H, self.W), np.uint8)
        e = np.empty((self.H, self.W), np.uint8)
        lib().oc_export_grid(self.ptr, _p(g), _p(e))
        return g, e

    def keys_u16(self, zp: np.ndarray, slice_of_zp: np.ndarray) -> np.ndarray:
        """16-bit keys of stored values (exact inverse of the dequantisation)."""
        p = self.params
        k = (zp.astype(np.float64) + p.X[slice_of_zp].astype(np.float64)) * p.Q
        return np.rint(k).astype(np.uint16)

    def calc_range(self, poses, nthreads: int = 1) -> np.ndarray:
        q = _f32(poses).reshape(-1, 3)
        out = np.empty(q.shape[0], np.float32)
        lib().oc_calc_range(self.ptr, _p(q), q.shape[0], _p(out), nthreads)
        return out

    def calc_range_info(self, poses):
        q = _f32(poses).reshape(-1, 3)
        n = q.shape[0]
        out = np.empty(n, np.float32)
        kb, zi, sl, b = (np.empty(n, np.int32) for _ in range(4))
        lib().oc_calc_range_info(self.ptr, _p(q), n, _p(out), _p(kb), _p(zi), _p(sl), _p(b))
        return out, kb, zi, sl, b

    def sensor_weights(self, particles, beam_off, obs, model: BeamModel, nthreads: int = 1,
                       want_ranges: bool = False):
        q = _f32(particles).reshape(-1, 3)
        bo, ob = _f32(beam_off), _f32(obs)
        P, B = q.shape[0], bo.size
        logw = np.empty(P, np.float64)
        ranges = np.empty((P, B), np.float32) if want_ranges else None
        lib().oc_sensor_weights(self.ptr, _p(q), P, _p(bo), _p(ob), B, C.byref(model), _p(logw),
                                _p(ranges) if want_ranges else None, nthreads)
        return (logw, ranges) if want_ranges else logw

    def sensor_grad(self, particles, beam_off, obs, model: BeamModel, grad_logw=None,
                    nthreads: int = 1):
        """(grad_xy float64 [P, 2], abs_terms float64 [P, 2]); abs_terms is the
        sum of the magnitudes of the per-beam terms (the summation's scale)."""
        q = _f32(particles).reshape(-1, 3)
        bo, ob = _f32(beam_off), _f32(obs)
        P, B = q.shape[0], bo.size
        gl = np.ones(P, np.float64) if grad_logw is None else np.ascontiguousarray(grad_logw, np.float64)
        g = np.empty((P, 2), np.float64)
        a = np.empty((P, 2), np.float64)
        lib().oc_sensor_grad(self.ptr, _p(q), P, _p(bo), _p(ob), B, C.byref(model), _p(gl),
                             _p(g), _p(a), nthreads)
        return g, a

    def logw_piecewise(self, x: float, y: float, theta: float, beam_off, obs, model: BeamModel):
        bo, ob = _f32(beam_off), _f32(obs)
        st = C.c_uint64()
        gr = np.empty(2, np.float64)
        v = lib().oc_logw_piecewise(self.ptr, x, y, float(theta), _p(bo), _p(ob), bo.size,
                                    C.byref(model), C.byref(st), _p(gr))
        return v, st.value, gr

    def prune(self, eps: float | None = None) -> int:
        if eps is None:
            eps = prune_eps(self.W, self.H)
        return lib().oc_prune(self.ptr, eps)

    def update(self, xy, occ) -> int:
        a = np.ascontiguousarray(xy, np.int32).reshape(-1, 2)
        o = _u8(occ)
        return lib().oc_update(self.ptr, _p(a), _p(o), a.shape[0])


def edge_map(grid) -> np.ndarray:
    g = _u8(grid)
    H, W = g.shape
    e = np.empty_like(g)
    lib().oc_edge_map(_p(g), W, H, _p(e))
    return e


def beam_eval(model: BeamModel, z, zs):
    z = np.ascontiguousarray(z, np.float64)
    zs = np.ascontiguousarray(zs, np.float64)
    p = np.empty_like(z)
    dp = np.empty_like(z)
    lib().oc_beam_eval(C.byref(model), _p(z), _p(zs), z.size, _p(p), _p(dp))
    return p, dp


def cast_exact(grid, poses, max_range: float, mode: int = 0) -> np.ndarray:
    g = _u8(grid)
    H, W = g.shape
    q = np.ascontiguousarray(poses, np.float64).reshape(-1, 3)
    out = np.empty(q.shape[0], np.float64)
    lib().oc_cast_exact(_p(g), W, H, _p(q), q.shape[0], max_range, mode, _p(out))
    return out


def cast_bresenham(grid, poses, max_range: float) -> np.ndarray:
    """Bresenham's line caster (Section II), float32 poses -> float32 ranges."""
    g = _u8(grid)
    H, W = g.shape
    q = np.ascontiguousarray(poses, np.float32).reshape(-1, 3)
    out = np.empty(q.shape[0], np.float32)
    lib().oc_cast_bresenham(_p(g), W, H, _p(q), q.shape[0], float(np.float32(max_range)), _p(out))
    return out


def dir_sincos(theta) -> tuple[np.ndarray, np.ndarray]:
    """(sin, cos) of float32 headings by the baseline casters' direction rule
    (reading D1)."""
    th = np.ascontiguousarray(theta, np.float32).reshape(-1)
    s = np.empty_like(th)
    c = np.empty_like(th)
    fs, fc = C.c_float(), C.c_float()
    fn = lib().oc_dir_sincos
    for i, t in enumerate(th.tolist()):
        fn(t, C.byref(fs), C.byref(fc))
        s[i], c[i] = fs.value, fc.value
    return s, c


def edt(grid) -> np.ndarray:
    """Euclidean distance transform for ray marching (Section II, reading
    RM1): float32 [H, W], each cell's distance from its centre to the nearest
    occupied cell's centre, sqrt of the exact integer squared distance taken
    in float64 and rounded to float32; W + H everywhere on a map with no
    occupied cell.  The nearest occupied cell comes from scipy's exact
    transform (its indices; the distance itself is recomputed here in
    integers)."""
    from scipy import ndimage

    occ = _u8(grid) != 0
    H, W = occ.shape
    if not occ.any():
        return np.full((H, W), np.float32(W + H), np.float32)
    idx = ndimage.distance_transform_edt(~occ, return_distances=False, return_indices=True)
    jj, ii = np.mgrid[0:H, 0:W]
    d2 = (jj - idx[0]).astype(np.int64) ** 2 + (ii - idx[1]).astype(np.int64) ** 2
    return np.sqrt(d2.astype(np.float64)).astype(np.float32)


def raymarch(dist, poses, max_range: float):
    """Ray marching over the transform ``dist`` (Section II, reading RM1):
    (ranges float32 [n], distance reads int32 [n])."""
    E = np.ascontiguousarray(dist, np.float32)
    H, W = E.shape
    q = np.ascontiguousarray(poses, np.float32).reshape(-1, 3)
    out = np.empty(q.shape[0], np.float32)
    steps = np.empty(q.shape[0], np.int32)
    lib().oc_raymarch(_p(E), W, H, _p(q), q.shape[0], float(np.float32(max_range)), _p(out), _p(steps))
    return out, steps


def openmp_threads() -> int:
    return lib().oc_has_openmp()
