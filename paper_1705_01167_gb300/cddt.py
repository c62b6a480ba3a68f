"""Thin Python binding of libcddt.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module checks
tensor shapes, dtypes and devices, passes raw device pointers and the current
torch CUDA stream, and turns status codes into exceptions.  There is no CPU
path: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

(CDDT_OK, CDDT_ERR_ARG, CDDT_ERR_CUDA, CDDT_ERR_OOM, CDDT_ERR_PRUNED, CDDT_ERR_TIMEOUT, CDDT_ERR_DEVICE,
 CDDT_ERR_BOUNDS) = range(8)
CDDT_ZP_U16 = 1
SEARCH_TREE, SEARCH_BINARY = 0, 1

EXPORTED = (
    "cddt_build", "cddt_destroy", "cddt_prune", "cddt_update_cells", "cddt_calc_range_many",
    "cddt_sensor_weights", "cddt_sensor_weights_backward", "cddt_sensor_weights_fwd_bwd",
    "cddt_plan_create", "cddt_plan_autotune", "cddt_plan_set_shape", "cddt_plan_get_shape",
    "cddt_plan_run", "cddt_plan_refine", "cddt_plan_launch_graph", "cddt_plan_items", "cddt_plan_destroy",
    "cddt_set_search", "cddt_get_stats", "cddt_get_status", "cddt_export", "cddt_export_grid",
    "cddt_sensor_work", "cddt_status_string", "cddt_version", "cddt_calc_range_many_noalloc", "cddt_plan_groups",
    "cddt_import", "cddt_gather_probe", "cddt_calc_range_timed", "cddt_motion", "cddt_resample",
    "cddt_lut_build", "cddt_lut_destroy", "cddt_lut_info", "cddt_lut_calc_range_many", "cddt_lut_sensor_weights",
    "cddt_cast_bresenham", "cddt_checked_build", "cddt_trace_enable", "cddt_trace_report",
    "cddt_rm_build", "cddt_rm_destroy", "cddt_rm_distances", "cddt_rm_calc_range_many",
)
NOALLOC_MAX_QUERIES = 262144
NOALLOC_MAX_THETA_DISC = 2048


class CDDTError(RuntimeError):
    """A failed C-ABI call: .status holds the cddt_status code."""
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class BeamModel(C.Structure):
    """cddt_beam_model: the beam sensor model mixture (Section VI)."""
    _fields_ = [("z_hit", C.c_float), ("z_short", C.c_float), ("z_max", C.c_float),
                ("z_rand", C.c_float), ("sigma_hit", C.c_float), ("lambda_short", C.c_float),
                ("max_range", C.c_float), ("hit_truncnorm", C.c_int32)]


def beam_model(max_range: float, z_hit=0.75, z_short=0.01, z_max=0.07, z_rand=0.12,
               sigma_hit=8.0, lambda_short=0.01, hit_truncnorm=0) -> BeamModel:
    """The beam sensor model's parameters (reading S9) as the C struct, ranges in cells."""
    return BeamModel(z_hit, z_short, z_max, z_rand, sigma_hit, lambda_short, max_range,
                     int(hit_truncnorm))


class Stats(C.Structure):
    """cddt_stats: sizes and timings of a handle (cddt_get_stats)."""
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("theta_disc", C.c_int32),
                ("n_slices", C.c_int32), ("max_range", C.c_float), ("flags", C.c_uint32),
                ("pruned", C.c_int32), ("total_bins", C.c_int64), ("n_zero_points", C.c_int64),
                ("n_edge_cells", C.c_int64), ("store_bytes", C.c_int64), ("max_bin", C.c_int64),
                ("build_ms", C.c_float), ("prune_ms", C.c_float), ("update_ms", C.c_float)]

    def as_dict(self):
        """The fields as a dict."""
        return {k: getattr(self, k) for k, _ in self._fields_}


class Filter(C.Structure):
    """cddt_filter: one filter of a plan (map handle, particles, scan, model, log-weights)."""
    _fields_ = [("map", C.c_void_p), ("particles_dev", C.c_void_p), ("P", C.c_int64),
                ("beam_off_dev", C.c_void_p), ("obs_dev", C.c_void_p), ("B", C.c_int32),
                ("pair_offset", C.c_int32), ("model", BeamModel), ("logw_dev", C.c_void_p),
                ("grad_xy_dev", C.c_void_p), ("particles_out_dev", C.c_void_p)]


def library_path() -> str:
    """Path of the in-tree libcddt.so."""
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcddt.so (building it first if it is missing or stale); with
    CDDT_CHECKED=1 in the environment, its bounds-checked variant."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        checked = os.environ.get("CDDT_CHECKED", "") == "1"
        path = _build.CHECKED_LIB if checked else _build.LIB
        if build_if_missing and not _build.up_to_date(path):
            _build.build_checked() if checked else _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libcddt.so is not built ({path}); run paper_1705_01167_gb300.build")
        L = C.CDLL(path)
        vp, i32, i64, u32, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_float
        st = C.c_int
        sig = {
            "cddt_build": (st, [vp, i32, i32, i32, f32, u32, vp, C.POINTER(vp)]),
            "cddt_destroy": (st, [vp]),
            "cddt_prune": (st, [vp, vp]),
            "cddt_update_cells": (st, [vp, vp, vp, i32, vp]),
            "cddt_calc_range_many": (st, [vp, vp, vp, i64, i32, vp]),
            "cddt_calc_range_many_noalloc": (st, [vp, vp, vp, i64, vp]),
            "cddt_sensor_weights": (st, [vp, vp, i64, vp, vp, i32, i32, C.POINTER(BeamModel), vp, vp, vp]),
            "cddt_sensor_weights_backward": (st, [vp, vp, i64, vp, vp, i32, i32, C.POINTER(BeamModel), vp, vp, vp]),
            "cddt_sensor_weights_fwd_bwd": (st, [vp, vp, i64, vp, vp, i32, i32, C.POINTER(BeamModel), vp, vp, vp]),
            "cddt_plan_create": (st, [C.POINTER(Filter), i32, vp, C.POINTER(vp)]),
            "cddt_plan_autotune": (st, [vp, vp]),
            "cddt_plan_set_shape": (st, [vp, i32, i32, i32, i32]),
            "cddt_plan_get_shape": (st, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
            "cddt_plan_run": (st, [vp, vp]),
            "cddt_plan_refine": (st, [vp, i32, f32, i32, vp]),
            "cddt_plan_launch_graph": (st, [vp, vp]),
            "cddt_plan_items": (i64, [vp]),
            "cddt_plan_groups": (st, [vp, vp]),
            "cddt_plan_destroy": (st, [vp]),
            "cddt_set_search": (st, [vp, i32]),
            "cddt_get_stats": (st, [vp, C.POINTER(Stats)]),
            "cddt_get_status": (st, [vp]),
            "cddt_export": (st, [vp, vp, vp, vp]),
            "cddt_import": (st, [vp, i32, i32, i32, f32, u32, i32, i64, vp, vp, vp, C.POINTER(vp)]),
            "cddt_gather_probe": (st, [vp, i64, i64, C.c_uint64, vp, vp]),
            "cddt_calc_range_timed": (st, [vp, vp, vp, i64, vp, vp]),
            "cddt_motion": (st, [vp, i64, vp, i32, vp, vp, vp]),
            "cddt_lut_build": (st, [vp, vp, C.POINTER(vp)]),
            "cddt_cast_bresenham": (st, [vp, vp, vp, i64, vp]),
            "cddt_rm_build": (st, [vp, vp, C.POINTER(vp)]),
            "cddt_checked_build": (i32, []),
            "cddt_trace_enable": (st, [i32]),
            "cddt_trace_report": (st, [C.c_char_p, i64, C.POINTER(i64)]),
            "cddt_rm_destroy": (st, [vp]),
            "cddt_rm_distances": (st, [vp, C.POINTER(vp), C.POINTER(i64)]),
            "cddt_rm_calc_range_many": (st, [vp, vp, vp, vp, i64, vp]),
            "cddt_lut_destroy": (st, [vp]),
            "cddt_lut_info": (st, [vp, C.POINTER(i64), C.POINTER(f32)]),
            "cddt_lut_calc_range_many": (st, [vp, vp, vp, i64, vp]),
            "cddt_lut_sensor_weights": (st, [vp, vp, i64, vp, i32, vp, vp, i32, C.POINTER(BeamModel), vp, vp]),
            "cddt_resample": (st, [vp, vp, vp, i32, vp, vp, vp, vp, vp]),
            "cddt_export_grid": (st, [vp, vp, vp]),
            "cddt_sensor_work": (st, [vp, vp, i64, vp, i32, i32, vp, vp]),
            "cddt_status_string": (C.c_char_p, [st]),
            "cddt_version": (i32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def status_string(s: int) -> str:
    """cddt_status_string: the text of a status code."""
    return load().cddt_status_string(s).decode()


def _check(rc: int, what: str):
    if rc != CDDT_OK:
        raise CDDTError(rc, what)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_or_pinned(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    """A CUDA tensor, or a page-locked host tensor (kernels address it
    directly under unified addressing)."""
    if isinstance(t, torch.Tensor) and not t.is_cuda and (t.is_pinned() or t.numel() == 0):
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t
    return _dev(t, dtype, name)


def _dev(t: torch.Tensor, dtype, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None:
        for i, s in enumerate(shape):
            if s is not None and t.shape[i] != s:
                raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
    return t


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def pair_offset(beam_off) -> int:
    """Index distance D with beam_off[i + D] - beam_off[i] = pi for every
    paired i (0 when the layout has none).  Host-side hint only: the kernels
    verify every pair and the result never depends on D."""
    import numpy as np
    b = np.asarray(beam_off.detach().cpu() if isinstance(beam_off, torch.Tensor) else beam_off,
                   dtype=np.float64)
    B = b.size
    for D in range((B + 1) // 2, B):
        d = b[D:] - b[:B - D]
        if np.all(np.abs(d - math.pi) < 1e-5):
            return D
    return 0


class CDDT:
    """One Compressed Directional Distance Transform on the current CUDA
    device (Section IV): ``cddt_build`` on a uint8 occupancy grid [H, W]."""

    def __init__(self, grid: torch.Tensor, theta_disc: int, max_range: float, u16: bool = False,
                 stream=None):
        L = load()
        _dev(grid, torch.uint8, "grid")
        if grid.dim() != 2:
            raise ValueError("grid must be [H, W]")
        self.H, self.W = grid.shape
        self.theta_disc = int(theta_disc)
        self.max_range = float(max_range)
        self.u16 = bool(u16)
        self.device = grid.device
        h = C.c_void_p()
        with torch.cuda.device(grid.device):
            rc = L.cddt_build(_ptr(grid), self.W, self.H, self.theta_disc, self.max_range,
                              CDDT_ZP_U16 if u16 else 0, _stream(stream), C.byref(h))
        _check(rc, "cddt_build")
        self._h = h

    @classmethod
    def from_export(cls, grid: torch.Tensor, theta_disc: int, max_range: float, bin_start, zp,
                    u16: bool = False, pruned: bool = False, stream=None) -> "CDDT":
        """``cddt_import``: a handle whose store is the CSR ``(bin_start, zp)``
        that ``export()`` returned for the same grid and parameters."""
        import numpy as np
        L = load()
        _dev(grid, torch.uint8, "grid")
        if grid.dim() != 2:
            raise ValueError("grid must be [H, W]")
        bs = np.ascontiguousarray(bin_start, np.int64)
        z = np.ascontiguousarray(zp, np.float32)
        if bs.ndim != 1 or bs.size < 1 or z.size < bs[-1]:
            raise ValueError("bin_start must be [bins + 1] and zp hold bin_start[-1] values")
        self = cls.__new__(cls)
        self.H, self.W = grid.shape
        self.theta_disc = int(theta_disc)
        self.max_range = float(max_range)
        self.u16 = bool(u16)
        self.device = grid.device
        h = C.c_void_p()
        with torch.cuda.device(grid.device):
            rc = L.cddt_import(_ptr(grid), self.W, self.H, self.theta_disc, self.max_range,
                               CDDT_ZP_U16 if u16 else 0, int(bool(pruned)), bs.size - 1,
                               bs.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p) if z.size else None,
                               _stream(stream), C.byref(h))
        _check(rc, "cddt_import")
        self._h = h
        return self

    @property
    def handle(self):
        """The C handle (cddt_t) as a ctypes pointer."""
        return self._h

    def close(self):
        """cddt_destroy: free the handle's device memory (idempotent)."""
        if getattr(self, "_h", None):
            load().cddt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- maintenance
    def prune(self, stream=None):
        """cddt_prune: drop the zero points no free-space query can return (Section IV-C)."""
        with torch.cuda.device(self.device):
            _check(load().cddt_prune(self._h, _stream(stream)), "cddt_prune")

    def update_cells(self, xy: torch.Tensor, occ: torch.Tensor, stream=None):
        """cddt_update_cells: write cells (xy int32 [n, 2], occ uint8 [n]) into the map and the store (Section IV-D)."""
        _dev(xy, torch.int32, "xy")
        _dev(occ, torch.uint8, "occ")
        n = occ.numel()
        if xy.numel() != 2 * n:
            raise ValueError("xy must be [n, 2] and occ [n]")
        with torch.cuda.device(self.device):
            _check(load().cddt_update_cells(self._h, _ptr(xy), _ptr(occ), n, _stream(stream)),
                   "cddt_update_cells")

    def set_search(self, search: int):
        """cddt_set_search: SEARCH_TREE (the default) or SEARCH_BINARY over the same store."""
        _check(load().cddt_set_search(self._h, search), "cddt_set_search")

    def stats(self) -> dict:
        """cddt_get_stats as a dict."""
        s = Stats()
        with torch.cuda.device(self.device):
            _check(load().cddt_get_stats(self._h, C.byref(s)), "cddt_get_stats")
        return s.as_dict()

    def status(self) -> int:
        """cddt_get_status: the device status word (read and cleared)."""
        with torch.cuda.device(self.device):
            return load().cddt_get_status(self._h)

    def export(self):
        """(slice_base int64 [S+1], bin_start int64 [bins+1], zp float32 [n]) on the host."""
        import numpy as np
        st = self.stats()
        sb = np.empty(st["n_slices"] + 1, np.int64)
        bs = np.empty(st["total_bins"] + 1, np.int64)
        zp = np.empty(max(st["n_zero_points"], 1), np.float32)
        with torch.cuda.device(self.device):
            _check(load().cddt_export(self._h, sb.ctypes.data_as(C.c_void_p),
                                      bs.ctypes.data_as(C.c_void_p),
                                      zp.ctypes.data_as(C.c_void_p)), "cddt_export")
        return sb, bs, zp[:bs[-1]].copy()

    def export_grid(self):
        """cddt_export_grid: (grid, edge map) as uint8 [H, W] host arrays."""
        import numpy as np
        g = np.empty((self.H, self.W), np.uint8)
        e = np.empty((self.H, self.W), np.uint8)
        with torch.cuda.device(self.device):
            _check(load().cddt_export_grid(self._h, g.ctypes.data_as(C.c_void_p),
                                           e.ctypes.data_as(C.c_void_p)), "cddt_export_grid")
        return g, e

    # ---- queries
    def calc_range_many(self, poses: torch.Tensor, sort_by_slice: bool = False,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """cddt_calc_range_many: ranges [n] of poses [n, 3] (optionally slice-sorted, same answers)."""
        _dev(poses, torch.float32, "poses")
        n = poses.numel() // 3
        if poses.numel() != 3 * n:
            raise ValueError("poses must be [n, 3]")
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=poses.device)
        _dev(out, torch.float32, "out")
        with torch.cuda.device(self.device):
            _check(load().cddt_calc_range_many(self._h, _ptr(poses), _ptr(out), n,
                                               int(bool(sort_by_slice)), _stream(stream)),
                   "cddt_calc_range_many")
        return out

    def calc_range_many_noalloc(self, poses: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """Slice-sorted ray casts into ``out`` with no device allocation (the
        library's fixed scratch; at most NOALLOC_MAX_QUERIES queries)."""
        _dev(poses, torch.float32, "poses")
        _dev(out, torch.float32, "out")
        n = poses.numel() // 3
        if poses.numel() != 3 * n or out.numel() != n:
            raise ValueError("poses must be [n, 3] and out [n]")
        with torch.cuda.device(self.device):
            _check(load().cddt_calc_range_many_noalloc(self._h, _ptr(poses), _ptr(out), n, _stream(stream)),
                   "cddt_calc_range_many_noalloc")
        return out

    def _sensor_args(self, particles, beam_off, obs, pinned_ok: bool = False):
        check = _dev_or_pinned if pinned_ok else _dev
        check(particles, torch.float32, "particles")
        check(beam_off, torch.float32, "beam_off")
        check(obs, torch.float32, "obs")
        P = particles.numel() // 3
        B = beam_off.numel()
        if particles.numel() != 3 * P or obs.numel() != B:
            raise ValueError("particles must be [P, 3] and obs [B] like beam_off")
        return P, B

    def cast_bresenham(self, poses: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """``cddt_cast_bresenham``: the Bresenham baseline caster on this map."""
        _dev(poses, torch.float32, "poses")
        n = poses.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=poses.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_cast_bresenham(self._h, _ptr(poses), _ptr(out), n, _stream(stream)),
                   "cddt_cast_bresenham")
        return out

    def calc_range_timed(self, poses: torch.Tensor, stream=None):
        """``cddt_calc_range_timed``: (ranges [n], SM cycles of each warp of 32
        consecutive queries [ceil(n / 32)])."""
        _dev(poses, torch.float32, "poses")
        n = poses.numel() // 3
        out = torch.empty(n, dtype=torch.float32, device=poses.device)
        cyc = torch.empty((n + 31) // 32, dtype=torch.int64, device=poses.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_calc_range_timed(self._h, _ptr(poses), _ptr(out), n, _ptr(cyc), _stream(stream)),
                   "cddt_calc_range_timed")
        return out, cyc

    def sensor_weights(self, particles, beam_off, obs, model: BeamModel, pair_offset: int = 0,
                       want_ranges: bool = False, logw=None, stream=None):
        """cddt_sensor_weights: log-weights [P] of particles [P, 3] (and the ranges [P, B] when asked)."""
        P, B = self._sensor_args(particles, beam_off, obs)
        if logw is None:
            logw = torch.empty(P, dtype=torch.float32, device=particles.device)
        ranges = torch.empty((P, B), dtype=torch.float32, device=particles.device) if want_ranges else None
        with torch.cuda.device(self.device):
            _check(load().cddt_sensor_weights(self._h, _ptr(particles), P, _ptr(beam_off), _ptr(obs),
                                              B, pair_offset, C.byref(model), _ptr(logw),
                                              _ptr(ranges), _stream(stream)),
                   "cddt_sensor_weights")
        return (logw, ranges) if want_ranges else logw

    def sensor_weights_backward(self, particles, beam_off, obs, model: BeamModel, grad_logw,
                                pair_offset: int = 0, grad_xy=None, stream=None):
        """cddt_sensor_weights_backward: d(log w)/d(x, y) [P, 2] scaled by grad_logw [P]."""
        P, B = self._sensor_args(particles, beam_off, obs)
        _dev(grad_logw, torch.float32, "grad_logw")
        if grad_xy is None:
            grad_xy = torch.empty((P, 2), dtype=torch.float32, device=particles.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_sensor_weights_backward(self._h, _ptr(particles), P, _ptr(beam_off),
                                                       _ptr(obs), B, pair_offset, C.byref(model),
                                                       _ptr(grad_logw), _ptr(grad_xy),
                                                       _stream(stream)),
                   "cddt_sensor_weights_backward")
        return grad_xy

    def sensor_weights_fwd_bwd(self, particles, beam_off, obs, model: BeamModel,
                               pair_offset: int = 0, logw=None, grad_xy=None, stream=None):
        """cddt_sensor_weights_fwd_bwd: log-weights and their gradient in one pass."""
        P, B = self._sensor_args(particles, beam_off, obs)
        if logw is None:
            logw = torch.empty(P, dtype=torch.float32, device=particles.device)
        if grad_xy is None:
            grad_xy = torch.empty((P, 2), dtype=torch.float32, device=particles.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_sensor_weights_fwd_bwd(self._h, _ptr(particles), P, _ptr(beam_off),
                                                      _ptr(obs), B, pair_offset, C.byref(model),
                                                      _ptr(logw), _ptr(grad_xy), _stream(stream)),
                   "cddt_sensor_weights_fwd_bwd")
        return logw, grad_xy

    def sensor_work(self, particles, beam_off, pair_offset: int = 0, stream=None):
        """Work figures of one sensor_weights launch (see cddt.h)."""
        import numpy as np
        _dev(particles, torch.float32, "particles")
        _dev(beam_off, torch.float32, "beam_off")
        out = np.zeros(7, np.int64)
        with torch.cuda.device(self.device):
            _check(load().cddt_sensor_work(self._h, _ptr(particles), particles.numel() // 3,
                                           _ptr(beam_off), beam_off.numel(), pair_offset,
                                           out.ctypes.data_as(C.c_void_p), _stream(stream)),
                   "cddt_sensor_work")
        keys = ("traversals", "beams", "nonempty", "probes", "paired", "passed", "sectors")
        return dict(zip(keys, (int(v) for v in out)))


class SensorWeights(torch.autograd.Function):
    """log w = cddt_sensor_weights(particles); backward = the adjoint kernel
    (d log w / d(x, y); the theta column receives zero gradient)."""

    @staticmethod
    def forward(ctx, particles, cddt: CDDT, beam_off, obs, model: BeamModel, pair_offset: int = 0):
        """The forward pass: log-weights of the particles."""
        p = particles.detach().contiguous()
        logw = cddt.sensor_weights(p, beam_off, obs, model, pair_offset)
        ctx.save_for_backward(p)
        ctx.cddt, ctx.beam_off, ctx.obs, ctx.model, ctx.D = cddt, beam_off, obs, model, pair_offset
        return logw

    @staticmethod
    def backward(ctx, grad_logw):
        """The adjoint: the gradient with respect to the particles' (x, y); theta gets 0."""
        (p,) = ctx.saved_tensors
        g = ctx.cddt.sensor_weights_backward(p, ctx.beam_off, ctx.obs, ctx.model,
                                             grad_logw.contiguous().float(), ctx.D)
        grad = torch.zeros_like(p)
        grad[:, :2] = g
        return grad, None, None, None, None, None


def gather_probe(buf: torch.Tensor, sectors: int, seed: int = 1, sink: torch.Tensor | None = None, stream=None):
    """``cddt_gather_probe``: read ``sectors`` random 32-byte sectors of the
    CUDA buffer ``buf`` (time it with CUDA events)."""
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int64, device=buf.device)
    with torch.cuda.device(buf.device):
        _check(load().cddt_gather_probe(_ptr(buf), buf.numel() * buf.element_size() // 32 * 32, int(sectors),
                                        int(seed), _ptr(sink), _stream(stream)), "cddt_gather_probe")
    return sink


class Lut:
    """``cddt_lut_*``: the paper's 3D lookup table of every discrete state's
    range (16-bit), built from a CDDT; queries snap to their state."""

    def __init__(self, cddt: "CDDT", stream=None):
        h = C.c_void_p()
        with torch.cuda.device(cddt.device):
            _check(load().cddt_lut_build(cddt.handle, _stream(stream), C.byref(h)), "cddt_lut_build")
        self._h = h
        self.device = cddt.device

    def info(self):
        """cddt_lut_info: {'bytes', 'scale'} of the table."""
        b, sc = C.c_int64(), C.c_float()
        _check(load().cddt_lut_info(self._h, C.byref(b), C.byref(sc)), "cddt_lut_info")
        return {"bytes": b.value, "scale": sc.value}

    def calc_range_many(self, poses: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """cddt_lut_calc_range_many: ranges [n] read from the table at each pose's state."""
        _dev(poses, torch.float32, "poses")
        n = poses.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=poses.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_lut_calc_range_many(self._h, _ptr(poses), _ptr(out), n, _stream(stream)),
                   "cddt_lut_calc_range_many")
        return out

    def sensor_weights(self, particles, seg_start, beam_off, obs, model: BeamModel, logw=None, stream=None):
        """obs [F, B] (one scan per filter segment of particles)."""
        _dev(particles, torch.float32, "particles")
        _dev(seg_start, torch.int64, "seg_start")
        _dev(beam_off, torch.float32, "beam_off")
        _dev(obs, torch.float32, "obs")
        P, F, B = particles.numel() // 3, seg_start.numel() - 1, beam_off.numel()
        if obs.numel() != F * B:
            raise ValueError("obs must be [F, B]")
        if logw is None:
            logw = torch.empty(P, dtype=torch.float32, device=particles.device)
        with torch.cuda.device(self.device):
            _check(load().cddt_lut_sensor_weights(self._h, _ptr(particles), P, _ptr(seg_start), F, _ptr(beam_off),
                                                  _ptr(obs), B, C.byref(model), _ptr(logw), _stream(stream)),
                   "cddt_lut_sensor_weights")
        return logw

    def close(self):
        """cddt_lut_destroy (idempotent)."""
        if getattr(self, "_h", None):
            load().cddt_lut_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_enable(on: bool = True):
    """``cddt_trace_enable``: time every C-ABI call with CUDA events on its
    stream (see ``trace_report``)."""
    _check(load().cddt_trace_enable(1 if on else 0), "cddt_trace_enable")


def trace_report() -> list[dict]:
    """``cddt_trace_report``: per entry point, the calls and their device
    time in ms (total, mean, min, max) since the last report, which it clears."""
    need = C.c_int64()
    buf = C.create_string_buffer(1 << 16)
    _check(load().cddt_trace_report(buf, len(buf), C.byref(need)), "cddt_trace_report")
    if need.value > len(buf):
        raise RuntimeError("cddt_trace_report: summary truncated")
    lines = buf.value.decode().strip().splitlines()
    out = []
    for ln in lines[1:]:
        name, calls, total, mean, lo, hi = ln.split(",")
        out.append({"entry": name, "calls": int(calls), "total_ms": float(total), "mean_ms": float(mean),
                    "min_ms": float(lo), "max_ms": float(hi)})
    return out


class RayMarch:
    """``cddt_rm_*``: the paper's ray marching baseline, a Euclidean distance
    transform of a CDDT's grid (a snapshot at construction) and a caster that
    steps each ray by it."""

    def __init__(self, cddt: "CDDT", stream=None):
        h = C.c_void_p()
        with torch.cuda.device(cddt.device):
            _check(load().cddt_rm_build(cddt.handle, _stream(stream), C.byref(h)), "cddt_rm_build")
        self._h = h
        self.device = cddt.device
        self.shape = (cddt.H, cddt.W)

    def distances(self) -> torch.Tensor:
        """A copy of the transform, float32 [H, W]."""
        p, b = C.c_void_p(), C.c_int64()
        _check(load().cddt_rm_distances(self._h, C.byref(p), C.byref(b)), "cddt_rm_distances")
        if b.value != 4 * self.shape[0] * self.shape[1]:
            raise RuntimeError("cddt_rm_distances: unexpected size")

        class _View:  # the object's own buffer, seen through the CUDA array interface
            __cuda_array_interface__ = {"shape": self.shape, "typestr": "<f4", "data": (p.value, False),
                                        "strides": None, "version": 3}

        with torch.cuda.device(self.device):
            return torch.as_tensor(_View(), device=self.device).clone()

    def calc_range_many(self, poses: torch.Tensor, out: torch.Tensor | None = None,
                        steps: torch.Tensor | None = None, stream=None):
        """Ranges [n] (and, into ``steps`` int32 [n] when given, the reads of
        each ray)."""
        _dev(poses, torch.float32, "poses")
        n = poses.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=poses.device)
        if steps is not None:
            _dev(steps, torch.int32, "steps")
            if steps.numel() != n:
                raise ValueError("steps must hold one int32 per pose")
        with torch.cuda.device(self.device):
            _check(load().cddt_rm_calc_range_many(self._h, _ptr(poses), _ptr(out),
                                                  _ptr(steps) if steps is not None else None, n,
                                                  _stream(stream)), "cddt_rm_calc_range_many")
        return out

    def close(self):
        """cddt_rm_destroy (idempotent)."""
        if getattr(self, "_h", None):
            load().cddt_rm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def motion(particles: torch.Tensor, seg_start: torch.Tensor, odom: torch.Tensor, noise: torch.Tensor,
           stream=None) -> torch.Tensor:
    """``cddt_motion``: odometry motion model, in place on particles [P, 3]
    (filters are the segments seg_start [F + 1] int64; odom [F, 3]; noise
    [P, 3])."""
    _dev(particles, torch.float32, "particles")
    _dev(seg_start, torch.int64, "seg_start")
    _dev(odom, torch.float32, "odom")
    _dev(noise, torch.float32, "noise")
    P, F = particles.numel() // 3, seg_start.numel() - 1
    if noise.numel() != 3 * P or odom.numel() != 3 * F or F < 1:
        raise ValueError("noise must be [P, 3], odom [F, 3] and seg_start [F + 1]")
    with torch.cuda.device(particles.device):
        _check(load().cddt_motion(_ptr(particles), P, _ptr(seg_start), F, _ptr(odom), _ptr(noise),
                                  _stream(stream)), "cddt_motion")
    return particles


def resample(particles: torch.Tensor, logw: torch.Tensor, seg_start: torch.Tensor, u0: torch.Tensor,
             out: torch.Tensor | None = None, index: torch.Tensor | None = None,
             scratch: torch.Tensor | None = None, stream=None):
    """``cddt_resample``: low-variance resampling of every filter segment;
    returns (out [P, 3], index [P] int32 or None)."""
    _dev(particles, torch.float32, "particles")
    _dev(logw, torch.float32, "logw")
    _dev(seg_start, torch.int64, "seg_start")
    _dev(u0, torch.float32, "u0")
    P, F = particles.numel() // 3, seg_start.numel() - 1
    if logw.numel() != P or u0.numel() != F or F < 1:
        raise ValueError("logw must be [P], u0 [F] and seg_start [F + 1]")
    if out is None:
        out = torch.empty_like(particles)
    if scratch is None:
        scratch = torch.empty(max(P, 1), dtype=torch.float64, device=particles.device)
    _dev(out, torch.float32, "out")
    _dev(scratch, torch.float64, "scratch")
    if index is not None:
        _dev(index, torch.int32, "index")
    with torch.cuda.device(particles.device):
        _check(load().cddt_resample(_ptr(particles), _ptr(logw), _ptr(seg_start), F, _ptr(u0), _ptr(out),
                                    _ptr(index) if index is not None else None, _ptr(scratch), _stream(stream)),
               "cddt_resample")
    return out, index


class Plan:
    """Many filters (maps of any size, any particle count) weighted in one
    persistent launch (``cddt_plan_*``), optionally replayed as a CUDA graph.
    Particles, scans and log-weights may be CUDA tensors or page-locked host
    tensors (read and written by the kernel across the host link)."""

    def __init__(self, filters: list[dict], stream=None):
        L = load()
        arr = (Filter * len(filters))()
        self._keep = []
        for i, f in enumerate(filters):
            m: CDDT = f["map"]
            P, B = m._sensor_args(f["particles"], f["beam_off"], f["obs"], pinned_ok=True)
            _dev_or_pinned(f["logw"], torch.float32, "logw")
            grad, pout = f.get("grad_xy"), f.get("particles_out")
            if grad is not None:
                _dev(grad, torch.float32, "grad_xy", (P, 2))
            if pout is not None:
                _dev(pout, torch.float32, "particles_out", (P, 3))
            arr[i] = Filter(m.handle.value, f["particles"].data_ptr(), P, f["beam_off"].data_ptr(),
                            f["obs"].data_ptr(), B, int(f.get("pair_offset", 0)), f["model"],
                            f["logw"].data_ptr(), grad.data_ptr() if grad is not None else None,
                            pout.data_ptr() if pout is not None else None)
            self._keep.append(f)
        h = C.c_void_p()
        _check(L.cddt_plan_create(arr, len(filters), _stream(stream), C.byref(h)), "cddt_plan_create")
        self._h = h

    def autotune(self, stream=None):
        """cddt_plan_autotune: time the candidate launch shapes on the plan's own work, keep the fastest."""
        _check(load().cddt_plan_autotune(self._h, _stream(stream)), "cddt_plan_autotune")
        return self.shape()

    def set_shape(self, tpp: int, ppi: int, block: int, regcap: int = 0):
        """cddt_plan_set_shape: lanes per particle, particles per item, block size, register cap."""
        _check(load().cddt_plan_set_shape(self._h, tpp, ppi, block, regcap), "cddt_plan_set_shape")

    def shape(self):
        """cddt_plan_get_shape as a dict."""
        a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().cddt_plan_get_shape(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
               "cddt_plan_get_shape")
        return {"tpp": a.value, "ppi": b.value, "block": c.value, "regcap": d.value}

    def run(self, stream=None):
        """cddt_plan_run: weight every filter of the plan in one persistent launch per key type."""
        _check(load().cddt_plan_run(self._h, _stream(stream)), "cddt_plan_run")

    def refine(self, steps: int, eta: float, tpp: int = 0, stream=None):
        """cddt_plan_refine: ``steps`` gradient pose refinement steps
        (x, y) += eta g / |g| of every particle, then a final evaluation, in
        one launch; writes each filter's ``logw``, ``grad_xy`` and
        ``particles_out``."""
        _check(load().cddt_plan_refine(self._h, int(steps), float(eta), int(tpp), _stream(stream)),
               "cddt_plan_refine")

    def launch_graph(self, stream=None):
        """cddt_plan_launch_graph: the same as a CUDA graph (captured on first use)."""
        _check(load().cddt_plan_launch_graph(self._h, _stream(stream)), "cddt_plan_launch_graph")

    @property
    def items(self) -> int:
        """cddt_plan_items: work items of the plan."""
        return load().cddt_plan_items(self._h)

    def groups(self):
        """Work items per launch: (f32 tree, f32 binary, u16 tree, u16 binary)."""
        import numpy as np
        out = np.zeros(4, np.int64)
        _check(load().cddt_plan_groups(self._h, out.ctypes.data_as(C.c_void_p)), "cddt_plan_groups")
        return tuple(int(v) for v in out)

    def close(self):
        """cddt_plan_destroy (idempotent)."""
        if getattr(self, "_h", None):
            load().cddt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
