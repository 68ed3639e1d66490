"""ctypes binding of the C-ABI in include/loc.h (argument marshalling only).

Host arrays are numpy arrays; every step of the filter runs in the CUDA library.  Errors
(negative loc_status) raise ``LocError`` with the library's message.  PyTorch is optional
plumbing: ``torch_stream()`` passes torch's current CUDA stream to ``loc_create`` and
``use_torch_allocator()`` makes the library take its device memory from torch's caching
allocator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "LOC_OK", "LOC_OK_DEFERRED", "LOC_WARN_REINIT", "LOC_ERR_INVALID_ARG", "LOC_ERR_OOM", "LOC_ERR_CUDA",
    "LOC_ERR_TIMEOUT", "LOC_ERR_STATE", "LOC_F32", "LOC_BF16", "LOC_F16", "LOC_MAP_SUM",
    "LOC_MAP_MAX", "LOC_KERNEL_AUTO", "LOC_KERNEL_GENERIC", "LOC_KERNEL_TILED", "LocError", "loc_params", "Handle", "library_path", "lib",
    "loc_params_default", "loc_set_allocator", "loc_create", "loc_step", "loc_lidar_update",
    "loc_lidar_update_cells", "loc_belief", "loc_marginal", "loc_argmax", "loc_set_belief",
    "loc_stats", "loc_sync", "loc_destroy", "loc_last_error", "torch_stream",
    "use_torch_allocator", "loc_propagate_noalloc", "loc_debug_fs_stall", "loc_samples", "loc_dither", "loc_ray_ranges",
    "loc_range_table", "loc_range_table_read", "loc_lidar_update_dense", "loc_estimate", "loc_map_difficulty",
    "loc_estimate_t",
    "LOC_BATCH_CONFIGS", "Batch", "loc_batch_create", "loc_batch_step", "loc_batch_sync",
    "loc_batch_info", "loc_batch_destroy", "loc_batch_last_error", "loc_session_bytes",
    "LOC_SESSION_PENDING", "LOC_SESSION_ACTIVE", "LOC_SESSION_CLOSED", "LOC_SESSION_FAILED",
    "loc_server_params", "loc_server_stats_t", "Server", "loc_server_params_default",
    "loc_server_create", "loc_server_open", "loc_server_close", "loc_server_odometry",
    "loc_server_scan", "loc_server_now", "loc_server_drain", "loc_server_stats",
    "loc_server_reset_stats", "loc_server_session", "loc_server_destroy", "loc_server_last_error",
]

LOC_OK, LOC_OK_DEFERRED, LOC_WARN_REINIT = 0, 1, 2
LOC_ERR_INVALID_ARG, LOC_ERR_OOM, LOC_ERR_CUDA, LOC_ERR_TIMEOUT, LOC_ERR_STATE = -1, -2, -3, -4, -5
LOC_F32, LOC_BF16, LOC_F16 = 0, 1, 2
LOC_MAP_SUM, LOC_MAP_MAX = 0, 1
LOC_KERNEL_AUTO, LOC_KERNEL_GENERIC, LOC_KERNEL_TILED = 0, 1, 2
LOC_BATCH_CONFIGS = 3
LOC_SESSION_PENDING, LOC_SESSION_ACTIVE, LOC_SESSION_CLOSED, LOC_SESSION_FAILED = 0, 1, 2, 3
_STORAGE = {"f32": LOC_F32, "bf16": LOC_BF16, "f16": LOC_F16}

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.environ.get("LOC_LIBRARY", os.path.join(_HERE, "libloc.so"))


class LocError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"loc status {status}: {msg}")
        self.status = status


class loc_params(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("K", ctypes.c_int),
                ("cell_m", ctypes.c_double), ("sigma_xy_cells", ctypes.c_double),
                ("sigma_theta_bins", ctypes.c_double), ("r_xy", ctypes.c_int),
                ("r_theta", ctypes.c_int), ("min_shift_cells", ctypes.c_double),
                ("storage", ctypes.c_int), ("n_samples", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("kernel", ctypes.c_int),
                ("tile", ctypes.c_int), ("sigma_cross_cells", ctypes.c_double)]


class loc_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("storage", ctypes.c_int),
                ("batching", ctypes.c_int), ("tile", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("n_streams", ctypes.c_int)]


class loc_server_stats_t(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_int), ("n_pending", ctypes.c_int), ("n_closed", ctypes.c_int),
                ("n_failed", ctypes.c_int), ("bytes_used", ctypes.c_double),
                ("bytes_budget", ctypes.c_double), ("n_ticks", ctypes.c_longlong),
                ("n_messages", ctypes.c_longlong), ("n_propagations", ctypes.c_longlong),
                ("n_scans", ctypes.c_longlong), ("cell_updates", ctypes.c_double),
                ("mean_batch", ctypes.c_double), ("step_p50_ms", ctypes.c_double),
                ("step_p99_ms", ctypes.c_double), ("step_max_ms", ctypes.c_double),
                ("scan_p50_ms", ctypes.c_double), ("scan_p99_ms", ctypes.c_double),
                ("scan_max_ms", ctypes.c_double), ("first_s", ctypes.c_double),
                ("last_s", ctypes.c_double), ("batch_device_ms", ctypes.c_double),
                ("batch_alg_bytes", ctypes.c_double), ("n_batches", ctypes.c_longlong),
                ("scan_device_ms", ctypes.c_double), ("n_scans_timed", ctypes.c_longlong),
                ("plain_device_ms", ctypes.c_double), ("plain_alg_bytes", ctypes.c_double),
                ("n_plain", ctypes.c_longlong), ("host_gather_ms", ctypes.c_double),
                ("host_batch_ms", ctypes.c_double), ("host_scan_ms", ctypes.c_double),
                ("host_plain_ms", ctypes.c_double)]


class loc_estimate_t(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("j", ctypes.c_int), ("i", ctypes.c_int),
                ("x", ctypes.c_double), ("y", ctypes.c_double), ("theta", ctypes.c_double),
                ("p", ctypes.c_double), ("mass_near", ctypes.c_double),
                ("second_j", ctypes.c_int), ("second_i", ctypes.c_int),
                ("second_p", ctypes.c_double), ("second_ratio", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "loc_params_default": (None, [ctypes.POINTER(loc_params)]),
    "loc_set_allocator": (None, [_ALLOC, _FREE, _P]),
    "loc_create": (ctypes.c_int, [_P, ctypes.POINTER(loc_params), ctypes.POINTER(_P)]),
    "loc_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "loc_lidar_update": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_double]),
    "loc_lidar_update_cells": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_double]),
    "loc_belief": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "loc_marginal": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.c_int]),
    "loc_argmax": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int)] * 3
                   + [ctypes.POINTER(ctypes.c_float)]),
    "loc_set_belief": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "loc_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong)]),
    "loc_sync": (ctypes.c_int, [_P]),
    "loc_destroy": (ctypes.c_int, [_P]),
    "loc_last_error": (ctypes.c_char_p, [_P]),
    "loc_debug_fs_stall": (ctypes.c_int, [ctypes.c_int, ctypes.c_double]),
    "loc_propagate_noalloc": (ctypes.c_int, [ctypes.POINTER(loc_params), _P, _P, _P, _P,
                                             ctypes.c_double, ctypes.c_double]),
    "loc_samples": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]),
    "loc_dither": (ctypes.c_int, [_P, _P, ctypes.c_float, _P, ctypes.POINTER(ctypes.c_int)]),
    "loc_ray_ranges": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_double, _P]),
    "loc_estimate": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(loc_estimate_t)]),
    "loc_map_difficulty": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int)]),
    "loc_range_table": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "loc_range_table_read": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "loc_lidar_update_dense": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_double]),
    "loc_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "loc_batch_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "loc_batch_sync": (ctypes.c_int, [_P]),
    "loc_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), _P]),
    "loc_batch_destroy": (ctypes.c_int, [_P]),
    "loc_batch_last_error": (ctypes.c_char_p, [_P]),
    "loc_session_bytes": (ctypes.c_int, [ctypes.POINTER(loc_params), ctypes.POINTER(ctypes.c_size_t)]),
    "loc_server_params_default": (None, [ctypes.POINTER(loc_server_params)]),
    "loc_server_create": (ctypes.c_int, [ctypes.POINTER(loc_server_params), ctypes.POINTER(_P)]),
    "loc_server_open": (ctypes.c_int, [_P, _P, ctypes.POINTER(loc_params), ctypes.POINTER(ctypes.c_int)]),
    "loc_server_close": (ctypes.c_int, [_P, ctypes.c_int]),
    "loc_server_odometry": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "loc_server_scan": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "loc_server_now": (ctypes.c_double, [_P]),
    "loc_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "loc_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(loc_server_stats_t)]),
    "loc_server_reset_stats": (ctypes.c_int, [_P]),
    "loc_server_session": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_P)]),
    "loc_server_destroy": (ctypes.c_int, [_P]),
    "loc_server_last_error": (ctypes.c_char_p, [_P]),
}


def lib():
    """The loaded CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
        _lib = L
    return _lib


class Handle:
    """A session handle plus the shape needed to size readback buffers."""

    def __init__(self, ptr: int, H: int, W: int, K: int):
        self.ptr, self.H, self.W, self.K = ptr, H, W, K

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def _check(h, status: int) -> int:
    if status < 0:
        if isinstance(h, Server) and h.ptr:
            msg = lib().loc_last_error(None)
            raise LocError(status, msg.decode() if msg else "")
        if isinstance(h, Batch) and h.ptr:
            msg = lib().loc_batch_last_error(h)
            raise LocError(status, msg.decode() if msg else "")
        ptr = h.ptr if isinstance(h, Handle) else None
        msg = lib().loc_last_error(ptr)
        raise LocError(status, msg.decode() if msg else "")
    return status


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def loc_params_default(**kw) -> loc_params:
    p = loc_params()
    lib().loc_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = _STORAGE[v]
        setattr(p, k, v)
    return p


_alloc_refs = []


def loc_set_allocator(alloc, free, ctx=None) -> None:
    """Register Python callables alloc(nbytes, stream) -> int and free(ptr, stream)."""
    if alloc is None:
        lib().loc_set_allocator(_ALLOC(0), _FREE(0), None)
        _alloc_refs.clear()
        return
    a = _ALLOC(lambda n, s, c: alloc(int(n), s or 0))
    f = _FREE(lambda p, s, c: free(p, s or 0))
    _alloc_refs[:] = [a, f]
    lib().loc_set_allocator(a, f, ctx)


def use_torch_allocator() -> None:
    """Take device memory from torch's caching allocator."""
    import torch
    loc_set_allocator(lambda n, s: torch.cuda.caching_allocator_alloc(n, stream=int(s)),
                      lambda p, s: torch.cuda.caching_allocator_delete(p))


def torch_stream() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def loc_create(occ: np.ndarray, params: loc_params) -> Handle:
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    if occ.shape != (params.H, params.W):
        raise ValueError(f"map shape {occ.shape} != ({params.H}, {params.W})")
    out = ctypes.c_void_p()
    _check(None, lib().loc_create(_ptr(occ), ctypes.byref(params), ctypes.byref(out)))
    return Handle(out.value, params.H, params.W, params.K)


def loc_step(h: Handle, u: float, v: float, w: float) -> int:
    return _check(h, lib().loc_step(h, float(u), float(v), float(w)))


def loc_lidar_update(h: Handle, ranges: np.ndarray, angle_min: float, angle_inc: float,
                     r_max: float, beam_stride: int, sigma_r: float) -> int:
    z = np.ascontiguousarray(ranges, dtype=np.float32)
    return _check(h, lib().loc_lidar_update(h, _ptr(z), int(z.size), float(angle_min),
                                            float(angle_inc), float(r_max), int(beam_stride),
                                            float(sigma_r)))


def loc_lidar_update_cells(h: Handle, cells: np.ndarray, ranges: np.ndarray, angle_min: float,
                           angle_inc: float, r_max: float, beam_stride: int,
                           sigma_r: float) -> int:
    c = np.ascontiguousarray(cells, dtype=np.int32)
    z = np.ascontiguousarray(ranges, dtype=np.float32)
    return _check(h, lib().loc_lidar_update_cells(h, _ptr(c), int(c.size), _ptr(z), int(z.size),
                                                  float(angle_min), float(angle_inc),
                                                  float(r_max), int(beam_stride), float(sigma_r)))


def loc_samples(h: Handle) -> np.ndarray:
    """Cells selected by the last loc_lidar_update (linear indices, raster order)."""
    n = ctypes.c_int()
    _check(h, lib().loc_samples(h, None, 0, ctypes.byref(n)))
    out = np.empty(max(n.value, 1), np.int32)
    _check(h, lib().loc_samples(h, _ptr(out), out.size, ctypes.byref(n)))
    return out[:n.value]


def loc_dither(h: Handle, m: np.ndarray, fs: float):
    """Floyd-Steinberg selection of the handle-shaped map m scaled by fs: (mask, count)."""
    m = np.ascontiguousarray(m, dtype=np.float32)
    if m.shape != (h.H, h.W):
        raise ValueError("map shape must match the handle")
    sel = np.empty((h.H, h.W), np.uint8)
    n = ctypes.c_int()
    _check(h, lib().loc_dither(h, _ptr(m), ctypes.c_float(fs), _ptr(sel), ctypes.byref(n)))
    return sel, n.value


def loc_ray_ranges(h: Handle, cells: np.ndarray, dirs: np.ndarray, r_max: float) -> np.ndarray:
    """Expected ranges (m) for each cell and FP32 unit direction: shape (n_cells, n_dirs)."""
    c = np.ascontiguousarray(cells, dtype=np.int32)
    d = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 2)
    out = np.empty((c.size, d.shape[0]), np.float32)
    _check(h, lib().loc_ray_ranges(h, _ptr(c), int(c.size), _ptr(d), int(d.shape[0]), float(r_max),
                                   _ptr(out)))
    return out


def loc_estimate(h: Handle, radius_m: float, dk: int) -> dict:
    """The pose estimate, the belief near it and the second hypothesis outside its disk."""
    e = loc_estimate_t()
    _check(h, lib().loc_estimate(h, float(radius_m), int(dk), ctypes.byref(e)))
    return {name: getattr(e, name) for name, _ in loc_estimate_t._fields_}


def loc_map_difficulty(h: Handle, probes: np.ndarray, probe_bin: int, beam_step: int, sigma_r: float,
                       c_m: float):
    """Eq. 11 on probe cells: (e_p per probe in metres, the number with e_p > c_m)."""
    p = np.ascontiguousarray(probes, dtype=np.int32)
    err = np.empty(max(p.size, 1), np.float64)
    n = ctypes.c_int()
    _check(h, lib().loc_map_difficulty(h, _ptr(p), int(p.size), int(probe_bin), int(beam_step), float(sigma_r),
                                       float(c_m), _ptr(err), ctypes.byref(n)))
    return err[:p.size], n.value


def loc_range_table(h: Handle, n_angles: int, r_max: float) -> None:
    """Build the session's expected-range table for the dense scan update."""
    _check(h, lib().loc_range_table(h, int(n_angles), float(r_max)))
    h.table_A = int(n_angles)


def loc_range_table_read(h: Handle) -> np.ndarray:
    """The table as uint8 [n_angles][H][W]."""
    A = getattr(h, "table_A", 0)
    out = np.empty((max(A, 1), h.H, h.W), np.uint8)
    _check(h, lib().loc_range_table_read(h, _ptr(out), A * h.H * h.W))
    return out


def loc_lidar_update_dense(h: Handle, ranges: np.ndarray, angle_min: float, angle_inc: float,
                           beam_stride: int, sigma_r: float) -> int:
    z = np.ascontiguousarray(ranges, dtype=np.float32)
    return _check(h, lib().loc_lidar_update_dense(h, _ptr(z), int(z.size), float(angle_min),
                                                  float(angle_inc), int(beam_stride), float(sigma_r)))


def loc_belief(h: Handle, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((h.K, h.H, h.W), np.float32)
    _check(h, lib().loc_belief(h, _ptr(out), out.size))
    return out


def loc_marginal(h: Handle, mode: int = LOC_MAP_MAX, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((h.H, h.W), np.float32)
    _check(h, lib().loc_marginal(h, _ptr(out), out.size, int(mode)))
    return out


def loc_argmax(h: Handle):
    k, j, i, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(h, lib().loc_argmax(h, ctypes.byref(k), ctypes.byref(j), ctypes.byref(i),
                               ctypes.byref(p)))
    return k.value, j.value, i.value, p.value


def loc_set_belief(h: Handle, b: np.ndarray) -> None:
    b = np.ascontiguousarray(b, dtype=np.float32)
    _check(h, lib().loc_set_belief(h, _ptr(b), b.size))


def loc_stats(h: Handle) -> dict:
    th, z, ls = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    npro, nre = ctypes.c_longlong(), ctypes.c_longlong()
    _check(h, lib().loc_stats(h, ctypes.byref(th), ctypes.byref(z), ctypes.byref(ls),
                              ctypes.byref(npro), ctypes.byref(nre)))
    return dict(theta=th.value, last_Z=z.value, logscale=ls.value, n_propagations=npro.value,
                n_reinit=nre.value)


def loc_sync(h: Handle) -> int:
    """Wait for the handle's work; LOC_OK, or LOC_WARN_REINIT once after new restarts."""
    return _check(h, lib().loc_sync(h))


def loc_destroy(h: Handle) -> None:
    if h is not None and h.ptr:
        lib().loc_destroy(h)
        h.ptr = None


def loc_last_error(h: Handle | None = None) -> str:
    m = lib().loc_last_error(h.ptr if h is not None else None)
    return m.decode() if m else ""


def loc_debug_fs_stall(stall: bool, wait_limit_s: float = 0.2) -> None:
    """Test hook: make the dithering's bounded block hand-offs wait on a flag nothing sets."""
    _check(None, lib().loc_debug_fs_stall(1 if stall else 0, float(wait_limit_s)))


def loc_propagate_noalloc(params: loc_params, occ_dev: int, b_in_dev: int, b_out_dev: int,
                          z_out_dev: int, dx_m: float, dy_m: float) -> None:
    """Allocation-free propagation on caller-owned device buffers (raw device pointers)."""
    _check(None, lib().loc_propagate_noalloc(ctypes.byref(params), ctypes.c_void_p(occ_dev),
                                             ctypes.c_void_p(b_in_dev), ctypes.c_void_p(b_out_dev),
                                             ctypes.c_void_p(z_out_dev), float(dx_m), float(dy_m)))


class Batch:
    """A batch of sessions stepped by one persistent launch per tick."""

    def __init__(self, ptr: int, handles):
        self.ptr, self.handles = ptr, list(handles)

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def loc_batch_create(handles, tile: int = 0, use_graph: bool = True) -> Batch:
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr for h in handles])
    out = ctypes.c_void_p()
    _check(None, lib().loc_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(handles), int(tile),
                                        int(bool(use_graph)), ctypes.byref(out)))
    return Batch(out.value, handles)


def loc_batch_step(b: Batch, u, v, w) -> int:
    """One tick; u, v, w hold one odometry increment per session.  Returns the number moved."""
    n = len(b.handles)
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), (n,))) for x in (u, v, w)]
    moved = ctypes.c_int()
    _check(b, lib().loc_batch_step(b, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), ctypes.byref(moved)))
    return moved.value


def loc_batch_sync(b: Batch) -> None:
    _check(b, lib().loc_batch_sync(b))


def loc_batch_info(b: Batch) -> dict:
    tile, items, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(LOC_BATCH_CONFIGS, np.float32)
    _check(b, lib().loc_batch_info(b, ctypes.byref(tile), ctypes.byref(items), ctypes.byref(grid), _ptr(ms)))
    return dict(tile=tile.value, n_items=items.value, grid=grid.value, tune_ms=ms.tolist())


def loc_batch_destroy(b: Batch) -> None:
    if b is not None and b.ptr:
        lib().loc_batch_destroy(b)
        b.ptr = None


def loc_batch_last_error(b: Batch | None) -> str:
    m = lib().loc_batch_last_error(b.ptr if b is not None else None)
    return m.decode() if m else ""


def loc_session_bytes(params: loc_params) -> int:
    out = ctypes.c_size_t()
    _check(None, lib().loc_session_bytes(ctypes.byref(params), ctypes.byref(out)))
    return out.value


class Server:
    """A serving loop (its worker and completion threads run inside the library)."""

    def __init__(self, ptr: int):
        self.ptr = ptr
        self.shapes = {}

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def loc_server_params_default(**kw) -> loc_server_params:
    p = loc_server_params()
    lib().loc_server_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = _STORAGE[v]
        setattr(p, k, v)
    return p


def loc_server_create(params: loc_server_params) -> Server:
    out = ctypes.c_void_p()
    _check(None, lib().loc_server_create(ctypes.byref(params), ctypes.byref(out)))
    return Server(out.value)


def loc_server_open(s: Server, occ: np.ndarray, params: loc_params) -> int:
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    if occ.shape != (params.H, params.W):
        raise ValueError(f"map shape {occ.shape} != ({params.H}, {params.W})")
    sid = ctypes.c_int()
    _check(s, lib().loc_server_open(s, _ptr(occ), ctypes.byref(params), ctypes.byref(sid)))
    s.shapes[sid.value] = (params.K, params.H, params.W)
    return sid.value


def loc_server_close(s: Server, sid: int) -> None:
    _check(s, lib().loc_server_close(s, int(sid)))


def loc_server_odometry(s: Server, ids, u, v, w, t_arrival=None) -> None:
    ids = np.ascontiguousarray(np.atleast_1d(ids), np.int32)
    n = ids.size
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), (n,))) for x in (u, v, w)]
    t = None if t_arrival is None else np.ascontiguousarray(np.broadcast_to(np.asarray(t_arrival, np.float64), (n,)))
    _check(s, lib().loc_server_odometry(s, n, _ptr(ids), _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                        None if t is None else _ptr(t)))


def loc_server_scan(s: Server, sid: int, ranges: np.ndarray, angle_min: float, angle_inc: float, r_max: float,
                    beam_stride: int, sigma_r: float, t_arrival: float = -1.0) -> None:
    r = np.ascontiguousarray(ranges, np.float32)
    _check(s, lib().loc_server_scan(s, int(sid), _ptr(r), r.size, float(angle_min), float(angle_inc),
                                    float(r_max), int(beam_stride), float(sigma_r), float(t_arrival)))


def loc_server_now(s: Server) -> float:
    return lib().loc_server_now(s)


def loc_server_drain(s: Server, timeout_s: float = 60.0) -> None:
    _check(s, lib().loc_server_drain(s, float(timeout_s)))


def loc_server_stats(s: Server) -> dict:
    st = loc_server_stats_t()
    _check(s, lib().loc_server_stats(s, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


def loc_server_reset_stats(s: Server) -> None:
    _check(s, lib().loc_server_reset_stats(s))


def loc_server_session(s: Server, sid: int):
    """(state, Handle or None); readbacks through the handle only after loc_server_drain."""
    state, h = ctypes.c_int(), ctypes.c_void_p()
    _check(s, lib().loc_server_session(s, int(sid), ctypes.byref(state), ctypes.byref(h)))
    if not h.value:
        return state.value, None
    K, H, W = s.shapes[sid]
    return state.value, Handle(h.value, H, W, K)


def loc_server_destroy(s: Server) -> None:
    if s is not None and s.ptr:
        lib().loc_server_destroy(s)
        s.ptr = None


def loc_server_last_error(s: Server | None) -> str:
    m = lib().loc_server_last_error(s.ptr if s is not None else None)
    return m.decode() if m else ""
