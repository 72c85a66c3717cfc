"""Thin ctypes binding of librmp.so (include/rmp.h): the same names as the C ABI, argument
marshalling only.  Device buffers are passed as torch CUDA tensors (their data_ptr) and
streams as torch.cuda.Stream objects (or raw cudaStream_t integers); every step of the
computation runs in the library's kernels.

Loading fails loudly (RuntimeError) when the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import importlib
import os
import struct
import threading
from typing import Optional

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None
_fast = None        # CPython marshalling of the synchronous calls (None: ctypes only)

RMP_OK, RMP_ERR_INVALID_ARG = 0, 1
STATUS_NAMES = {0: "RMP_OK", 1: "RMP_ERR_INVALID_ARG", 2: "RMP_ERR_NO_MEMORY", 3: "RMP_ERR_CUDA",
                4: "RMP_ERR_TIMEOUT", 5: "RMP_ERR_BUSY", 6: "RMP_ERR_UNKNOWN_MAP",
                7: "RMP_ERR_NOT_READY"}
STATUS_CODES = {v: k for k, v in STATUS_NAMES.items()}
RMP_RAY_HIT, RMP_RAY_MISS_RANGE, RMP_RAY_MISS_EXIT = 1, 2, 3
RMP_MAP_DENSE_U8, RMP_MAP_HASHED_TSDF = 0, 1
RMP_PRESET_STATIC_MAP, RMP_PRESET_LIDAR = 0, 1
RMP_REDUCE_KAHAN32, RMP_REDUCE_FP64 = 0, 1
RMP_TUNE_BLOCK, RMP_TUNE_LG_SEGMENTS, RMP_TUNE_RAY_ORDER, RMP_TUNE_SPLIT_BUDGET = 1, 2, 3, 4
RMP_TUNE_CELL_SKIP = 5


class RmpError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, STATUS_NAMES.get(status, "?"), status))
        self.status = status


class rmp_params_t(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eta_rep", "nu_rep", "eta_damp", "nu_damp", "r", "c",
                                          "eps", "max_range", "min_range")] + \
               [(n, C.c_uint32) for n in ("halton_offset", "w_mode", "reduce_mode", "flags")]


class rmp_result_t(C.Structure):
    _fields_ = [("f", C.c_double * 3), ("A", C.c_double * 6), ("Af", C.c_double * 3),
                ("eig", C.c_double * 3), ("n_rays", C.c_uint32), ("n_hits", C.c_uint32),
                ("n_active", C.c_uint32), ("rank", C.c_uint32), ("status", C.c_int32),
                ("reserved", C.c_uint32)]


class rmp_ray_hit_t(C.Structure):
    _fields_ = [("voxel", C.c_int32 * 3), ("steps", C.c_uint32), ("d", C.c_float),
                ("status", C.c_uint8), ("pad", C.c_uint8), ("blocks", C.c_uint16)]


class rmp_map_desc_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("data_on_device", C.c_int32), ("voxel_size", C.c_double),
                ("origin", C.c_double * 3), ("dims", C.c_int32 * 3), ("n_blocks", C.c_uint32),
                ("occ", C.c_void_p), ("block_keys", C.c_void_p), ("tsdf", C.c_void_p)]


class rmp_launch_info_t(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("block", "grid", "lg_segments", "ctas_per_sm", "sm_count",
                                         "smem_bytes", "ray_cells", "reserved")]


class rmp_rollout_params_t(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("dt", C.c_double),
                ("goal_tol", C.c_double), ("max_steps", C.c_uint32), ("seg_steps", C.c_uint32),
                ("n_rays", C.c_uint32), ("metric_mean", C.c_uint32)]


class rmp_rollout_result_t(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("xdot", C.c_double * 3), ("path_length", C.c_double),
                ("smoothness", C.c_double), ("status", C.c_uint32), ("steps", C.c_uint32),
                ("smooth_segments", C.c_uint32), ("reserved", C.c_uint32)]


RMP_ROLLOUT_RUNNING, RMP_ROLLOUT_REACHED, RMP_ROLLOUT_COLLIDED = 0, 1, 2
RMP_ROLLOUT_TIMEOUT, RMP_ROLLOUT_LEFT_MAP, RMP_ROLLOUT_FAILED = 3, 4, 5


class rmp_server_config_t(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("max_batch_states", C.c_uint32), ("max_rays", C.c_uint32),
                ("reserved", C.c_uint32), ("mem_budget_bytes", C.c_uint64)]


class rmp_server_stats_t(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "rejected", "batches",
                                          "batched_states", "pending", "max_inflight",
                                          "mem_high_water")]


class rmp_primitive_t(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("reserved", C.c_uint32), ("center", C.c_double * 3),
                ("size", C.c_double * 3)]


RMP_PRIM_SPHERE, RMP_PRIM_BOX = 0, 1


class rmp_map_info_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_bricks", C.c_uint32), ("hash_capacity", C.c_uint32),
                ("layout", C.c_uint32), ("device_bytes", C.c_uint64)]


assert C.sizeof(rmp_result_t) == 144 and C.sizeof(rmp_ray_hit_t) == 24

RESULT_BYTES = C.sizeof(rmp_result_t)
HIT_DTYPE = np.dtype([("voxel", "<i4", (3,)), ("steps", "<u4"), ("d", "<f4"),
                      ("status", "u1"), ("pad", "u1"), ("blocks", "<u2")])

_P = C.c_void_p
_SIGNATURES = {
    "rmp_ctx_create": [C.POINTER(C.c_void_p), C.c_int],
    "rmp_ctx_destroy": [_P],
    "rmp_params_preset": [C.c_int, C.POINTER(rmp_params_t)],
    "rmp_map_upload": [_P, C.POINTER(rmp_map_desc_t), _P, C.POINTER(C.c_uint32)],
    "rmp_map_release": [_P, C.c_uint32],
    "rmp_map_info": [_P, C.c_uint32, C.POINTER(rmp_map_info_t)],
    "rmp_map_cell_distances": [_P, C.c_uint32, _P, _P, _P, C.c_uint64],
    "rmp_workspace_init": [_P, C.c_size_t, _P],
    "rmp_raycast_eval": [_P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(rmp_params_t), _P,
                         C.POINTER(rmp_result_t), _P, _P],
    "rmp_raycast_eval_async": [_P, C.c_uint32, _P, C.c_uint32, C.POINTER(rmp_params_t), _P,
                               C.c_size_t, _P, _P, _P, _P],
    "rmp_scan_eval": [_P, _P, C.c_uint32, _P, _P, C.POINTER(rmp_params_t), _P,
                      C.POINTER(rmp_result_t), _P],
    "rmp_scan_eval_async": [_P, _P, C.c_uint32, _P, C.POINTER(rmp_params_t), _P, C.c_size_t, _P,
                            _P, _P],
    "rmp_tune_set": [_P, C.c_int, C.c_int],
    "rmp_eval_launch_info": [_P, C.c_uint32, C.c_uint32, C.POINTER(rmp_params_t),
                             C.POINTER(rmp_launch_info_t)],
    "rmp_tune_get": [_P, C.c_int, C.POINTER(C.c_int)],
    "rmp_raycast_eval_batch_async": [_P, C.c_uint32, _P, _P, C.c_uint32, C.c_uint32,
                                     C.POINTER(rmp_params_t), _P, C.c_size_t, _P, _P, _P, _P],
    "rmp_raycast_eval_batch": [_P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(rmp_params_t), _P,
                               _P],
    "rmp_combined_eval_batch_async": [_P, C.c_uint32, _P, _P, C.c_uint32, C.c_uint32,
                                      C.POINTER(rmp_params_t), _P, C.c_double, C.c_double,
                                      C.c_uint32, _P, C.c_size_t, _P, _P],
    "rmp_rollout": [_P, C.c_uint32, _P, C.c_uint32, C.POINTER(rmp_params_t),
                    C.POINTER(rmp_rollout_params_t), _P, _P],
    "rmp_raycast_eval_batch_static": [_P, C.c_uint32, _P, _P, C.c_uint32, C.c_uint32,
                                      C.POINTER(rmp_params_t), _P, _P],
    "rmp_scan_pipeline_create": [_P, C.c_uint32, C.c_uint32, C.POINTER(C.c_void_p)],
    "rmp_scan_pipeline_destroy": [_P],
    "rmp_scan_pipeline_submit": [_P, _P, C.c_uint32, _P, _P, C.POINTER(rmp_params_t),
                                 C.POINTER(C.c_uint64)],
    "rmp_scan_pipeline_wait": [_P, C.c_uint64, C.POINTER(rmp_result_t)],
    "rmp_server_config_default": [C.POINTER(rmp_server_config_t)],
    "rmp_server_create": [_P, C.POINTER(rmp_server_config_t), C.POINTER(C.c_void_p)],
    "rmp_server_destroy": [_P],
    "rmp_server_submit": [_P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(rmp_params_t),
                          C.POINTER(C.c_uint64)],
    "rmp_server_poll": [_P, C.c_uint64, C.POINTER(rmp_result_t), C.POINTER(C.c_double)],
    "rmp_server_wait": [_P, C.c_uint64, C.c_uint32, C.POINTER(rmp_result_t), C.POINTER(C.c_double)],
    "rmp_server_stats": [_P, C.POINTER(rmp_server_stats_t)],
    "rmp_batch_autotune": [_P, C.c_uint32, _P, _P, C.c_uint32, C.c_uint32, C.POINTER(rmp_params_t),
                           _P, C.c_size_t, _P, _P, C.c_int, _P, C.c_int],
    "rmp_probe_l2_read": [_P, _P, C.c_size_t, C.c_uint32, _P, _P],
    "rmp_esdf_upload": [_P, _P, C.c_uint32, C.POINTER(C.c_uint32)],
    "rmp_esdf_release": [_P, C.c_uint32],
    "rmp_esdf_eval_async": [_P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(rmp_params_t), C.c_double,
                            C.c_double, _P, _P, _P],
    "rmp_rollout_esdf": [_P, C.c_uint32, C.c_uint32, _P, C.c_uint32, C.POINTER(rmp_params_t),
                         C.POINTER(rmp_rollout_params_t), _P, _P],
}
# Symbols every build must export (checked by the not-gpu ABI test against include/rmp.h).
EXPORTS = sorted(list(_SIGNATURES) + ["rmp_status_string", "rmp_workspace_bytes",
                                       "rmp_batch_workspace_bytes"])


def lib_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load librmp.so (building it if the sources are newer).  Raises if unavailable."""
    global _lib, _fast
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                try:
                    _build.build()
                except Exception as e:  # no toolchain: fail loudly, never fall back
                    raise RuntimeError("librmp.so is missing or stale and could not be built: %s"
                                       % e) from e
            L = C.CDLL(path)
            for name, args in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.rmp_status_string.argtypes = [C.c_int]
            L.rmp_status_string.restype = C.c_char_p
            L.rmp_workspace_bytes.argtypes = []
            L.rmp_workspace_bytes.restype = C.c_size_t
            L.rmp_batch_workspace_bytes.argtypes = [C.c_uint32, C.c_uint32]
            L.rmp_batch_workspace_bytes.restype = C.c_size_t
            if os.path.exists(_build.FAST) and _build.fast_up_to_date():
                try:    # linked against the library just loaded (same file, one copy)
                    _fast = importlib.import_module(__package__ + "._rmp_fast")
                except ImportError:
                    _fast = None
            _lib = L
    return _lib


def fast_binding() -> bool:
    """True when the synchronous calls go through the CPython extension."""
    lib()
    return _fast is not None


def _check(status: int, what: str):
    if status != RMP_OK:
        raise RmpError(status, what)


_torch = None
_raw_stream = None      # torch's C accessors of the current stream and device, once found


def _current_stream() -> Optional[int]:
    """Handle of torch's current CUDA stream (None without a usable torch CUDA)."""
    global _torch, _raw_stream
    try:
        if _raw_stream is not None:         # the C accessors directly (no Python-level init check)
            return _raw_stream[0](_raw_stream[1]())
        if _torch is None:
            import torch
            _torch = torch
        raw = getattr(_torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(_torch._C, "_cuda_getDevice", None)
        if raw is not None:                 # one call instead of building a Stream object
            h = raw(_torch.cuda.current_device())     # initialises CUDA in torch if needed
            if dev is not None:
                _raw_stream = (raw, dev)
            return h
        return _torch.cuda.current_stream().cuda_stream
    except Exception:
        return None


def _stream(stream) -> Optional[int]:
    if stream is None:
        return _current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


_D3 = C.c_double * 3


def _vec3(v):
    if not (isinstance(v, np.ndarray) and v.shape == (3,)):
        v = np.asarray(v, np.float64).reshape(3)
    return _D3(*v.tolist())


def make_params(d: dict, max_range: float) -> rmp_params_t:
    p = rmp_params_t()
    for k in ("eta_rep", "nu_rep", "eta_damp", "nu_damp", "r", "c", "eps", "min_range"):
        setattr(p, k, float(d[k]))
    p.max_range = float(max_range)
    p.halton_offset = int(d.get("halton_offset", 1))
    p.w_mode = int(d.get("w_mode", 0))
    p.reduce_mode = int(d.get("reduce_mode", 0))
    p.flags = 0
    return p


def result_dict(r: rmp_result_t) -> dict:
    v = np.frombuffer(r, np.float64, 15)    # f (3), sum A (6), sum A f (3), eig (3): views
    return dict(f=v[0:3], sumA=v[3:9], sumAf=v[9:12], eig=v[12:15], n_rays=r.n_rays,
                n_hits=r.n_hits, n_active=r.n_active, rank=r.rank, status=r.status)


def result_from_bytes(b: bytes) -> dict:
    return result_dict(rmp_result_t.from_buffer_copy(b))


def _result_from_raw(b: bytes) -> dict:
    v = np.frombuffer(bytearray(b), np.float64, 15)   # f, sum A, sum A f, eig (writable)
    n_rays, n_hits, n_active, rank, status, _ = struct.unpack_from("<IIIIiI", b, 120)
    return dict(f=v[0:3], sumA=v[3:9], sumAf=v[9:12], eig=v[12:15], n_rays=n_rays,
                n_hits=n_hits, n_active=n_active, rank=rank, status=status)


# ----------------------------------------------------------------------------- C-named calls
def rmp_status_string(status: int) -> str:
    return lib().rmp_status_string(int(status)).decode()


def rmp_params_preset(preset: int) -> rmp_params_t:
    p = rmp_params_t()
    _check(lib().rmp_params_preset(int(preset), C.byref(p)), "rmp_params_preset")
    return p


def rmp_workspace_bytes() -> int:
    return int(lib().rmp_workspace_bytes())


def rmp_ctx_create(device: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().rmp_ctx_create(C.byref(h), int(device)), "rmp_ctx_create")
    return h.value


def rmp_ctx_destroy(ctx: int):
    _check(lib().rmp_ctx_destroy(ctx), "rmp_ctx_destroy")


def rmp_map_upload(ctx: int, desc: rmp_map_desc_t, stream=None) -> int:
    mid = C.c_uint32()
    _check(lib().rmp_map_upload(ctx, C.byref(desc), _stream(stream), C.byref(mid)), "rmp_map_upload")
    return int(mid.value)


def rmp_map_release(ctx: int, map_id: int):
    _check(lib().rmp_map_release(ctx, int(map_id)), "rmp_map_release")


def rmp_map_info(ctx: int, map_id: int) -> dict:
    info = rmp_map_info_t()
    _check(lib().rmp_map_info(ctx, int(map_id), C.byref(info)), "rmp_map_info")
    return dict(kind=info.kind, n_bricks=info.n_bricks, hash_capacity=info.hash_capacity,
                layout=info.layout, device_bytes=info.device_bytes)


def rmp_map_cell_distances(ctx: int, map_id: int):
    """(grid_min, grid_dim, cells): the grid's first block and bricks per axis (x, y, z),
    and the 4-bit cell free distances, 8 uint32 words per brick in brick order."""
    gmin = (C.c_int32 * 3)()
    gdim = (C.c_int32 * 3)()
    _check(lib().rmp_map_cell_distances(ctx, int(map_id), gmin, gdim, None, 0),
           "rmp_map_cell_distances")
    n = 8 * gdim[0] * gdim[1] * gdim[2]
    cells = np.zeros(n, np.uint32)
    _check(lib().rmp_map_cell_distances(ctx, int(map_id), gmin, gdim, cells.ctypes.data, n),
           "rmp_map_cell_distances")
    return np.array(gmin[:]), np.array(gdim[:]), cells


def rmp_workspace_init(workspace, stream=None):
    _check(lib().rmp_workspace_init(_dptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)), "rmp_workspace_init")


def rmp_raycast_eval(ctx: int, map_id: int, x, xdot, n_rays: int, params: rmp_params_t,
                     stream=None, hits=None, per_ray=None) -> dict:
    L = _lib if _lib is not None else lib()
    if _fast is not None:
        st, raw = _fast.raycast_eval(ctx, int(map_id), x, xdot, int(n_rays), C.addressof(params),
                                     _stream(stream), _dptr(hits), _dptr(per_ray))
        _check(st, "rmp_raycast_eval")
        return _result_from_raw(raw)
    out = rmp_result_t()
    _check(L.rmp_raycast_eval(ctx, int(map_id), _vec3(x), _vec3(xdot), int(n_rays),
                                  C.byref(params), _stream(stream), C.byref(out), _dptr(hits),
                                  _dptr(per_ray)), "rmp_raycast_eval")
    return result_dict(out)


def rmp_raycast_eval_async(ctx: int, map_id: int, state, n_rays: int, params: rmp_params_t,
                           workspace, out, stream=None, hits=None, per_ray=None):
    _check(lib().rmp_raycast_eval_async(ctx, int(map_id), _dptr(state), int(n_rays), C.byref(params),
                                        _dptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream), _dptr(out), _dptr(hits), _dptr(per_ray)),
           "rmp_raycast_eval_async")


def rmp_scan_eval(ctx: int, points, x, xdot, params: rmp_params_t, stream=None,
                  per_ray=None) -> dict:
    lib()
    n = points.shape[0]
    if _fast is not None:
        st, raw = _fast.scan_eval(ctx, _dptr(points), int(n), x, xdot, C.addressof(params),
                                  _stream(stream), _dptr(per_ray))
        _check(st, "rmp_scan_eval")
        return _result_from_raw(raw)
    out = rmp_result_t()
    _check(lib().rmp_scan_eval(ctx, _dptr(points), int(n), _vec3(x), _vec3(xdot), C.byref(params),
                               _stream(stream), C.byref(out), _dptr(per_ray)), "rmp_scan_eval")
    return result_dict(out)


def rmp_scan_eval_async(ctx: int, points, state, params: rmp_params_t, workspace, out,
                        stream=None, per_ray=None):
    n = points.shape[0]
    _check(lib().rmp_scan_eval_async(ctx, _dptr(points), int(n), _dptr(state), C.byref(params),
                                     _dptr(workspace), workspace.numel() * workspace.element_size(),
                                     _stream(stream), _dptr(out), _dptr(per_ray)),
           "rmp_scan_eval_async")


def rmp_batch_workspace_bytes(n_states: int, max_rays: int) -> int:
    return int(lib().rmp_batch_workspace_bytes(int(n_states), int(max_rays)))


def rmp_raycast_eval_batch_async(ctx: int, map_id: int, states, n_rays, n_states: int,
                                 max_rays: int, params: rmp_params_t, workspace, out, stream=None,
                                 hits=None, per_ray=None):
    """states: device float64 (n_states, 6); n_rays: device int32/uint32 (n_states,);
    out: device buffer of n_states results (RESULT_BYTES each)."""
    _check(lib().rmp_raycast_eval_batch_async(
        ctx, int(map_id), _dptr(states), _dptr(n_rays), int(n_states), int(max_rays),
        C.byref(params), _dptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream), _dptr(out), _dptr(hits), _dptr(per_ray)), "rmp_raycast_eval_batch_async")


def rmp_raycast_eval_batch_static(ctx: int, map_id: int, states, n_rays, n_states: int,
                                  max_rays: int, params: rmp_params_t, out, stream=None):
    """As rmp_raycast_eval_batch_async with the library's static device scratch (no
    workspace argument; batches up to 4 MiB of workspace)."""
    _check(lib().rmp_raycast_eval_batch_static(ctx, int(map_id), _dptr(states), _dptr(n_rays),
                                               int(n_states), int(max_rays), C.byref(params),
                                               _stream(stream), _dptr(out)),
           "rmp_raycast_eval_batch_static")


def rmp_combined_eval_batch_async(ctx: int, map_id: int, states, n_rays, n_states: int,
                                  max_rays: int, params: rmp_params_t, goals, alpha: float,
                                  beta: float, workspace, out, stream=None,
                                  metric_mean: bool = False):
    """Batched raycasting policy combined with per-state goal attractors (Eq. 1)."""
    _check(lib().rmp_combined_eval_batch_async(
        ctx, int(map_id), _dptr(states), _dptr(n_rays), int(n_states), int(max_rays),
        C.byref(params), _dptr(goals), float(alpha), float(beta), int(bool(metric_mean)),
        _dptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream), _dptr(out)),
        "rmp_combined_eval_batch_async")


def rollout_params(alpha, beta, dt, goal_tol, max_steps, seg_steps, n_rays,
                   metric_mean: bool = False) -> rmp_rollout_params_t:
    rp = rmp_rollout_params_t()
    rp.alpha, rp.beta, rp.dt, rp.goal_tol = float(alpha), float(beta), float(dt), float(goal_tol)
    rp.max_steps, rp.seg_steps, rp.n_rays = int(max_steps), int(seg_steps), int(n_rays)
    rp.metric_mean = int(bool(metric_mean))
    return rp


def rmp_rollout(ctx: int, map_id: int, robots, params: rmp_params_t, rp: rmp_rollout_params_t,
                stream=None) -> list:
    """robots: host (n, 9) float64 [start x, start xdot, goal]; returns one dict per robot."""
    rb = np.ascontiguousarray(robots, np.float64).reshape(-1, 9)
    out = (rmp_rollout_result_t * rb.shape[0])()
    _check(lib().rmp_rollout(ctx, int(map_id), rb.ctypes.data, int(rb.shape[0]), C.byref(params),
                             C.byref(rp), _stream(stream), out), "rmp_rollout")
    return [dict(x=np.array(r.x[:]), xdot=np.array(r.xdot[:]), path_length=r.path_length,
                 smoothness=r.smoothness, status=int(r.status), steps=int(r.steps),
                 smooth_n=int(r.smooth_segments)) for r in out]


def primitives(prims) -> "C.Array":
    """rmp_primitive_t records from objects with .kind ("sphere" / "box"), .center and .size
    (sphere: radius; box: half-extents)."""
    arr = (rmp_primitive_t * max(1, len(prims)))()
    for i, pr in enumerate(prims):
        arr[i].kind = RMP_PRIM_SPHERE if pr.kind == "sphere" else RMP_PRIM_BOX
        sz = np.asarray(pr.size, np.float64).reshape(-1)
        for a in range(3):
            arr[i].center[a] = float(pr.center[a])
            arr[i].size[a] = float(sz[a] if sz.size == 3 else sz[0])
    return arr


def rmp_probe_l2_read(ctx: int, buf, passes: int, checksum, stream=None):
    """L2 read-bandwidth probe over the device tensor buf (contiguous, bytes % 16 == 0);
    checksum: device uint64 tensor with at least SMs x 4 entries."""
    _check(lib().rmp_probe_l2_read(ctx, _dptr(buf), buf.numel() * buf.element_size(),
                                   int(passes), _stream(stream), _dptr(checksum)),
           "rmp_probe_l2_read")


def rmp_esdf_upload(ctx: int, prims) -> int:
    """Upload an ESDF of primitives (see primitives()); returns its id."""
    arr = primitives(prims)
    out = C.c_uint32(0)
    _check(lib().rmp_esdf_upload(ctx, C.cast(arr, C.c_void_p), len(prims), C.byref(out)),
           "rmp_esdf_upload")
    return out.value


def rmp_esdf_release(ctx: int, esdf_id: int):
    _check(lib().rmp_esdf_release(ctx, int(esdf_id)), "rmp_esdf_release")


def rmp_esdf_eval_async(ctx: int, esdf_id: int, states, goals, n_states: int,
                        params: rmp_params_t, alpha: float, beta: float, out, query=None,
                        stream=None):
    """ESDF policy (Sec. III-D) for n_states device states (n x 6 float64), with the attractor
    when goals (n x 3 float64, device) is given; out: n x RESULT_BYTES device bytes."""
    _check(lib().rmp_esdf_eval_async(ctx, int(esdf_id), _dptr(states), _dptr(goals),
                                     int(n_states), C.byref(params), float(alpha), float(beta),
                                     _stream(stream), _dptr(out), _dptr(query)),
           "rmp_esdf_eval_async")


def rmp_rollout_esdf(ctx: int, map_id: int, esdf_id: int, robots, params: rmp_params_t,
                     rp: rmp_rollout_params_t, stream=None) -> list:
    """As rmp_rollout with the ESDF policy (collisions from the voxel map)."""
    rb = np.ascontiguousarray(robots, np.float64).reshape(-1, 9)
    out = (rmp_rollout_result_t * rb.shape[0])()
    _check(lib().rmp_rollout_esdf(ctx, int(map_id), int(esdf_id), rb.ctypes.data,
                                  int(rb.shape[0]), C.byref(params), C.byref(rp),
                                  _stream(stream), out), "rmp_rollout_esdf")
    return [dict(x=np.array(r.x[:]), xdot=np.array(r.xdot[:]), path_length=r.path_length,
                 smoothness=r.smoothness, status=int(r.status), steps=int(r.steps),
                 smooth_n=int(r.smooth_segments)) for r in out]


def rmp_raycast_eval_batch(ctx: int, map_id: int, states, n_rays, params: rmp_params_t,
                           stream=None) -> list:
    """states: host (n_states, 6) float64 [x, xdot]; n_rays: host counts.  Returns one result
    dict per state."""
    st = np.ascontiguousarray(states, np.float64).reshape(-1, 6)
    nr = np.ascontiguousarray(n_rays, np.uint32).reshape(-1)
    assert st.shape[0] == nr.shape[0]
    out = (rmp_result_t * st.shape[0])()
    _check(lib().rmp_raycast_eval_batch(ctx, int(map_id), st.ctypes.data, nr.ctypes.data,
                                        int(st.shape[0]), C.byref(params), _stream(stream), out),
           "rmp_raycast_eval_batch")
    return [result_dict(r) for r in out]


def rmp_batch_autotune(ctx: int, map_id: int, states, n_rays, n_states: int, max_rays: int,
                       params: rmp_params_t, workspace, out, reps: int = 5, stream=None) -> list:
    """Runs the autotuner (leaves the fastest knobs in the context); returns the 9 median
    times in ms (block-major, then segments)."""
    times = (C.c_float * 9)()
    _check(lib().rmp_batch_autotune(
        ctx, int(map_id), _dptr(states), _dptr(n_rays), int(n_states), int(max_rays),
        C.byref(params), _dptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream), _dptr(out), int(reps), times, 9), "rmp_batch_autotune")
    return [float(t) for t in times]


def rmp_tune_set(ctx: int, knob: int, value: int):
    _check(lib().rmp_tune_set(ctx, int(knob), int(value)), "rmp_tune_set")


def rmp_eval_launch_info(ctx: int, map_id: int, n_rays: int, params: rmp_params_t) -> dict:
    info = rmp_launch_info_t()
    _check(lib().rmp_eval_launch_info(ctx, int(map_id), int(n_rays), C.byref(params), C.byref(info)),
           "rmp_eval_launch_info")
    return {n: getattr(info, n) for n, _ in rmp_launch_info_t._fields_ if n != "reserved"}


def rmp_tune_get(ctx: int, knob: int) -> int:
    v = C.c_int()
    _check(lib().rmp_tune_get(ctx, int(knob), C.byref(v)), "rmp_tune_get")
    return int(v.value)


# ----------------------------------------------------------------------------- map descriptors
def dense_desc(occ, voxel_size: float, origin) -> rmp_map_desc_t:
    """occ: uint8 array or CUDA tensor shaped (nz, ny, nx) (x fastest)."""
    d = rmp_map_desc_t()
    d.kind = RMP_MAP_DENSE_U8
    d.voxel_size = float(voxel_size)
    for a in range(3):
        d.origin[a] = float(origin[a])
    nz, ny, nx = occ.shape
    d.dims[0], d.dims[1], d.dims[2] = nx, ny, nz
    if isinstance(occ, np.ndarray):
        occ = np.ascontiguousarray(occ, np.uint8)
        d.data_on_device = 0
        d.occ = occ.ctypes.data
        d._keep = occ
    else:
        d.data_on_device = 1
        d.occ = _dptr(occ)
    return d


def hashed_desc(keys, tsdf, voxel_size: float) -> rmp_map_desc_t:
    """keys: (n, 3) int32, tsdf: (n, 512) float32 -- numpy (host) or CUDA tensors."""
    d = rmp_map_desc_t()
    d.kind = RMP_MAP_HASHED_TSDF
    d.voxel_size = float(voxel_size)
    d.n_blocks = int(keys.shape[0])
    if isinstance(keys, np.ndarray):
        keys = np.ascontiguousarray(keys, np.int32)
        tsdf = np.ascontiguousarray(tsdf, np.float32)
        d.data_on_device = 0
        d.block_keys = keys.ctypes.data if keys.size else None
        d.tsdf = tsdf.ctypes.data if tsdf.size else None
        d._keep = (keys, tsdf)
    else:
        d.data_on_device = 1
        d.block_keys = _dptr(keys)
        d.tsdf = _dptr(tsdf)
    return d


def rmp_server_config_default() -> rmp_server_config_t:
    cfg = rmp_server_config_t()
    _check(lib().rmp_server_config_default(C.byref(cfg)), "rmp_server_config_default")
    return cfg


def rmp_server_create(ctx: int, cfg: rmp_server_config_t) -> int:
    h = C.c_void_p()
    _check(lib().rmp_server_create(ctx, C.byref(cfg), C.byref(h)), "rmp_server_create")
    return h.value


def rmp_server_destroy(server: int):
    _check(lib().rmp_server_destroy(server), "rmp_server_destroy")


def rmp_server_submit(server: int, map_id: int, x, xdot, n_rays: int, params: rmp_params_t) -> int:
    t = C.c_uint64()
    _check(lib().rmp_server_submit(server, int(map_id), _vec3(x), _vec3(xdot), int(n_rays),
                                   C.byref(params), C.byref(t)), "rmp_server_submit")
    return int(t.value)


def rmp_server_poll(server: int, ticket: int):
    """(result dict, latency s) or None if not ready."""
    out = rmp_result_t()
    lat = C.c_double()
    st = lib().rmp_server_poll(server, int(ticket), C.byref(out), C.byref(lat))
    if st == 7:                               # RMP_ERR_NOT_READY
        return None
    _check(st, "rmp_server_poll")
    return result_dict(out), float(lat.value)


def rmp_server_wait(server: int, ticket: int, timeout_ms: int = 10000):
    out = rmp_result_t()
    lat = C.c_double()
    _check(lib().rmp_server_wait(server, int(ticket), int(timeout_ms), C.byref(out), C.byref(lat)),
           "rmp_server_wait")
    return result_dict(out), float(lat.value)


def rmp_server_stats(server: int) -> dict:
    st = rmp_server_stats_t()
    _check(lib().rmp_server_stats(server, C.byref(st)), "rmp_server_stats")
    return {n: int(getattr(st, n)) for n, _ in rmp_server_stats_t._fields_}


class ScanPipeline:
    """Owns one rmp_scan_pipeline: streamed LiDAR scans with copy/compute overlap.  Points
    are host arrays (float32 (n, 3)); pass pinned torch tensors for asynchronous copies and
    keep them unchanged until their result has been waited for."""

    def __init__(self, ctx: "Context", max_points: int, slots: int = 2):
        h = C.c_void_p()
        _check(lib().rmp_scan_pipeline_create(ctx.handle, int(max_points), int(slots),
                                              C.byref(h)), "rmp_scan_pipeline_create")
        self.handle = h.value

    def submit(self, points, x, xdot, params: rmp_params_t) -> int:
        t = C.c_uint64()
        if isinstance(points, np.ndarray):
            assert points.dtype == np.float32 and points.flags.c_contiguous
            ptr, n = points.ctypes.data, points.shape[0]
        else:
            ptr, n = points.data_ptr(), points.shape[0]
        _check(lib().rmp_scan_pipeline_submit(self.handle, ptr, int(n), _vec3(x), _vec3(xdot),
                                              C.byref(params), C.byref(t)),
               "rmp_scan_pipeline_submit")
        return int(t.value)

    def wait(self, ticket: int) -> dict:
        out = rmp_result_t()
        _check(lib().rmp_scan_pipeline_wait(self.handle, int(ticket), C.byref(out)),
               "rmp_scan_pipeline_wait")
        return result_dict(out)

    def close(self):
        if self.handle:
            _check(lib().rmp_scan_pipeline_destroy(self.handle), "rmp_scan_pipeline_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Owns one rmp_server (continuous-batching request server) of a Context."""

    def __init__(self, ctx: "Context", slots: int = 4, max_batch_states: int = 256,
                 max_rays: int = 262144, mem_budget_bytes: int = 1 << 30):
        cfg = rmp_server_config_default()
        cfg.slots, cfg.max_batch_states, cfg.max_rays = slots, max_batch_states, max_rays
        cfg.mem_budget_bytes = mem_budget_bytes
        self.handle = rmp_server_create(ctx.handle, cfg)

    def submit(self, map_id, x, xdot, n_rays, params) -> int:
        return rmp_server_submit(self.handle, map_id, x, xdot, n_rays, params)

    def poll(self, ticket):
        return rmp_server_poll(self.handle, ticket)

    def wait(self, ticket, timeout_ms: int = 10000):
        return rmp_server_wait(self.handle, ticket, timeout_ms)

    def stats(self) -> dict:
        return rmp_server_stats(self.handle)

    def close(self):
        if self.handle:
            rmp_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Context:
    """Owns one rmp_ctx; convenience wrapper over the C-named calls above."""

    def __init__(self, device: int = 0):
        self.handle = rmp_ctx_create(device)

    def close(self):
        if self.handle:
            rmp_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def upload(self, m, stream=None) -> int:
        """Upload a workloads.DenseMap / workloads.HashedMap."""
        if hasattr(m, "occ"):
            return rmp_map_upload(self.handle, dense_desc(m.occ, m.voxel_size, m.origin), stream)
        return rmp_map_upload(self.handle, hashed_desc(m.keys, m.tsdf, m.voxel_size), stream)
