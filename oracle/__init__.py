"""CPU oracle for raycast-RMP evaluation -- TEST INFRASTRUCTURE.

A ctypes wrapper around ``rmp_oracle.c``, the plain single-threaded C statement of the
method (Sec. III of arXiv 2301.08068).  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference legs may import this package; the library
in ``paper_2301_08068_gb300`` never does, and the two share no code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmp_oracle.c")
_SO = os.path.join(_HERE, "librmp_oracle.so")
_lock = threading.Lock()
_lib = None

HIT, MISS_RANGE, MISS_EXIT = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/librmp_oracle.so (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rmp_oracle.h"))):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eta_rep", "nu_rep", "eta_damp", "nu_damp", "r", "c",
                                          "eps", "max_range", "min_range")] + \
               [("halton_offset", C.c_uint32), ("w_mode", C.c_uint32)]


class Hit(C.Structure):
    _fields_ = [("voxel", C.c_int32 * 3), ("steps", C.c_uint32), ("d", C.c_float),
                ("status", C.c_uint8), ("pad", C.c_uint8), ("blocks", C.c_uint16)]


class Result(C.Structure):
    _fields_ = [("sumA", C.c_double * 6), ("sumAf", C.c_double * 3), ("f", C.c_double * 3),
                ("eig", C.c_double * 3), ("n_rays", C.c_uint32), ("n_hits", C.c_uint32),
                ("n_active", C.c_uint32), ("rank", C.c_uint32)]


class MapT(C.Structure):
    _fields_ = [("kind", C.c_int), ("voxel_size", C.c_double), ("origin", C.c_double * 3),
                ("dims", C.c_int32 * 3), ("occ", C.c_void_p), ("n_blocks", C.c_uint32),
                ("keys", C.c_void_p), ("tsdf", C.c_void_p), ("sorted", C.c_void_p)]


HIT_DTYPE = np.dtype([("voxel", "<i4", (3,)), ("steps", "<u4"), ("d", "<f4"),
                      ("status", "u1"), ("pad", "u1"), ("blocks", "<u2")])
assert HIT_DTYPE.itemsize == C.sizeof(Hit) == 24


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            sig = {
                "orc_halton2": (C.c_float, [C.c_uint32]),
                "orc_halton3": (C.c_float, [C.c_uint32]),
                "orc_halton3_numerator": (C.c_uint32, [C.c_uint32]),
                "orc_halton_batch": (None, [C.c_uint32, C.c_uint32, P, P, P]),
                "orc_sincos_batch": (None, [C.c_uint32, P, P, P]),
                "orc_ray_dirs": (None, [C.c_uint32, C.c_uint32, P]),
                "orc_quantize_dirs": (None, [C.c_uint32, P, P]),
                "orc_quantize_pos": (C.c_int64, [C.c_double, C.c_double, C.c_double]),
                "orc_range_fx": (C.c_int64, [C.c_double, C.c_double]),
                "orc_map_prepare": (C.c_int, [P]),
                "orc_map_free": (None, [P]),
                "orc_dda_batch": (C.c_int, [P, C.c_uint32, P, P, C.c_int64, P]),
                "orc_ray_policy": (None, [P, P, C.c_double, P, C.c_int, C.c_int, P, P]),
                "orc_active32": (C.c_int, [P, P]),
                "orc_pinv3": (None, [P, P, P, P]),
                "orc_raycast_eval": (C.c_int, [P, P, P, C.c_uint32, P, P, P, P]),
                "orc_scan_eval": (C.c_int, [P, C.c_uint32, P, P, P, P, P]),
                "orc_attractor": (None, [P, P, P, C.c_double, C.c_double, C.c_double, P]),
                "orc_combined_eval": (C.c_int, [P, P, P, C.c_uint32, P, P, C.c_double,
                                                C.c_double, C.c_int, P]),
                "orc_rollout_step": (None, [P, P, P, P, P]),
                "orc_esdf_query": (C.c_int, [P, C.c_uint32, P, P, P]),
                "orc_esdf_eval": (None, [P, C.c_uint32, P, P, P, P, C.c_double, C.c_double,
                                         P, P]),
                "orc_esdf_rollout_step": (None, [P, P, C.c_uint32, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class RolloutParams(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("dt", C.c_double),
                ("goal_tol", C.c_double), ("max_steps", C.c_uint32), ("seg_steps", C.c_uint32),
                ("n_rays", C.c_uint32), ("metric_mean", C.c_uint32)]


class RolloutState(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("xdot", C.c_double * 3), ("path_length", C.c_double),
                ("smooth_sum", C.c_double), ("seg_start", C.c_double * 3),
                ("prev_seg", C.c_double * 3), ("status", C.c_uint32), ("steps", C.c_uint32),
                ("smooth_n", C.c_uint32), ("have_prev", C.c_uint32)]


ROLL_RUNNING, ROLL_REACHED, ROLL_COLLIDED, ROLL_TIMEOUT, ROLL_LEFT_MAP = 0, 1, 2, 3, 4


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_params(d: dict, max_range: float) -> Params:
    p = Params()
    for k in ("eta_rep", "nu_rep", "eta_damp", "nu_damp", "r", "c", "eps", "min_range"):
        setattr(p, k, float(d[k]))
    p.max_range = float(max_range)
    p.halton_offset = int(d.get("halton_offset", 1))
    p.w_mode = int(d.get("w_mode", 0))
    return p


class OracleMap:
    """Oracle view of a workloads.DenseMap or workloads.HashedMap (keeps arrays alive)."""

    def __init__(self, m):
        self.m = MapT()
        self._keep = []
        self.m.voxel_size = float(m.voxel_size)
        if hasattr(m, "occ"):
            occ = np.ascontiguousarray(m.occ, np.uint8)
            self._keep.append(occ)
            self.m.kind = 0
            for a in range(3):
                self.m.origin[a] = float(m.origin[a])
                self.m.dims[a] = int(m.dims[a])
            self.m.occ = occ.ctypes.data
        else:
            keys = np.ascontiguousarray(m.keys, np.int32)
            tsdf = np.ascontiguousarray(m.tsdf, np.float32)
            self._keep += [keys, tsdf]
            self.m.kind = 1
            self.m.n_blocks = keys.shape[0]
            self.m.keys = keys.ctypes.data if keys.size else None
            self.m.tsdf = tsdf.ctypes.data if tsdf.size else None
        rc = lib().orc_map_prepare(C.byref(self.m))
        if rc != 0:
            raise ValueError("oracle map rejected (duplicate block keys?)")

    @property
    def ref(self):
        return C.byref(self.m)

    def __del__(self):
        try:
            lib().orc_map_free(C.byref(self.m))
        except Exception:
            pass


def halton(n: int, offset: int = 1):
    u = np.empty(n, np.float32)
    v = np.empty(n, np.float32)
    num = np.empty(n, np.uint32)
    lib().orc_halton_batch(n, offset, _ptr(u), _ptr(v), _ptr(num))
    return u, v, num


def sincos_turns(v: np.ndarray):
    v = np.ascontiguousarray(v, np.float32)
    c = np.empty_like(v)
    s = np.empty_like(v)
    lib().orc_sincos_batch(v.size, _ptr(v), _ptr(c), _ptr(s))
    return c, s


def ray_dirs(n: int, offset: int = 1) -> np.ndarray:
    out = np.empty((n, 3), np.float32)
    lib().orc_ray_dirs(n, offset, _ptr(out))
    return out


def quantize_dirs(dirs: np.ndarray) -> np.ndarray:
    dirs = np.ascontiguousarray(dirs, np.float32)
    D = np.empty(dirs.shape, np.int32)
    lib().orc_quantize_dirs(dirs.shape[0], _ptr(dirs), _ptr(D))
    return D


def quantize_pos(x, origin, vs) -> np.ndarray:
    return np.array([lib().orc_quantize_pos(float(x[a]), float(origin[a]), float(vs))
                     for a in range(3)], np.int64)


def range_fx(max_range: float, vs: float) -> int:
    return int(lib().orc_range_fx(float(max_range), float(vs)))


def dda(omap: OracleMap, P: np.ndarray, D: np.ndarray, R_fx: int) -> np.ndarray:
    """March rays (P (n,3) int64 fixed point, D (n,3) int32) -> hit records."""
    P = np.ascontiguousarray(np.broadcast_to(P, D.shape), np.int64)
    D = np.ascontiguousarray(D, np.int32)
    out = np.zeros(D.shape[0], HIT_DTYPE)
    lib().orc_dda_batch(omap.ref, D.shape[0], _ptr(P), _ptr(D), int(R_fx), _ptr(out))
    return out


def ray_policy(params: Params, r, d: float, xdot, active: bool, in_radius: bool):
    r = np.ascontiguousarray(r, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    f = np.zeros(3)
    A = np.zeros(6)
    lib().orc_ray_policy(C.byref(params), _ptr(r), float(d), _ptr(xd), int(active),
                         int(in_radius), _ptr(f), _ptr(A))
    return f, A


def active32(xdot, u) -> bool:
    xd = np.ascontiguousarray(xdot, np.float64)
    uu = np.ascontiguousarray(u, np.float32)
    return bool(lib().orc_active32(_ptr(xd), _ptr(uu)))


def pinv3(S6):
    S = np.ascontiguousarray(S6, np.float64)
    P = np.zeros(6)
    eig = np.zeros(3)
    rank = C.c_uint32(0)
    lib().orc_pinv3(_ptr(S), _ptr(P), _ptr(eig), C.byref(rank))
    return P, eig, int(rank.value)


def attractor(x, xdot, goal, alpha: float, beta: float, c: float) -> np.ndarray:
    """Attractor force f_a (Sec. III-B, Eq. attractorPolicy); its metric is I."""
    xx = np.ascontiguousarray(x, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    g = np.ascontiguousarray(goal, np.float64)
    fa = np.zeros(3)
    lib().orc_attractor(_ptr(xx), _ptr(xd), _ptr(g), float(alpha), float(beta), float(c), _ptr(fa))
    return fa


def combined_eval(omap: "OracleMap", x, xdot, n_rays: int, params: Params, goal, alpha: float,
                  beta: float, metric_mean: bool = False) -> dict:
    """Raycasting policy combined with the attractor by Eq. (1); sums include I and f_a
    (ray sums divided by the ray count first when metric_mean)."""
    xx = np.ascontiguousarray(x, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    g = np.ascontiguousarray(goal, np.float64)
    res = Result()
    lib().orc_combined_eval(omap.ref, _ptr(xx), _ptr(xd), int(n_rays), C.byref(params), _ptr(g),
                            float(alpha), float(beta), int(bool(metric_mean)), C.byref(res))
    return _result(res)


def rollout_params(alpha, beta, dt, goal_tol, max_steps, seg_steps, n_rays,
                   metric_mean: bool = False) -> RolloutParams:
    rp = RolloutParams()
    rp.alpha, rp.beta, rp.dt, rp.goal_tol = float(alpha), float(beta), float(dt), float(goal_tol)
    rp.max_steps, rp.seg_steps, rp.n_rays = int(max_steps), int(seg_steps), int(n_rays)
    rp.metric_mean = int(bool(metric_mean))
    return rp


def rollout_state(x0, xdot0) -> RolloutState:
    st = RolloutState()
    for a in range(3):
        st.x[a] = float(x0[a])
        st.xdot[a] = float(xdot0[a])
        st.seg_start[a] = float(x0[a])
    return st


def rollout_step(omap: "OracleMap", params: Params, rp: RolloutParams, goal, st: RolloutState):
    g = np.ascontiguousarray(goal, np.float64)
    lib().orc_rollout_step(omap.ref, C.byref(params), C.byref(rp), _ptr(g), C.byref(st))


def rollout(omap: "OracleMap", params: Params, rp: RolloutParams, x0, xdot0, goal,
            steps: Optional[int] = None, want_path: bool = False):
    """Closed-loop rollout until the robot stops running (or `steps` steps); returns the
    final state as a dict (and the positions after each step if want_path)."""
    st = rollout_state(x0, xdot0)
    path = []
    n = rp.max_steps if steps is None else steps
    for _ in range(n):
        if st.status != ROLL_RUNNING:
            break
        rollout_step(omap, params, rp, goal, st)
        if want_path:
            path.append(np.array(st.x[:]))
    out = dict(x=np.array(st.x[:]), xdot=np.array(st.xdot[:]), status=int(st.status),
               steps=int(st.steps), path_length=float(st.path_length),
               smoothness=float(st.smooth_sum / st.smooth_n) if st.smooth_n else 1.0,
               smooth_n=int(st.smooth_n))
    return (out, np.array(path)) if want_path else out


# ----------------------------------------------------------------------------- ESDF policy
PRIM_DTYPE = np.dtype([("kind", "<u4"), ("reserved", "<u4"), ("center", "<f8", (3,)),
                       ("size", "<f8", (3,))])
PRIM_SPHERE, PRIM_BOX = 0, 1


def prims_array(prims) -> np.ndarray:
    """Primitives (objects with .kind "sphere"/"box", .center, .size) as the oracle's records
    (sphere: size[0] = radius; box: half-extents)."""
    a = np.zeros(len(prims), PRIM_DTYPE)
    for i, pr in enumerate(prims):
        a[i]["kind"] = PRIM_SPHERE if pr.kind == "sphere" else PRIM_BOX
        a[i]["center"] = pr.center
        sz = np.asarray(pr.size, np.float64)
        a[i]["size"] = np.repeat(sz, 3) if sz.size == 1 else sz
    return a


def esdf_query(prims: np.ndarray, x):
    """(d, gradient, index of the minimising primitive) of the exact ESDF of prims at x."""
    xx = np.ascontiguousarray(x, np.float64)
    d = C.c_double(0.0)
    g = np.zeros(3)
    i = lib().orc_esdf_query(_ptr(prims) if len(prims) else None, len(prims), _ptr(xx),
                             C.byref(d), _ptr(g))
    return float(d.value), g, int(i)


def esdf_eval(prims: np.ndarray, x, xdot, params: Params, goal=None, alpha: float = 0.0,
              beta: float = 0.0):
    """The ESDF policy (Sec. III-D), with the attractor by Eq. (1) when a goal is given;
    returns the result dict and the query (d, gradient) as 4 doubles."""
    xx = np.ascontiguousarray(x, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    g = None if goal is None else np.ascontiguousarray(goal, np.float64)
    res = Result()
    q = np.zeros(4)
    lib().orc_esdf_eval(_ptr(prims) if len(prims) else None, len(prims), _ptr(xx), _ptr(xd),
                        C.byref(params), None if g is None else _ptr(g), float(alpha),
                        float(beta), C.byref(res), _ptr(q))
    return _result(res), q


def esdf_rollout(omap: "OracleMap", prims: np.ndarray, params: Params, rp: RolloutParams, x0,
                 xdot0, goal, steps: Optional[int] = None):
    """Closed-loop rollout with the ESDF policy (collisions from the voxel map)."""
    st = rollout_state(x0, xdot0)
    g = np.ascontiguousarray(goal, np.float64)
    n = rp.max_steps if steps is None else steps
    for _ in range(n):
        if st.status != ROLL_RUNNING:
            break
        lib().orc_esdf_rollout_step(omap.ref, _ptr(prims) if len(prims) else None, len(prims),
                                    C.byref(params), C.byref(rp), _ptr(g), C.byref(st))
    return dict(x=np.array(st.x[:]), xdot=np.array(st.xdot[:]), status=int(st.status),
                steps=int(st.steps), path_length=float(st.path_length),
                smoothness=float(st.smooth_sum / st.smooth_n) if st.smooth_n else 1.0,
                smooth_n=int(st.smooth_n))


def _result(res: Result) -> dict:
    return dict(sumA=np.array(res.sumA[:]), sumAf=np.array(res.sumAf[:]), f=np.array(res.f[:]),
                eig=np.array(res.eig[:]), n_rays=res.n_rays, n_hits=res.n_hits,
                n_active=res.n_active, rank=res.rank)


def raycast_eval(omap: OracleMap, x, xdot, n_rays: int, params: Params,
                 want_hits: bool = True, want_per_ray: bool = True):
    x = np.ascontiguousarray(x, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    res = Result()
    hits = np.zeros(n_rays, HIT_DTYPE) if want_hits else None
    per = np.zeros((n_rays, 9)) if want_per_ray else None
    lib().orc_raycast_eval(omap.ref, _ptr(x), _ptr(xd), int(n_rays), C.byref(params),
                           C.byref(res), _ptr(hits) if want_hits else None,
                           _ptr(per) if want_per_ray else None)
    return _result(res), hits, per


def scan_eval(points: np.ndarray, x, xdot, params: Params, want_per_ray: bool = True):
    pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    x = np.ascontiguousarray(x, np.float64)
    xd = np.ascontiguousarray(xdot, np.float64)
    res = Result()
    per = np.zeros((pts.shape[0], 9)) if want_per_ray else None
    lib().orc_scan_eval(_ptr(pts), pts.shape[0], _ptr(x), _ptr(xd), C.byref(params),
                        C.byref(res), _ptr(per) if want_per_ray else None)
    return _result(res), per
