"""Seeded synthetic inputs for raycast-RMP evaluation.

This module is the one place both the CUDA path and the CPU oracle take their inputs
from.  It holds none of the method's arithmetic (no Halton directions, no ray
marching, no policy, no reduction): only random numbers, scene primitives, voxel maps
computed from those primitives, robot states, LiDAR-like scans and the parameter
tables of the paper.

Workloads (all seeded, all synthetic; they stand in for the paper's random maps of
Sec. IV-A and its LiDAR scans of Sec. IV-B):

* ``dense_scene``: a dense uint8 occupancy grid of axis-aligned boxes (a voxel is
  occupied iff its centre lies inside a box).
* ``hashed_scene``: boxes and spheres merged by union (minimum of the primitives'
  exact signed distances), stored voxblox-style as blocks of 8^3 float32 TSDF values
  truncated at 0.3 m; a block exists iff one of its voxels lies within the truncation
  band or inside an obstacle.
* ``lidar_scan``: a 64-beam x 1024-column scan ray-cast analytically (FP64) against a
  primitive scene, with N(0, 0.02 m) range noise; beams without a return within 30 m
  give NaN points.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with one stream per workload; normal
deviates use the Box-Muller transform in FP64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

SEED_BASE = 0x230108068

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Table I of the paper: tuning of the obstacle policy for the static-map and LiDAR
# experiments.  eps is not given in the paper (Sec. III-C only says 0 < eps << 1);
# 1e-3 is this project's reading.  min_range is the small-range exclusion of
# Sec. V-B (no value given; 0.2 m is this project's reading).
PARAMS_STATIC_MAP = dict(eta_rep=88.0, nu_rep=1.4, eta_damp=140.0, nu_damp=1.2,
                         r=2.4, c=0.2, eps=1e-3, min_range=0.0,
                         halton_offset=1, w_mode=0, reduce_mode=0)
PARAMS_LIDAR = dict(eta_rep=1.2, nu_rep=1.5, eta_damp=3.0, nu_damp=1.0,
                    r=1.3, c=1.0, eps=1e-3, min_range=0.2,
                    halton_offset=1, w_mode=0, reduce_mode=0)
# Attractor gains of Table I (used only by the attractor combination, Eq. 3).
ATTRACTOR_STATIC_MAP = dict(alpha=10.0, beta=15.0)
ATTRACTOR_LIDAR = dict(alpha=0.8, beta=1.6)

TSDF_TRUNCATION = 0.3
BLOCK = 8


class SplitMix64:
    """SplitMix64 stream; ``uniform``/``normal`` draw vectors in FP64."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + k * _GOLDEN
            if n:
                self.state = z[-1]
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0,1]
        z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
        return sigma * z[:n]

    def integers(self, n: int, hi: int) -> np.ndarray:
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)


# --------------------------------------------------------------------------- scenes
@dataclasses.dataclass
class Primitive:
    kind: str            # "box" (half-extents) or "sphere" (radius)
    center: np.ndarray   # (3,) FP64
    size: np.ndarray     # box: (3,) half-extents; sphere: (1,) radius

    def sdf(self, p: np.ndarray) -> np.ndarray:
        """Exact Euclidean signed distance at points p (..., 3), FP64."""
        q = p - self.center
        if self.kind == "sphere":
            return np.linalg.norm(q, axis=-1) - self.size[0]
        q = np.abs(q) - self.size
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
        inside = np.minimum(np.max(q, axis=-1), 0.0)
        return outside + inside

    def extent(self) -> np.ndarray:
        return self.size if self.kind == "box" else np.repeat(self.size, 3)

    def ray_entry(self, o: np.ndarray, u: np.ndarray) -> np.ndarray:
        """First parameter t >= 0 where rays o + t u (u unit, (n,3)) enter the solid;
        +inf where they miss.  Origins are outside every primitive."""
        if self.kind == "sphere":
            oc = o - self.center
            b = np.einsum("ij,ij->i", oc, u)
            c = np.einsum("ij,ij->i", oc, oc) - self.size[0] ** 2
            disc = b * b - c
            t = -b - np.sqrt(np.maximum(disc, 0.0))
            return np.where((disc >= 0) & (t >= 0), t, np.inf)
        lo = self.center - self.size
        hi = self.center + self.size
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / u
            t1 = (lo - o) * inv
            t2 = (hi - o) * inv
        tmin = np.where(np.isnan(t1), -np.inf, np.minimum(t1, t2))
        tmax = np.where(np.isnan(t1), np.inf, np.maximum(t1, t2))
        # axis-parallel rays outside the slab never enter
        par = (u == 0)
        outside_slab = par & ((o < lo) | (o > hi))
        tmin = np.where(par, -np.inf, tmin)
        tmax = np.where(par, np.inf, tmax)
        tn = tmin.max(axis=1)
        tf = tmax.min(axis=1)
        hit = (tn <= tf) & (tf >= 0) & ~outside_slab.any(axis=1)
        return np.where(hit, np.maximum(tn, 0.0), np.inf)


def scene_sdf(prims: List[Primitive], p: np.ndarray) -> np.ndarray:
    """Union of primitives: minimum of their signed distances (FP64)."""
    out = np.full(p.shape[:-1], np.inf)
    for pr in prims:
        out = np.minimum(out, pr.sdf(p))
    return out


def random_boxes(rng: SplitMix64, n: int, lo: np.ndarray, hi: np.ndarray,
                 edge_lo: float, edge_hi: float) -> List[Primitive]:
    c = np.stack([rng.uniform(n, lo[a], hi[a]) for a in range(3)], axis=1)
    e = rng.uniform(3 * n, edge_lo, edge_hi).reshape(n, 3)
    return [Primitive("box", c[i], 0.5 * e[i]) for i in range(n)]


def random_mixed(rng: SplitMix64, n: int, lo: np.ndarray, hi: np.ndarray,
                 size_lo: float, size_hi: float) -> List[Primitive]:
    """Half spheres (radius U[size_lo, size_hi]), half boxes (half-edges U[...])."""
    c = np.stack([rng.uniform(n, lo[a], hi[a]) for a in range(3)], axis=1)
    kinds = rng.uniform(n) < 0.5
    sz = rng.uniform(3 * n, size_lo, size_hi).reshape(n, 3)
    prims = []
    for i in range(n):
        if kinds[i]:
            prims.append(Primitive("sphere", c[i], sz[i, :1].copy()))
        else:
            prims.append(Primitive("box", c[i], sz[i].copy()))
    return prims


# --------------------------------------------------------------------------- maps
@dataclasses.dataclass
class DenseMap:
    occ: np.ndarray          # uint8, shape (nz, ny, nx): x fastest in memory
    voxel_size: float
    origin: np.ndarray       # (3,) FP64, world position of voxel (0,0,0)'s low corner

    @property
    def dims(self) -> Tuple[int, int, int]:
        nz, ny, nx = self.occ.shape
        return (nx, ny, nz)


@dataclasses.dataclass
class HashedMap:
    keys: np.ndarray         # int32 (n, 3): block coordinates (bx, by, bz)
    tsdf: np.ndarray         # float32 (n, 512): voxel lx + 8 ly + 64 lz of each block
    voxel_size: float        # world-anchored: voxel k covers [k vs, (k+1) vs)

    @property
    def n_blocks(self) -> int:
        return int(self.keys.shape[0])


def voxelise_boxes_dense(prims: List[Primitive], dims, vs: float,
                         origin=(0.0, 0.0, 0.0)) -> DenseMap:
    nx, ny, nz = dims
    origin = np.asarray(origin, np.float64)
    occ = np.zeros((nz, ny, nx), np.uint8)
    for pr in prims:
        lo = pr.center - pr.extent()
        hi = pr.center + pr.extent()
        k0 = np.maximum(np.floor((lo - origin) / vs - 0.5).astype(int), 0)
        k1 = np.minimum(np.ceil((hi - origin) / vs - 0.5).astype(int), [nx - 1, ny - 1, nz - 1])
        if np.any(k1 < k0):
            continue
        zs, ys, xs = [origin[a] + (np.arange(k0[a], k1[a] + 1) + 0.5) * vs for a in (2, 1, 0)]
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        inside = pr.sdf(np.stack([X, Y, Z], axis=-1)) < 0.0
        occ[k0[2]:k1[2] + 1, k0[1]:k1[1] + 1, k0[0]:k1[0] + 1] |= inside.astype(np.uint8)
    return DenseMap(occ, vs, origin)


def tsdf_blocks(prims: List[Primitive], extent, vs: float,
                trunc: float = TSDF_TRUNCATION) -> HashedMap:
    """Voxelise the union of primitives into 8^3 TSDF blocks over [0, extent)."""
    nvox = [int(round(e / vs)) for e in extent]
    nb = [-(-n // BLOCK) for n in nvox]
    NX, NY, NZ = [b * BLOCK for b in nb]
    sdf = np.full((NZ, NY, NX), trunc, np.float32)
    for pr in prims:
        ext = pr.extent() + trunc
        k0 = np.maximum(np.floor((pr.center - ext) / vs).astype(int), 0)
        k1 = np.minimum(np.ceil((pr.center + ext) / vs).astype(int), [NX - 1, NY - 1, NZ - 1])
        if np.any(k1 < k0):
            continue
        zs, ys, xs = [(np.arange(k0[a], k1[a] + 1) + 0.5) * vs for a in (2, 1, 0)]
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        d = pr.sdf(np.stack([X, Y, Z], axis=-1)).astype(np.float32)
        sub = sdf[k0[2]:k1[2] + 1, k0[1]:k1[1] + 1, k0[0]:k1[0] + 1]
        np.minimum(sub, d, out=sub)
    alloc_vox = sdf < np.float32(trunc)
    np.clip(sdf, -trunc, trunc, out=sdf)
    bz, by, bx = nb[2], nb[1], nb[0]
    blocks = sdf.reshape(bz, BLOCK, by, BLOCK, bx, BLOCK).transpose(0, 2, 4, 1, 3, 5)
    alloc = alloc_vox.reshape(bz, BLOCK, by, BLOCK, bx, BLOCK).any(axis=(1, 3, 5))
    iz, iy, ix = np.nonzero(alloc)
    keys = np.stack([ix, iy, iz], axis=1).astype(np.int32)
    tsdf = np.ascontiguousarray(blocks[iz, iy, ix].reshape(-1, BLOCK ** 3), np.float32)
    return HashedMap(keys, tsdf, vs)


def free_points(rng: SplitMix64, prims: List[Primitive], lo, hi, n: int,
                clearance: float) -> np.ndarray:
    """n uniform points in [lo, hi) whose scene SDF exceeds ``clearance``."""
    out = []
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    while len(out) < n:
        m = max(64, 2 * (n - len(out)))
        p = np.stack([rng.uniform(m, lo[a], hi[a]) for a in range(3)], axis=1)
        ok = scene_sdf(prims, p) > clearance
        out.extend(p[ok][: n - len(out)])
    return np.asarray(out, np.float64)


# --------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class State:
    x: np.ndarray      # (3,) FP64 position (world frame)
    xdot: np.ndarray   # (3,) FP64 velocity


@dataclasses.dataclass
class DenseWorkload:
    map: DenseMap
    states: List[State]
    n_rays: int
    max_range: float
    params: dict


@dataclasses.dataclass
class HashedWorkload:
    map: HashedMap
    prims: List[Primitive]
    extent: Tuple[float, float, float]
    states: List[State]
    n_rays: List[int]
    max_range: float
    params: dict


@dataclasses.dataclass
class ScanWorkload:
    points: np.ndarray  # float32 (n, 3), sensor frame; NaN rows = no return
    x: np.ndarray       # sensor position in the points' frame (zeros)
    xdot: np.ndarray
    sensor_world: np.ndarray
    max_range: float
    params: dict


def dense_box_workload(n_states: int = 1, n_rays: int = 1024, jitter: bool = False,
                       dims=(64, 64, 64), vs: float = 0.1, n_boxes: int = 20,
                       max_range: float = 5.0, seed_index: int = 0) -> DenseWorkload:
    """Dense uint8 grid, 64^3 at 0.1 m, 20 boxes with edges U[0.2, 1.5] m; robots at
    centres of random free voxels (optionally jittered by +-0.25 voxel); velocity
    N(0, 1 m/s) per axis; 1024 rays; max range 5 m; Table I static-map parameters."""
    rng = SplitMix64(SEED_BASE + seed_index)
    ext = np.asarray(dims, np.float64) * vs
    prims = random_boxes(rng, n_boxes, np.zeros(3), ext, 0.2, 1.5)
    m = voxelise_boxes_dense(prims, dims, vs)
    free = np.argwhere(m.occ == 0)              # (z, y, x)
    states = []
    pick = rng.integers(n_states, len(free))
    jit = rng.uniform(3 * n_states, -0.25, 0.25).reshape(n_states, 3)
    vel = rng.normal(3 * n_states).reshape(n_states, 3)
    for s in range(n_states):
        z, y, x = free[pick[s]]
        p = m.origin + (np.array([x, y, z], np.float64) + 0.5) * vs
        if jitter:
            p = p + jit[s] * vs
        states.append(State(p, vel[s].copy()))
    return DenseWorkload(m, states, n_rays, max_range, dict(PARAMS_STATIC_MAP))


_HASHED_CACHE = {}


def hashed_scene(extent=(40.0, 40.0, 10.0), vs: float = 0.1, n_prims: int = 200,
                 size_range=(0.2, 2.0), seed_index: int = 1):
    """Hashed TSDF scene: n_prims boxes/spheres, union, truncation 0.3 m."""
    key = (tuple(extent), vs, n_prims, tuple(size_range), seed_index)
    if key not in _HASHED_CACHE:
        rng = SplitMix64(SEED_BASE + seed_index)
        prims = random_mixed(rng, n_prims, np.zeros(3), np.asarray(extent, np.float64),
                             *size_range)
        hm = tsdf_blocks(prims, extent, vs)
        _HASHED_CACHE[key] = (hm, prims)
    return _HASHED_CACHE[key]


def hashed_workload(n_states: int = 1, n_rays: int = 65536, max_range: float = 10.0,
                    extent=(40.0, 40.0, 10.0), vs: float = 0.1, n_prims: int = 200,
                    seed_index: int = 1, state_seed_index: Optional[int] = None,
                    uneven_rays: Optional[Tuple[int, int]] = None) -> HashedWorkload:
    """Hashed TSDF, 8^3 blocks, 0.1 m over 40x40x10 m, 200 primitives (radius or
    half-edge U[0.2, 2] m), robot at uniform free points (SDF > 0.3 m), velocity
    N(0, 1) per axis, 65536 rays, max range 10 m.  ``uneven_rays=(lo, hi)`` draws
    per-state ray counts log-uniform in [lo, hi]."""
    hm, prims = hashed_scene(extent, vs, n_prims, seed_index=seed_index)
    rng = SplitMix64(SEED_BASE + (seed_index if state_seed_index is None else state_seed_index)
                     + 0x1000)
    pts = free_points(rng, prims, np.zeros(3), np.asarray(extent), n_states, TSDF_TRUNCATION)
    vel = rng.normal(3 * n_states).reshape(n_states, 3)
    states = [State(pts[i], vel[i].copy()) for i in range(n_states)]
    if uneven_rays is None:
        rays = [int(n_rays)] * n_states
    else:
        lo, hi = uneven_rays
        u = rng.uniform(n_states, math.log(lo), math.log(hi))
        rays = [int(round(math.exp(v))) for v in u]
    return HashedWorkload(hm, prims, tuple(extent), states, rays, max_range,
                          dict(PARAMS_STATIC_MAP))


def lidar_directions(beams: int = 64, columns: int = 1024,
                     fov_deg: float = 45.0) -> np.ndarray:
    """Beam directions (beams*columns, 3) FP64: elevations evenly spread over
    [-fov/2, +fov/2], azimuth 2 pi k / columns; beam-major order."""
    el = np.deg2rad(np.linspace(-fov_deg / 2, fov_deg / 2, beams))
    az = 2 * np.pi * np.arange(columns) / columns
    E, Az = np.meshgrid(el, az, indexing="ij")
    u = np.stack([np.cos(E) * np.cos(Az), np.cos(E) * np.sin(Az), np.sin(E)], axis=-1)
    return u.reshape(-1, 3)


def lidar_workload(beams: int = 64, columns: int = 1024, max_return: float = 30.0,
                   noise: float = 0.02, seed_index: int = 2,
                   fov_deg: float = 45.0) -> ScanWorkload:
    """A 64 x 1024 scan of the hashed scene's primitives from a free sensor position,
    analytic first-hit ranges (FP64) plus N(0, 0.02 m); no return within 30 m -> NaN.
    (OS-0 sizing: 128 beams x 2048 columns over a 90 degree vertical field of view.)"""
    hm, prims = hashed_scene()
    rng = SplitMix64(SEED_BASE + seed_index)
    sensor = free_points(rng, prims, np.zeros(3), np.array([40.0, 40.0, 10.0]), 1,
                         TSDF_TRUNCATION)[0]
    u = lidar_directions(beams, columns, fov_deg)
    o = np.broadcast_to(sensor, u.shape)
    t = np.full(u.shape[0], np.inf)
    for pr in prims:
        t = np.minimum(t, pr.ray_entry(o, u))
    rng_noise = rng.normal(u.shape[0], noise)
    ret = t <= max_return
    rngs = np.where(ret, np.where(ret, t, 0.0) + rng_noise, np.nan)
    pts = (u * rngs[:, None]).astype(np.float32)
    xdot = rng.normal(3)
    return ScanWorkload(pts, np.zeros(3), xdot, sensor, max_return, dict(PARAMS_LIDAR))


def sphere_shell_scan(n: int, radius: float, seed_index: int = 7) -> np.ndarray:
    """n float32 points on a sphere of the given radius around the origin, directions
    uniform on the sphere (seeded): a LiDAR view from the centre of a hollow sphere."""
    rng = SplitMix64(SEED_BASE + seed_index)
    g = rng.normal(3 * n).reshape(n, 3)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * radius).astype(np.float32)


def served_workloads(n_states: int = 64):
    """The three resident maps of the served stream, max range 10 m: dense 128^3 at 0.05 m
    with 40 boxes; the hashed 40x40x10 m map at 0.1 m; hashed 100x100x20 m at 0.2 m with
    2500 primitives (the 40x40x10 m density scaled by volume)."""
    return [dense_box_workload(n_states=n_states, dims=(128, 128, 128), vs=0.05, n_boxes=40,
                               max_range=10.0, seed_index=6),
            hashed_workload(n_states=n_states, state_seed_index=7),
            hashed_workload(n_states=n_states, extent=(100.0, 100.0, 20.0), vs=0.2,
                            n_prims=2500, seed_index=5, state_seed_index=8)]


def poisson_requests(n_maps: int, rate: float, duration: float, ray_lo: int, ray_hi: int,
                     seed_index: int = 4):
    """Poisson arrival times (s), map index (uniform) and log-uniform ray counts."""
    rng = SplitMix64(SEED_BASE + seed_index)
    n_est = int(rate * duration * 1.2 + 100)
    gaps = -np.log1p(-rng.uniform(n_est)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    n = len(t)
    maps = rng.integers(n, n_maps)
    rays = np.rint(np.exp(rng.uniform(n, math.log(ray_lo), math.log(ray_hi)))).astype(np.int64)
    vel = rng.normal(3 * n).reshape(n, 3)
    return t, maps, rays, vel


@dataclasses.dataclass
class RolloutTasks:
    map: HashedMap
    prims: List[Primitive]
    starts: np.ndarray   # (n, 3)
    goals: np.ndarray    # (n, 3)
    max_range: float
    params: dict


def rollout_tasks(n_pairs: int, n_prims: int = 100, extent=(10.0, 10.0, 10.0), vs: float = 0.1,
                  max_range: float = 10.0, size_range=(0.2, 2.0),
                  seed_index: int = 9) -> RolloutTasks:
    """Start/goal pairs across a random map shaped like the paper's planning maps (Sec. IV-A:
    seeded spheres and boxes in a 10 m cube; radius / half-edge uniform in size_range):
    starts uniform in the slab x in [0.5, 1.5] m, goals in x in [8.5, 9.5] m, y and z in
    [0.5, 9.5] m, both at least 0.3 m from every obstacle (SDF > 0.3)."""
    hm, prims = hashed_scene(tuple(extent), vs, n_prims, size_range=tuple(size_range),
                             seed_index=seed_index)
    rng = SplitMix64(SEED_BASE + seed_index + 0x2000)
    e = np.asarray(extent, np.float64)
    starts = free_points(rng, prims, [0.5, 0.5, 0.5], [1.5, e[1] - 0.5, e[2] - 0.5], n_pairs,
                         TSDF_TRUNCATION)
    goals = free_points(rng, prims, [e[0] - 1.5, 0.5, 0.5], [e[0] - 0.5, e[1] - 0.5, e[2] - 0.5],
                        n_pairs, TSDF_TRUNCATION)
    return RolloutTasks(hm, prims, starts, goals, max_range, dict(PARAMS_STATIC_MAP))


def sphere_lattice_scan(n: int, radius: float) -> np.ndarray:
    """n float32 points of a spherical Fibonacci lattice of the given radius around the
    origin (z_k = 1 - (2k+1)/n, azimuth 2 pi k / golden ratio): an evenly spread view
    from the centre of a hollow sphere."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    phi = 2.0 * np.pi * k * (2.0 / (1.0 + math.sqrt(5.0)))
    s = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    p = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1) * radius
    return p.astype(np.float32)
