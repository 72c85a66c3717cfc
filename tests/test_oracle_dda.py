"""Pins for the oracle's raycast R(x, r) (Sec. III-E/III-F): the exact fixed-point DDA.

The DDA is checked against (a) hand-computed voxel sequences, including the tie rule
(x before y before z) on designed ties, (b) brute force: every voxel of a tiny scene is
tested with exact integer/rational slab intersection and the first occupied one by
entry parameter must be the DDA's hit, and (c) the analytic ray-box entry distance.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from paper_2301_08068_gb300 import workloads as W

FX = 1 << 16
DIRQ = 1 << 24


def dense_map(occ_xyz: np.ndarray, vs=0.1, origin=(0.0, 0.0, 0.0)):
    """occ_xyz indexed [x, y, z] -> workloads.DenseMap (stored z, y, x)."""
    return W.DenseMap(np.ascontiguousarray(np.transpose(occ_xyz, (2, 1, 0)).astype(np.uint8)),
                      vs, np.asarray(origin, np.float64))


def center_fx(k):
    return np.array([ki * FX + FX // 2 for ki in k], np.int64)


def march(orc, m, P, D, R_fx):
    om = orc.OracleMap(m)
    return orc.dda(om, np.asarray(P, np.int64).reshape(1, 3), np.asarray(D, np.int32).reshape(1, 3),
                   R_fx)[0]


# ----------------------------------------------------------------------------- hand cases
@pytest.mark.parametrize("axis,sign", list(itertools.product(range(3), (1, -1))))
def test_axis_aligned(orc, axis, sign):
    occ = np.zeros((9, 9, 9), np.uint8)
    hit = [4, 4, 4]
    hit[axis] = 4 + 3 * sign
    occ[tuple(hit)] = 1
    D = [0, 0, 0]
    D[axis] = sign * DIRQ
    h = march(orc, dense_map(occ), center_fx([4, 4, 4]), D, 100 * FX)
    assert h["status"] == orc.HIT
    assert list(h["voxel"]) == hit
    assert h["steps"] == 3
    assert h["d"] == np.float32(np.float32(2.5) * np.float32(0.1))   # 2.5 voxels


def test_start_voxel_occupied(orc):
    occ = np.zeros((4, 4, 4), np.uint8)
    occ[1, 2, 3] = 1
    h = march(orc, dense_map(occ), center_fx([1, 2, 3]), [DIRQ, 0, 0], 10 * FX)
    assert (h["status"], h["steps"], h["d"]) == (orc.HIT, 0, 0.0)


def test_diagonal_tie_steps_x_before_y(orc):
    occ = np.zeros((8, 8, 8), np.uint8)
    occ[2, 1, 0] = 1     # reached at step 3 if x steps first at each tie
    occ[1, 2, 0] = 1     # reached at step 3 if y stepped first
    c = 1 << 23
    h = march(orc, dense_map(occ), center_fx([0, 0, 0]), [c, c, 0], 100 * FX)
    assert list(h["voxel"]) == [2, 1, 0] and h["steps"] == 3


def test_triple_tie_order_xyz(orc):
    occ = np.zeros((8, 8, 8), np.uint8)
    occ[1, 1, 0] = occ[1, 0, 1] = occ[0, 1, 1] = 1
    c = 9_000_000
    h = march(orc, dense_map(occ), center_fx([0, 0, 0]), [c, c, c], 100 * FX)
    assert list(h["voxel"]) == [1, 1, 0] and h["steps"] == 2


def test_negative_diagonal_tie(orc):
    occ = np.zeros((8, 8, 8), np.uint8)
    occ[3, 4, 0] = occ[4, 3, 0] = 1
    c = 1 << 23
    h = march(orc, dense_map(occ), center_fx([5, 5, 0]), [-c, -c, 0], 100 * FX)
    # (5,5)->(4,5)->(4,4)->(3,4)
    assert list(h["voxel"]) == [3, 4, 0] and h["steps"] == 3


def test_start_on_boundary_moving_down(orc):
    occ = np.zeros((8, 8, 8), np.uint8)
    occ[2, 4, 4] = 1
    P = np.array([3 * FX, 4 * FX + 100, 4 * FX + 100], np.int64)   # exactly on x = 3
    h = march(orc, dense_map(occ), P, [-DIRQ, 0, 0], 100 * FX)
    assert list(h["voxel"]) == [2, 4, 4] and h["steps"] == 1 and h["d"] == 0.0


def test_range_limit_inclusive(orc):
    occ = np.zeros((12, 3, 3), np.uint8)
    occ[6, 1, 1] = 1
    P = np.array([FX * 1 + FX // 2, FX + FX // 2, FX + FX // 2], np.int64)
    # obstacle entered at 4.5 voxels; a range of exactly 4.5 voxels still reaches it
    h = march(orc, dense_map(occ), P, [DIRQ, 0, 0], 4 * FX + FX // 2)
    assert h["status"] == orc.HIT and list(h["voxel"]) == [6, 1, 1]
    h = march(orc, dense_map(occ), P, [DIRQ, 0, 0], 4 * FX + FX // 2 - 1)
    assert h["status"] == orc.MISS_RANGE and list(h["voxel"]) == [5, 1, 1] and h["steps"] == 4


def test_empty_maps_all_miss(orc):
    occ = np.zeros((16, 16, 16), np.uint8)
    m = dense_map(occ)
    d = orc.ray_dirs(512, 1)
    D = orc.quantize_dirs(d)
    hs = orc.dda(orc.OracleMap(m), center_fx([8, 8, 8]), D, 100 * FX)
    assert np.all(hs["status"] == orc.MISS_EXIT)
    assert np.all(np.abs(hs["voxel"] - 8).sum(axis=1) == hs["steps"])
    hm = W.HashedMap(np.zeros((0, 3), np.int32), np.zeros((0, 512), np.float32), 0.1)
    hs = orc.dda(orc.OracleMap(hm), center_fx([0, 0, 0]), D, 30 * FX)
    assert np.all(hs["status"] == orc.MISS_RANGE)


def test_start_outside_dense_grid(orc):
    occ = np.ones((4, 4, 4), np.uint8)
    h = march(orc, dense_map(occ), center_fx([-1, 0, 0]), [DIRQ, 0, 0], 10 * FX)
    assert (h["status"], h["steps"]) == (orc.MISS_EXIT, 0)


# ----------------------------------------------------------------------------- brute force
def slab(k, P, D):
    """Parameter interval [lo, hi) in which the ray P + t D lies in slab k (exact)."""
    lo_b, hi_b = k * FX, (k + 1) * FX
    if D == 0:
        return (Fraction(-10 ** 30), Fraction(10 ** 30)) if lo_b <= P < hi_b else None
    a, b = Fraction(lo_b - P, D), Fraction(hi_b - P, D)
    return (min(a, b), max(a, b))


def brute(occupied, inside, P, D, R_fx):
    """Expected (status, voxel, steps, exact entry parameter, distinct 8^3 blocks tested)
    by exhaustive search.
    Returns None if the ray has a tie (two axes cross at the same parameter)."""
    tmax = Fraction(R_fx, DIRQ)
    # tie detection: boundary crossings of different axes at the same parameter
    events = {}
    for a in range(3):
        if D[a] == 0:
            continue
        k0 = P[a] // FX
        ks = range(k0 - 40, k0 + 41)
        for k in ks:
            t = Fraction(k * FX - P[a], D[a])
            if 0 <= t <= tmax:
                if t in events and events[t] != a:
                    return None
                events[t] = a
    ranges = []
    for a in range(3):
        end = P[a] + tmax * D[a]
        lo = min(P[a], end) // FX - 1
        hi = max(P[a], end) // FX + 1
        ranges.append(range(int(lo), int(hi) + 1))
    cands = []
    for k in itertools.product(*ranges):
        iv = [slab(k[a], P[a], D[a]) for a in range(3)]
        if any(v is None for v in iv):
            continue
        lo = max(v[0] for v in iv)
        hi = min(v[1] for v in iv)
        if lo < hi and hi > 0 and lo <= tmax:
            cands.append((max(lo, Fraction(0)) if lo < 0 else lo, k))
    cands.sort()
    start = tuple(int(P[a] // FX) for a in range(3))
    assert cands[0][1] == start
    l1 = lambda k: sum(abs(k[a] - start[a]) for a in range(3))
    blk = lambda k: tuple(x // 8 for x in k)
    if not inside(start):
        return ("exit", start, 0, Fraction(0), 0)
    tested = {blk(start)}
    if occupied(start):
        return ("hit", start, 0, Fraction(0), 1)
    prev = (start, Fraction(0))
    for t, k in cands[1:]:
        if not inside(k):
            return ("exit", k, l1(k), t, len(tested))
        tested.add(blk(k))
        if occupied(k):
            return ("hit", k, l1(k), t, len(tested))
        prev = (k, t)
    k, t = prev
    return ("range", k, l1(k), t, len(tested))


STATUS = {"hit": 1, "range": 2, "exit": 3}


def check_against_brute(orc, m, occupied, inside, P, Ds, R_fx, vs):
    hs = orc.dda(orc.OracleMap(m), np.asarray(P, np.int64), np.asarray(Ds, np.int32), R_fx)
    checked = 0
    assert np.mean(hs["steps"]) >= 2.0          # the rays really travel
    for D, h in zip(Ds, hs):
        exp = brute(occupied, inside, [int(p) for p in P], [int(x) for x in D], R_fx)
        if exp is None:
            continue
        st, k, steps, t, blocks = exp
        assert h["status"] == STATUS[st], (P, D, exp, h)
        assert tuple(h["voxel"]) == k, (P, D, exp, h)
        assert h["steps"] == steps
        assert h["blocks"] == blocks
        d_exact = float(t * 256 * Fraction(float(np.float32(vs))))
        assert abs(float(h["d"]) - d_exact) <= 4 * np.spacing(np.float32(max(d_exact, 1e-30))), (h, d_exact)
        checked += 1
    return checked


def test_brute_force_dense_small_directions(orc):
    rng = np.random.default_rng(11)
    occ = (rng.random((12, 12, 12)) < 0.06).astype(np.uint8)
    m = dense_map(occ)
    occupied = lambda k: bool(occ[k])
    inside = lambda k: all(0 <= k[a] < 12 for a in range(3))
    total = 0
    for trial in range(6):
        P = [int(x) for x in rng.integers(2 * FX, 10 * FX, 3)]
        while occupied(tuple(p // FX for p in P)):
            P = [int(x) for x in rng.integers(2 * FX, 10 * FX, 3)]
        Ds = rng.integers(-DIRQ, DIRQ + 1, (40, 3)).astype(np.int32)
        Ds[:4, 0] = 0                       # axis-parallel components too
        Ds[4:6, 1:] = 0
        total += check_against_brute(orc, m, occupied, inside, P, Ds, 5 * FX, 0.1)
    assert total >= 200


def test_brute_force_dense_halton_directions(orc):
    rng = np.random.default_rng(12)
    occ = (rng.random((14, 14, 14)) < 0.05).astype(np.uint8)
    m = dense_map(occ)
    occupied = lambda k: bool(occ[k])
    inside = lambda k: all(0 <= k[a] < 14 for a in range(3))
    Ds = orc.quantize_dirs(orc.ray_dirs(96, 1))
    P = [int(x) for x in rng.integers(5 * FX, 9 * FX, 3)]
    while occupied(tuple(p // FX for p in P)):
        P = [int(x) for x in rng.integers(5 * FX, 9 * FX, 3)]
    assert check_against_brute(orc, m, occupied, inside, P, Ds, 6 * FX, 0.1) >= 90


def test_brute_force_hashed_negative_blocks(orc):
    """Blocks on both sides of the origin: floor division of voxel and block keys."""
    rng = np.random.default_rng(13)
    keys, tsdf = [], []
    for bz in (-1, 0):
        for by in (-1, 0):
            for bx in (-1, 0):
                if (bx, by, bz) == (0, -1, 0):
                    continue                          # one unallocated block
                keys.append((bx, by, bz))
                t = rng.uniform(-0.3, 0.3, 512).astype(np.float32)
                t[t > -0.25] = np.abs(t[t > -0.25]) + 0.01    # ~8% occupied
                tsdf.append(t)
    hm = W.HashedMap(np.array(keys, np.int32), np.array(tsdf, np.float32), 0.05)
    kset = {k: i for i, k in enumerate(keys)}

    def occupied(k):
        b = tuple(x // 8 for x in k)
        if b not in kset:
            return False
        lx, ly, lz = [x - 8 * bb for x, bb in zip(k, b)]
        return bool(hm.tsdf[kset[b], lx + 8 * ly + 64 * lz] <= 0)

    inside = lambda k: True
    total = 0
    for trial in range(4):
        P = [int(x) for x in rng.integers(-3 * FX, 3 * FX, 3)]
        while occupied(tuple(p // FX for p in P)):
            P = [int(x) for x in rng.integers(-3 * FX, 3 * FX, 3)]
        Ds = rng.integers(-DIRQ, DIRQ + 1, (40, 3)).astype(np.int32)
        total += check_against_brute(orc, hm, occupied, inside, P, Ds, 6 * FX, 0.05)
    assert total >= 120


def test_steps_equal_l1_distance(orc):
    wl = W.dense_box_workload(n_states=4, jitter=True)
    om = orc.OracleMap(wl.map)
    D = orc.quantize_dirs(orc.ray_dirs(1024, 1))
    for s in wl.states:
        P = orc.quantize_pos(s.x, wl.map.origin, wl.map.voxel_size)
        hs = orc.dda(om, P, D, orc.range_fx(wl.max_range, wl.map.voxel_size))
        start = P // FX
        assert np.all(np.abs(hs["voxel"] - start).sum(axis=1) == hs["steps"])


def test_voxel_aligned_box_entry_distance(orc):
    """Rays hitting a voxel-aligned box: the reported d equals the analytic slab entry
    distance of the box within the fixed-point quantisation of x and r."""
    vs = 0.1
    occ = np.zeros((32, 32, 32), np.uint8)
    lo_k, hi_k = np.array([10, 12, 8]), np.array([14, 16, 20])
    occ[10:15, 12:17, 8:21] = 1
    m = dense_map(occ, vs)
    x = np.array([0.537, 1.911, 1.402])
    dirs = orc.ray_dirs(4096, 1)
    D = orc.quantize_dirs(dirs)
    P = orc.quantize_pos(x, np.zeros(3), vs)
    hs = orc.dda(orc.OracleMap(m), P, D, orc.range_fx(3.2, vs))
    hit = hs["status"] == orc.HIT
    assert hit.sum() > 50
    u = dirs[hit].astype(np.float64)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    lo, hi = lo_k * vs, (hi_k + 1) * vs
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (lo - x) / u, (hi - x) / u
    t_in = np.nanmax(np.where(u == 0, -np.inf, np.minimum(t1, t2)), axis=1)
    d = hs["d"][hit].astype(np.float64)
    tol = np.sqrt(3) * vs * 2.0 ** -16 + t_in * 2.0 ** -21
    assert np.all(np.abs(d - t_in) <= tol)
    assert np.all((hs["voxel"][hit] >= lo_k).all(axis=1) & (hs["voxel"][hit] <= hi_k).all(axis=1))
