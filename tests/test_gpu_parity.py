"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Hit records are compared bit for bit; floats within the tolerances stated in
gpu_helpers.  Sizes span several CTAs with ragged tails, and the full configurations
(dense 64^3 x 1024 rays; hashed 40x40x10 m x 65536 rays; 64 x 1024 LiDAR scan) run whole.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import (assert_hits_exact, assert_per_ray_close, assert_result_close,
                         gpu_raycast, gpu_scan, scan_abs_term, torch_cuda)

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = R.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def dense(ctx):
    wl = W.dense_box_workload(n_states=8, jitter=True)
    return wl, ctx.upload(wl.map), O.OracleMap(wl.map)


@pytest.fixture(scope="module")
def hashed(ctx):
    wl = W.hashed_workload(n_states=6)
    return wl, ctx.upload(wl.map), O.OracleMap(wl.map)


def check_raycast(ctx, mid, om, x, xdot, n, pdict, max_range):
    pg = R.make_params(pdict, max_range)
    po = O.make_params(pdict, max_range)
    rg, hg, pgr = gpu_raycast(ctx, mid, x, xdot, n, pg)
    ro, ho, por = O.raycast_eval(om, x, xdot, n, po)
    assert_hits_exact(hg, ho)
    assert_per_ray_close(pgr, por)
    assert_result_close(rg, ro, por)
    return rg, ro


# ----------------------------------------------------------------------------- dense map
def test_dense_box_map_full_config(ctx):
    wl = W.dense_box_workload()
    mid = ctx.upload(wl.map)
    s = wl.states[0]
    rg, ro = check_raycast(ctx, mid, O.OracleMap(wl.map), s.x, s.xdot, wl.n_rays, wl.params,
                           wl.max_range)
    assert ro["n_hits"] > 0 and ro["n_active"] > 0


def test_dense_jittered_states(ctx, dense):
    wl, mid, om = dense
    for s in wl.states:
        check_raycast(ctx, mid, om, s.x, s.xdot, 1024, wl.params, wl.max_range)


@pytest.mark.parametrize("n", [1, 31, 129, 1000, 4097, 20000])
def test_dense_ragged_ray_counts(ctx, dense, n):
    wl, mid, om = dense
    s = wl.states[n % len(wl.states)]
    check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)


def test_dense_ray_count_sweep_paper_range(ctx, dense):
    """Sec. IV-A varies the ray count from 4^2 to 256^2."""
    wl, mid, om = dense
    s = wl.states[1]
    for n in (16, 64, 256, 1024, 4096, 16384, 65536):
        check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)


def test_dense_robot_outside_grid_all_exit(ctx, dense):
    wl, mid, om = dense
    x = wl.map.origin - 0.35
    rg, ro = check_raycast(ctx, mid, om, x, np.array([1.0, 0.5, 0.0]), 500, wl.params, wl.max_range)
    assert ro["n_hits"] == 0 and np.all(rg["f"] == 0)


def test_w_mode_cubic_and_pole_ray(ctx, dense):
    wl, mid, om = dense
    s = wl.states[2]
    p = dict(wl.params, w_mode=1, halton_offset=0)
    check_raycast(ctx, mid, om, s.x, s.xdot, 3000, p, wl.max_range)


# ----------------------------------------------------------------------------- hashed map
def test_hashed_tsdf_full_config(ctx, hashed):
    wl, mid, om = hashed
    s = wl.states[0]
    rg, ro = check_raycast(ctx, mid, om, s.x, s.xdot, 65536, wl.params, wl.max_range)
    assert ro["n_hits"] > 1000


@pytest.mark.parametrize("n", [7, 257, 5000, 12345])
def test_hashed_ragged(ctx, hashed, n):
    wl, mid, om = hashed
    for s in wl.states[1:4]:
        check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)


def test_hashed_fp64_reduction(ctx, hashed):
    wl, mid, om = hashed
    s = wl.states[4]
    p = dict(wl.params, reduce_mode=R.RMP_REDUCE_FP64)
    rg, ro = check_raycast(ctx, mid, om, s.x, s.xdot, 65536, p, wl.max_range)
    pk = dict(wl.params, reduce_mode=R.RMP_REDUCE_KAHAN32)
    rk, _, _ = gpu_raycast(ctx, mid, s.x, s.xdot, 65536, R.make_params(pk, wl.max_range), want=False)
    # both reductions agree with the FP64 oracle far inside the f tolerance
    for r in (rg, rk):
        assert np.linalg.norm(r["f"] - ro["f"]) <= 1e-5 * np.linalg.norm(ro["f"])


def test_hashed_zero_velocity(ctx, hashed):
    wl, mid, om = hashed
    rg, ro = check_raycast(ctx, mid, om, wl.states[0].x, np.zeros(3), 4096, wl.params, wl.max_range)
    assert rg["n_active"] == 0 and np.all(rg["f"] == 0) and rg["rank"] == 0


def test_hashed_map_from_device_buffers(ctx, hashed):
    torch = torch_cuda()
    wl, mid, om = hashed
    keys = torch.from_numpy(wl.map.keys).cuda()
    tsdf = torch.from_numpy(wl.map.tsdf).cuda()
    mid2 = R.rmp_map_upload(ctx.handle, R.hashed_desc(keys, tsdf, wl.map.voxel_size))
    s = wl.states[5]
    pg = R.make_params(wl.params, wl.max_range)
    r1, h1, p1 = gpu_raycast(ctx, mid, s.x, s.xdot, 8192, pg)
    r2, h2, p2 = gpu_raycast(ctx, mid2, s.x, s.xdot, 8192, pg)
    assert h1.tobytes() == h2.tobytes() and np.array_equal(p1, p2)
    assert np.array_equal(r1["f"], r2["f"])
    R.rmp_map_release(ctx.handle, mid2)


def test_empty_hashed_map(ctx):
    hm = W.HashedMap(np.zeros((0, 3), np.int32), np.zeros((0, 512), np.float32), 0.1)
    mid = ctx.upload(hm)
    p = dict(W.PARAMS_STATIC_MAP)
    rg, ro = check_raycast(ctx, mid, O.OracleMap(hm), np.array([1.0, 2.0, 3.0]),
                           np.array([1.0, 0.0, 0.0]), 3000, p, 10.0)
    assert rg["n_hits"] == 0 and np.all(rg["f"] == 0)


def test_negative_block_keys(ctx):
    rng = np.random.default_rng(4)
    keys = np.array([(x, y, z) for x in (-2, -1, 0) for y in (-1, 0) for z in (-1, 0)], np.int32)
    tsdf = rng.uniform(-0.05, 0.3, (len(keys), 512)).astype(np.float32)
    hm = W.HashedMap(keys, tsdf, 0.05)
    mid = ctx.upload(hm)
    p = dict(W.PARAMS_STATIC_MAP)
    check_raycast(ctx, mid, O.OracleMap(hm), np.array([-0.01, 0.013, -0.2]),
                  np.array([0.3, -1.0, 0.7]), 5000, p, 1.0)


# ----------------------------------------------------------------------------- LiDAR
def test_lidar_scan_full_config(ctx):
    sw = W.lidar_workload()
    pg = R.make_params(sw.params, sw.max_range)
    po = O.make_params(sw.params, sw.max_range)
    rg, pgr = gpu_scan(ctx, sw.points, sw.x, sw.xdot, pg)
    ro, por = O.scan_eval(sw.points, sw.x, sw.xdot, po)
    at = scan_abs_term(sw.points, sw.x, sw.xdot, sw.params)
    assert_per_ray_close(pgr, por, at)
    assert_result_close(rg, ro, por, at)


@pytest.mark.parametrize("n", [1, 100, 3333])
def test_lidar_ragged_and_offset_sensor(ctx, n):
    sw = W.lidar_workload()
    pts = sw.points[:n] + np.float32(3.0)
    x = np.array([3.0, 3.0, 3.0])
    xdot = np.array([0.4, -1.2, 0.3])
    for red in (0, 1):
        p = dict(sw.params, reduce_mode=red)
        rg, pgr = gpu_scan(ctx, pts, x, xdot, R.make_params(p, sw.max_range))
        ro, por = O.scan_eval(pts, x, xdot, O.make_params(p, sw.max_range))
        at = scan_abs_term(pts, x, xdot, p)
        assert_per_ray_close(pgr, por, at)
        assert_result_close(rg, ro, por, at)


def test_lidar_centred_sphere(ctx):
    p = dict(W.PARAMS_LIDAR, min_range=0.0)
    pts = W.sphere_lattice_scan(65536, 0.8)
    xdot = np.array([0.36, 0.48, 0.8]) * 1.7
    rg, pgr = gpu_scan(ctx, pts, np.zeros(3), xdot, R.make_params(p, 30.0))
    ro, por = O.scan_eval(pts, np.zeros(3), xdot, O.make_params(p, 30.0))
    at = scan_abs_term(pts, np.zeros(3), xdot, p)
    assert_per_ray_close(pgr, por, at)
    assert_result_close(rg, ro, por, at)


# ----------------------------------------------------------------------------- async / determinism
def test_async_matches_sync_bitwise(ctx, hashed):
    torch = torch_cuda()
    wl, mid, om = hashed
    s = wl.states[2]
    pg = R.make_params(wl.params, wl.max_range)
    r_sync, _, _ = gpu_raycast(ctx, mid, s.x, s.xdot, 30000, pg, want=False)
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    state = torch.tensor(np.concatenate([s.x, s.xdot]), dtype=torch.float64, device="cuda")
    out = torch.empty(R.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        R.rmp_raycast_eval_async(ctx.handle, mid, state, 30000, pg, ws, out)
        r = R.result_from_bytes(out.cpu().numpy().tobytes())
        for k in ("f", "sumA", "sumAf", "eig"):
            assert np.array_equal(r[k], r_sync[k]), k
        assert (r["n_hits"], r["n_active"], r["rank"]) == (r_sync["n_hits"], r_sync["n_active"],
                                                            r_sync["rank"])


def test_workspace_left_ready_and_poisoned_state(ctx, hashed):
    """Each evaluation leaves its workspace as rmp_workspace_init does (header zero, every
    partial slot back to all-ones); a workspace whose header is marked poisoned (the state
    a finish whose bounded wait expired leaves) makes a multi-CTA evaluation report
    RMP_ERR_TIMEOUT until it is initialised again, after which results are bit-identical
    to the synchronous call."""
    torch = torch_cuda()
    wl, mid, om = hashed
    s = wl.states[1]
    pg = R.make_params(wl.params, wl.max_range)
    r_sync, _, _ = gpu_raycast(ctx, mid, s.x, s.xdot, 30000, pg, want=False)
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    fresh = ws.cpu().numpy().copy()
    assert np.all(fresh[:1024] == 0) and np.all(fresh[1024:] == 0xFF)
    state = torch.tensor(np.concatenate([s.x, s.xdot]), dtype=torch.float64, device="cuda")
    out = torch.empty(R.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    R.rmp_raycast_eval_async(ctx.handle, mid, state, 30000, pg, ws, out)
    assert R.result_from_bytes(out.cpu().numpy().tobytes())["status"] == 0
    assert np.array_equal(ws.cpu().numpy(), fresh)
    ws[0] = 1                                          # header: poisoned
    for _ in range(2):
        R.rmp_raycast_eval_async(ctx.handle, mid, state, 30000, pg, ws, out)
        assert R.result_from_bytes(out.cpu().numpy().tobytes())["status"] == 4
    R.rmp_workspace_init(ws)
    R.rmp_raycast_eval_async(ctx.handle, mid, state, 30000, pg, ws, out)
    r = R.result_from_bytes(out.cpu().numpy().tobytes())
    assert r["status"] == 0
    for k in ("f", "sumA", "sumAf", "eig"):
        assert np.array_equal(r[k], r_sync[k]), k


def test_async_bad_state_reports_invalid(ctx, hashed):
    torch = torch_cuda()
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    out = torch.empty(R.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for bad in (np.nan, np.inf, 1e12):
        state = torch.tensor([bad, 1.0, 1.0, 0.0, 0.0, 0.0], dtype=torch.float64, device="cuda")
        R.rmp_raycast_eval_async(ctx.handle, mid, state, 1000, pg, ws, out)
        r = R.result_from_bytes(out.cpu().numpy().tobytes())
        assert r["status"] == 1
        assert np.all(r["f"] == 0) and r["n_hits"] == 0
    # the workspace is still usable afterwards
    s = wl.states[0]
    state = torch.tensor(np.concatenate([s.x, s.xdot]), dtype=torch.float64, device="cuda")
    R.rmp_raycast_eval_async(ctx.handle, mid, state, 1000, pg, ws, out)
    assert R.result_from_bytes(out.cpu().numpy().tobytes())["status"] == 0


def test_repeated_runs_bitwise_identical(ctx, hashed):
    wl, mid, om = hashed
    s = wl.states[3]
    pg = R.make_params(wl.params, wl.max_range)
    a = gpu_raycast(ctx, mid, s.x, s.xdot, 65536, pg)
    b = gpu_raycast(ctx, mid, s.x, s.xdot, 65536, pg)
    assert np.array_equal(a[0]["f"], b[0]["f"]) and np.array_equal(a[0]["sumA"], b[0]["sumA"])
    assert a[1].tobytes() == b[1].tobytes() and np.array_equal(a[2], b[2])


# ----------------------------------------------------------------------------- argument errors
def test_argument_errors(ctx, hashed):
    wl, mid, om = hashed
    s = wl.states[0]
    good = dict(wl.params)
    with pytest.raises(R.RmpError) as e:
        R.rmp_raycast_eval(ctx.handle, 9999, s.x, s.xdot, 10, R.make_params(good, 10.0))
    assert e.value.status == 6
    for bad in (dict(good, nu_rep=0.0), dict(good, c=-1.0), dict(good, w_mode=2),
                dict(good, reduce_mode=5), dict(good, eps=float("nan"))):
        with pytest.raises(R.RmpError) as e:
            R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 10, R.make_params(bad, 10.0))
        assert e.value.status == 1
    with pytest.raises(R.RmpError):                      # more than 16384 voxels of range
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 10, R.make_params(good, 1700.0))
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 0, R.make_params(good, 10.0))
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 1 << 24, R.make_params(good, 10.0))
    # the largest accepted range still works: 16384 voxels
    R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 64, R.make_params(good, 1638.4))


def test_map_upload_errors(ctx):
    keys = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0]], np.int32)
    tsdf = np.ones((3, 512), np.float32)
    with pytest.raises(R.RmpError) as e:
        ctx.upload(W.HashedMap(keys, tsdf, 0.1))
    assert e.value.status == 1
    keys = np.array([[1 << 20, 0, 0]], np.int32)
    with pytest.raises(R.RmpError):
        ctx.upload(W.HashedMap(keys, np.ones((1, 512), np.float32), 0.1))
    with pytest.raises(R.RmpError):
        ctx.upload(W.DenseMap(np.zeros((4, 4, 4), np.uint8), 0.0, np.zeros(3)))
    # the context is still usable
    mid = ctx.upload(W.DenseMap(np.zeros((4, 4, 4), np.uint8), 0.1, np.zeros(3)))
    info = R.rmp_map_info(ctx.handle, mid)
    assert info["n_bricks"] == 1 and info["kind"] == 0
    R.rmp_map_release(ctx.handle, mid)
    with pytest.raises(R.RmpError):
        R.rmp_map_release(ctx.handle, mid)


# ----------------------------------------------------------------------------- block skipping
@pytest.mark.parametrize("max_range", [0.37, 1.33, 3.3, 7.77])
def test_hashed_ranges_ending_inside_skipped_blocks(ctx, hashed, max_range):
    wl, mid, om = hashed
    for s in wl.states[:3]:
        check_raycast(ctx, mid, om, s.x, s.xdot, 6000, wl.params, max_range)


def test_dense_grid_not_multiple_of_eight(ctx):
    rng = W.SplitMix64(W.SEED_BASE + 99)
    prims = W.random_boxes(rng, 12, np.zeros(3), np.array([4.5, 3.7, 2.9]), 0.2, 1.0)
    m = W.voxelise_boxes_dense(prims, (45, 37, 29), 0.1)
    mid = ctx.upload(m)
    om = O.OracleMap(m)
    free = np.argwhere(m.occ == 0)
    for t in range(4):
        z, y, x = free[(t * 7919) % len(free)]
        c = (np.array([x, y, z]) + 0.5) * 0.1                      # voxel centre: tie-prone
        check_raycast(ctx, mid, om, c, np.array([0.5, -1.0, 0.3]), 4000, W.PARAMS_STATIC_MAP, 5.0)
        check_raycast(ctx, mid, om, c + 0.0123, np.array([-0.2, 0.4, 1.1]), 4000, W.PARAMS_STATIC_MAP, 2.2)


def test_layouts_grid_and_hash_fallback(ctx, hashed):
    wl, mid, om = hashed
    info = R.rmp_map_info(ctx.handle, mid)
    assert info["layout"] == 0 and info["hash_capacity"] == 0        # grid over the bbox
    rng = np.random.default_rng(8)
    keys = np.array([(x, y, z) for x in (-2, -1, 0) for y in (-1, 0) for z in (-1, 0)]
                    + [(5000, 4000, 700), (-6000, 10, -900)], np.int32)
    tsdf = rng.uniform(-0.05, 0.3, (len(keys), 512)).astype(np.float32)
    hm = W.HashedMap(keys, tsdf, 0.05)
    mid2 = ctx.upload(hm)
    info2 = R.rmp_map_info(ctx.handle, mid2)
    assert info2["layout"] == 1 and info2["hash_capacity"] >= 4 * len(keys)
    p = dict(W.PARAMS_STATIC_MAP)
    for x in (np.array([-0.01, 0.013, -0.2]), np.array([0.11, -0.05, 0.02])):
        check_raycast(ctx, mid2, O.OracleMap(hm), x, np.array([0.3, -1.0, 0.7]), 5000, p, 1.0)
    # the same blocks without the far ones use the grid layout and give identical hits
    hm3 = W.HashedMap(keys[:-2], tsdf[:-2], 0.05)
    mid3 = ctx.upload(hm3)
    assert R.rmp_map_info(ctx.handle, mid3)["layout"] == 0
    pg = R.make_params(p, 1.0)
    x = np.array([-0.01, 0.013, -0.2])
    a = gpu_raycast(ctx, mid2, x, np.array([0.3, -1.0, 0.7]), 5000, pg)
    b = gpu_raycast(ctx, mid3, x, np.array([0.3, -1.0, 0.7]), 5000, pg)
    assert a[1].tobytes() == b[1].tobytes()


@pytest.mark.parametrize("cells,lgs", [(1, 0), (1, 2), (0, 0), (1, 4), (0, 3), (1, 5), (0, 5)])
def test_cell_skip_keeps_results(ctx, hashed, dense, cells, lgs):
    """Voxel-box skipping inside occupied blocks on or off changes nothing: hit records
    bit-identical to the oracle's, values within tolerance (single-state kernel)."""
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_CELL_SKIP, cells)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, lgs)
    try:
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_CELL_SKIP) == cells
        wl, mid, om = hashed
        for s, n in ((wl.states[0], 65536), (wl.states[5], 3001)):
            check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)
        wl, mid, om = dense
        for s, n in ((wl.states[1], 4096), (wl.states[7], 1000)):
            check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_CELL_SKIP, -1)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, -1)
    with pytest.raises(R.RmpError):
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_CELL_SKIP, 2)


@pytest.mark.parametrize("order,budget,lgs", [(0, 1, 0), (0, 2, 2), (1, 3, 0), (1, 24, 1),
                                               (0, 0, 0), (1, -1, -1), (0, 7, 1)])
def test_split_and_ray_order_keep_results(ctx, hashed, dense, order, budget, lgs):
    """Ray order and the warp split of long pieces (budgets down to one iteration, so that
    nearly every warp splits, with and without static segments) leave hit records
    bit-identical to the oracle's and values within tolerance, on the hashed map and on the
    dense map, whose rays also leave the map."""
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_RAY_ORDER, order)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET, budget)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, lgs)
    try:
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET) == budget
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_RAY_ORDER) == order
        wl, mid, om = hashed
        for s, n in ((wl.states[3], 65536), (wl.states[4], 777)):
            check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)
        wl, mid, om = dense
        for s, n in ((wl.states[5], 4097), (wl.states[6], 1024)):
            check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_RAY_ORDER, 0)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET, -1)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, -1)
    for knob, bad in ((R.RMP_TUNE_RAY_ORDER, 2), (R.RMP_TUNE_SPLIT_BUDGET, -2),
                      (R.RMP_TUNE_SPLIT_BUDGET, 65537)):
        with pytest.raises(R.RmpError):
            R.rmp_tune_set(ctx.handle, knob, bad)


@pytest.mark.parametrize("block,lgs", [(64, 0), (128, 1), (256, 2), (128, -1), (0, -1),
                                       (256, 3), (128, 4), (64, 4), (256, 5), (64, 5)])
def test_tuning_knobs_keep_results(ctx, hashed, block, lgs):
    """Block size and ray segmentation change the launch shape only: hit records stay
    bit-identical to the oracle's, values within tolerance."""
    wl, mid, om = hashed
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, block)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, lgs)
    try:
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_BLOCK) == block
        for s, n in ((wl.states[1], 65536), (wl.states[2], 777)):
            check_raycast(ctx, mid, om, s.x, s.xdot, n, wl.params, wl.max_range)
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 0)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, -1)
    with pytest.raises(R.RmpError):
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 100)
    with pytest.raises(R.RmpError):
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, 6)


def test_automatic_block_size(ctx, hashed):
    """Launch shape by default: as many segments per ray (up to 32) as keep the launch within
    one wave of 256-thread CTAs (occupancy x SMs), 256 threads per CTA while it fits, 128
    beyond it; an explicit setting wins."""
    wl, mid, om = hashed
    p = R.make_params(wl.params, wl.max_range)
    assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_BLOCK) == 0
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 256)
    info = R.rmp_eval_launch_info(ctx.handle, mid, 65536, p)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 0)
    wave = info["sm_count"] * info["ctas_per_sm"] * 256
    assert wave >= 65536                       # the headline evaluation fits in one wave
    for n in (1, 1024, 4096, 16384, 19456, 19457, 32768, 38912, 38913, 65536, 262144, 1 << 20):
        li = R.rmp_eval_launch_info(ctx.handle, mid, n, p)
        # segments per ray: the most (up to 32) that keep the launch within one wave
        lg = 5
        while lg > 0 and (n << lg) > wave:
            lg -= 1
        assert li["lg_segments"] == lg, (n, li)
        threads = n << li["lg_segments"]
        assert li["block"] == (256 if threads <= wave else 128), (n, li)
        assert li["grid"] == min(4096, (threads + li["block"] - 1) // li["block"])
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 64)
    try:
        assert R.rmp_eval_launch_info(ctx.handle, mid, 65536, p)["block"] == 64
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 0)


def _grid_occupancy(m, gmin, gdim):
    """Occupancy [z, y, x] of the grid's voxels from the map description (outside: free)."""
    V = np.zeros((8 * gdim[2], 8 * gdim[1], 8 * gdim[0]), bool)
    if isinstance(m, W.DenseMap):
        assert np.all(gmin == 0)
        nz, ny, nx = m.occ.shape
        V[:nz, :ny, :nx] = m.occ != 0
        return V
    for key, t in zip(m.keys, m.tsdf):
        occ = (t <= 0).reshape(8, 8, 8)
        b = key - gmin
        if np.any(b < 0) or np.any(b >= gdim):
            assert not occ.any()              # every occupied block lies inside the grid
            continue
        V[8 * b[2]:8 * b[2] + 8, 8 * b[1]:8 * b[1] + 8, 8 * b[0]:8 * b[0] + 8] = occ
    return V


def _dilate(D):
    """One voxel of Chebyshev dilation (3^3 maximum), nothing beyond the volume."""
    for ax in range(3):
        E = D.copy()
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[ax], lo[ax] = slice(1, None), slice(None, -1)
        E[tuple(hi)] |= D[tuple(lo)]
        E[tuple(lo)] |= D[tuple(hi)]
        D = E
    return D


@pytest.mark.parametrize("which", ["dense", "hashed"])
def test_cell_distances_brute_force(ctx, dense, hashed, which):
    """The voxel-box data (4-bit Chebyshev distance of each 2^3 cell to the nearest occupied
    voxel, capped at 4) equals a brute-force distance transform of the map's occupancy:
    an overestimate would let the march skip an occupied voxel."""
    wl, mid, _ = dense if which == "dense" else hashed
    gmin, gdim, cells = R.rmp_map_cell_distances(ctx.handle, mid)
    V = _grid_occupancy(wl.map, gmin, gdim)
    dist = np.where(V, 0, 4).astype(np.uint8)
    D = V
    for k in range(1, 4):
        D = _dilate(D)
        dist[(dist == 4) & D] = k
    gx, gy, gz = (int(v) for v in gdim)
    cell = dist.reshape(4 * gz, 2, 4 * gy, 2, 4 * gx, 2).min(axis=(1, 3, 5))
    per_brick = cell.reshape(gz, 4, gy, 4, gx, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)
    occupied = V.reshape(gz, 8, gy, 8, gx, 8).any(axis=(1, 3, 5)).reshape(-1)
    per_brick[~occupied] = 0
    nib = per_brick.reshape(-1, 8, 8).astype(np.uint32) << (4 * np.arange(8, dtype=np.uint32))
    expect = np.bitwise_or.reduce(nib, axis=2).reshape(-1)
    assert cells.shape == expect.shape
    assert occupied.sum() > 10 and np.any(per_brick[occupied] == 4) and np.any(per_brick == 1)
    bad = np.nonzero(cells != expect)[0]
    assert bad.size == 0, (bad[:8], cells[bad[:8]], expect[bad[:8]])


def test_maximum_ray_count_sampled(ctx, dense):
    """The largest evaluation the ABI allows (2^24 - 1 rays with Halton offset 1): the hit
    counts add up over all rays, and 3000 sampled rays match the oracle ray by ray (hit
    record bit-exact, per-ray policy within tolerance)."""
    torch = torch_cuda()
    wl, mid, om = dense
    s = wl.states[3]
    n = (1 << 24) - 1
    pg = R.make_params(wl.params, wl.max_range)
    po = O.make_params(wl.params, wl.max_range)
    hits = torch.empty(n * 24, dtype=torch.uint8, device="cuda")
    per = torch.empty(n * 9, dtype=torch.float32, device="cuda")
    res = R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, n, pg, hits=hits, per_ray=per)
    h = hits.cpu().numpy().view(R.HIT_DTYPE)
    assert res["status"] == 0 and res["n_rays"] == n
    assert res["n_hits"] == int(np.count_nonzero(h["status"] == R.RMP_RAY_HIT))
    idx = np.random.default_rng(12).choice(n, 3000, replace=False)
    P = O.quantize_pos(s.x, wl.map.origin, wl.map.voxel_size)
    R_fx = O.range_fx(wl.max_range, wl.map.voxel_size)
    dirs = np.concatenate([O.ray_dirs(1, int(j) + 1) for j in idx])
    ho = O.dda(om, P, O.quantize_dirs(dirs), R_fx)
    assert_hits_exact(h[idx], ho)
    pv = per.view(n, 9)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    por = np.zeros((len(idx), 9))
    for i, (rec, d) in enumerate(zip(ho, dirs)):
        if rec["status"] != R.RMP_RAY_HIT:
            continue
        r = -d.astype(np.float64)
        f, A = O.ray_policy(po, r, float(rec["d"]), s.xdot, O.active32(s.xdot, d),
                            float(rec["d"]) < po.r)
        por[i, :3], por[i, 3:] = f, A
    assert_per_ray_close(pv, por)
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, n + 1, pg)


def test_fast_binding_matches_ctypes(ctx, hashed):
    """The synchronous calls through the CPython extension and through ctypes reach the
    same C functions: results bitwise equal (raycast and scan)."""
    if not R.fast_binding():
        pytest.skip("CPython extension not built")
    torch = torch_cuda()
    wl, mid, om = hashed
    p = R.make_params(wl.params, wl.max_range)
    s = wl.states[2]
    pts = torch.tensor(np.random.default_rng(4).uniform(-6, 6, (5000, 3)).astype(np.float32),
                       device="cuda")
    got = (R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, 65536, p),
           R.rmp_scan_eval(ctx.handle, pts, s.x, s.xdot, p))
    fast, R._fast = R._fast, None
    try:
        ref = (R.rmp_raycast_eval(ctx.handle, mid, list(s.x), list(s.xdot), 65536, p),
               R.rmp_scan_eval(ctx.handle, pts, s.x, s.xdot, p))
    finally:
        R._fast = fast
    for g, o in zip(got, ref):
        for k in ("f", "sumA", "sumAf", "eig"):
            assert g[k].tobytes() == o[k].tobytes(), k
        for k in ("n_rays", "n_hits", "n_active", "rank", "status"):
            assert g[k] == o[k], k
