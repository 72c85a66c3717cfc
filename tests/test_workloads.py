"""Checks of the seeded input generators shared by the oracle and the GPU tests
(paper_2301_08068_gb300/workloads.py): the SplitMix64 stream against its published
definition and first outputs, draws that do not depend on how a stream is chunked, and
the invariants the workloads promise (robots in free space, ordered request streams)."""
import numpy as np

from paper_2301_08068_gb300 import workloads as W

MASK = (1 << 64) - 1


def splitmix64_scalar(state, n):
    """Steele, Lea and Flood's SplitMix64, one value at a time with Python integers."""
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out, state


def test_splitmix64_first_outputs_for_seed_zero():
    assert [int(v) for v in W.SplitMix64(0).u64(4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_matches_scalar_definition_across_chunks():
    seed = W.SEED_BASE + 7
    expect, end_state = splitmix64_scalar(seed, 1000)
    r = W.SplitMix64(seed)
    got = np.concatenate([r.u64(1), r.u64(0), r.u64(37), r.u64(962)])
    assert [int(v) for v in got] == expect
    assert int(r.state) == end_state


def test_uniform_and_normal_draws():
    r = W.SplitMix64(W.SEED_BASE + 3)
    u = r.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))     # 53-bit values
    assert abs(u.mean() - 0.5) < 3e-3
    z = W.SplitMix64(W.SEED_BASE + 4).normal(200001)
    assert z.shape == (200001,)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    k = W.SplitMix64(W.SEED_BASE + 5).integers(10000, 7)
    assert k.min() == 0 and k.max() == 6


def test_dense_robots_start_in_free_voxels():
    wl = W.dense_box_workload(n_states=32, jitter=True)
    occ = wl.map.occ
    for s in wl.states:
        v = np.floor((s.x - wl.map.origin) / wl.map.voxel_size).astype(int)   # x, y, z
        assert occ[v[2], v[1], v[0]] == 0
    assert 0.0 < occ.mean() < 0.5


def test_hashed_robots_start_outside_the_truncation_band():
    wl = W.hashed_workload(n_states=16)
    x = np.stack([s.x for s in wl.states])
    sdf = W.scene_sdf(wl.prims, x)
    assert np.all(sdf > W.TSDF_TRUNCATION)
    assert wl.map.keys.shape == (wl.map.n_blocks, 3) and wl.map.tsdf.shape == (wl.map.n_blocks, 512)
    assert np.all(np.abs(wl.map.tsdf) <= W.TSDF_TRUNCATION + 1e-6)


def test_poisson_request_stream():
    t, maps, rays, vel = W.poisson_requests(3, 20000.0, 0.5, 1024, 262144, seed_index=9)
    assert np.all(np.diff(t) > 0) and t[0] >= 0.0 and t[-1] < 0.5
    assert abs(len(t) - 10000) < 400                  # Poisson count, mean 10000
    assert set(np.unique(maps)) == {0, 1, 2}
    assert rays.min() >= 1024 and rays.max() <= 262144
    assert vel.shape == (len(t), 3)


def test_lidar_scan_points():
    sw = W.lidar_workload(beams=16, columns=256)
    pts = sw.points.reshape(-1, 3)
    assert pts.shape == (16 * 256, 3) and pts.dtype == np.float32
    finite = np.all(np.isfinite(pts), axis=1)
    assert finite.any()
    r = np.linalg.norm(pts[finite].astype(np.float64), axis=1)
    assert r.min() > 0.0 and r.max() < 31.0
