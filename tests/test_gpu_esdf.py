"""GPU parity of the ESDF single-query policy (Sec. III-D) against the CPU oracle: the
distance to the closest obstacle and its gradient bit for bit (one FP64 operation order on
both sides), the policy with and without the goal attractor within the stated tolerances,
inside and far from obstacles, with no obstacle, invalid states, many states per launch,
and closed-loop rollouts step for step."""
import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import eig_tolerance, torch_cuda

pytestmark = pytest.mark.gpu

ALPHA, BETA = 10.0, 15.0          # Table I, static map


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = R.Context(0)
    yield c
    c.close()


def run_esdf(ctx, eid, states, goals, params):
    torch = torch_cuda()
    states = np.asarray(states, np.float64).reshape(-1, 6)
    n = len(states)
    st = torch.tensor(states, device="cuda")
    gl = None if goals is None else torch.tensor(np.asarray(goals, np.float64).reshape(-1, 3),
                                                  device="cuda")
    out = torch.empty((n, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    q = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    R.rmp_esdf_eval_async(ctx.handle, eid, st, gl, n, params, ALPHA, BETA, out, q)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return [R.result_from_bytes(o[i].tobytes()) for i in range(n)], q.cpu().numpy()


def assert_esdf_close(g, o):
    """Both sides evaluate the policy in FP64 (library exp / log1p within a few ulp): the sums
    within 1e-12 of their largest entry; f within 1e-9 relative at full rank (the resolve's
    FP64 adjugate solve) and within the stated 1e-4 at rank 1 (the obstacle metric alone,
    resolved through FP32 eigenvectors refined in FP64); the eigenvalues as in gpu_helpers."""
    assert g["status"] == 0
    assert (g["n_rays"], g["n_hits"], g["n_active"]) == (o["n_rays"], o["n_hits"], o["n_active"])
    nA = max(np.abs(o["sumA"]).max(), 1e-300)
    nb = max(np.abs(o["sumAf"]).max(), 1e-300)
    assert np.abs(g["sumA"] - o["sumA"]).max() <= 1e-12 * nA, (g["sumA"], o["sumA"])
    assert np.abs(g["sumAf"] - o["sumAf"]).max() <= 1e-12 * nb, (g["sumAf"], o["sumAf"])
    assert np.all(np.abs(g["eig"] - o["eig"]) <= eig_tolerance(o["eig"], 3e-12 * nA))
    assert g["rank"] == o["rank"]
    nf = np.linalg.norm(o["f"])
    tol = 1e-9 if o["rank"] == 3 else 1e-4
    assert np.linalg.norm(g["f"] - o["f"]) <= tol * nf + 1e-300, (g["f"], o["f"])


def check_states(ctx, eid, pr, states, goals, pdict, max_range=10.0):
    pg = R.make_params(pdict, max_range)
    po = O.make_params(pdict, max_range)
    res, q = run_esdf(ctx, eid, states, goals, pg)
    for i, s in enumerate(np.asarray(states).reshape(-1, 6)):
        ro, qo = O.esdf_eval(pr, s[:3], s[3:], po, goal=None if goals is None else goals[i],
                             alpha=ALPHA, beta=BETA)
        assert np.array_equal(q[i], qo), (i, q[i], qo)          # d and gradient bit for bit
        assert_esdf_close(res[i], ro)
    return res, q


def scene(n_prims=200, extent=(10.0, 10.0, 10.0), size=(0.2, 0.6), seed=9):
    hm, prims = W.hashed_scene(extent, 0.1, n_prims, size_range=size, seed_index=seed)
    return hm, prims


def test_query_and_policy_match_oracle(ctx):
    hm, prims = scene()
    pr = O.prims_array(prims)
    eid = R.rmp_esdf_upload(ctx.handle, prims)
    try:
        rng = np.random.default_rng(3)
        x = rng.uniform(0.0, 10.0, (300, 3))
        x[-20:] = rng.uniform(13.0, 20.0, (20, 3))           # beyond the radius of every obstacle
        v = rng.normal(0.0, 1.0, (300, 3))
        states = np.concatenate([x, v], 1)
        goals = rng.uniform(0.0, 10.0, (300, 3))
        res, q = check_states(ctx, eid, pr, states, goals, W.PARAMS_STATIC_MAP)
        assert np.any(q[:, 0] == 0.0) and np.any(q[:, 0] > 2.4)   # inside and out of radius
        assert sum(r["n_active"] for r in res) > 20
        check_states(ctx, eid, pr, states[:100], None, W.PARAMS_STATIC_MAP)
        check_states(ctx, eid, pr, states[:50], goals[:50], dict(W.PARAMS_STATIC_MAP, w_mode=1))
    finally:
        R.rmp_esdf_release(ctx.handle, eid)


def test_large_boxes_and_spheres_scene(ctx):
    """The 40 x 40 x 10 m scene of the headline map (200 primitives up to 2 m)."""
    wl = W.hashed_workload(n_states=64)
    pr = O.prims_array(wl.prims)
    eid = R.rmp_esdf_upload(ctx.handle, wl.prims)
    try:
        states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states])
        goals = states[::-1, :3].copy()
        check_states(ctx, eid, pr, states, goals, W.PARAMS_STATIC_MAP)
    finally:
        R.rmp_esdf_release(ctx.handle, eid)


def test_no_obstacle_and_invalid_states(ctx):
    torch = torch_cuda()
    eid = R.rmp_esdf_upload(ctx.handle, [])
    try:
        states = np.array([[1.0, 2.0, 3.0, 0.5, -0.5, 0.2]])
        goals = np.array([[4.0, 4.0, 4.0]])
        res, q = check_states(ctx, eid, O.prims_array([]), states, goals, W.PARAMS_STATIC_MAP)
        assert res[0]["n_hits"] == 0 and q[0, 0] == np.inf
        fa = O.attractor(states[0, :3], states[0, 3:], goals[0], ALPHA, BETA,
                         W.PARAMS_STATIC_MAP["c"])
        assert np.allclose(res[0]["f"], fa, rtol=1e-12)
    finally:
        R.rmp_esdf_release(ctx.handle, eid)
    hm, prims = scene(20)
    eid = R.rmp_esdf_upload(ctx.handle, prims)
    try:
        pg = R.make_params(W.PARAMS_STATIC_MAP, 10.0)
        bad = np.array([[np.nan, 1, 1, 0, 0, 0], [1, 1, 1, np.inf, 0, 0], [2, 2, 2, 0, 0, 0.1]])
        res, _ = run_esdf(ctx, eid, bad, None, pg)
        assert [r["status"] for r in res] == [1, 1, 0]
        with pytest.raises(R.RmpError) as e:
            R.rmp_esdf_eval_async(ctx.handle, 99999, torch.zeros((1, 6), dtype=torch.float64,
                                                                 device="cuda"), None, 1, pg,
                                  ALPHA, BETA, torch.empty((1, 144), dtype=torch.uint8,
                                                           device="cuda"))
        assert e.value.status == R.STATUS_CODES["RMP_ERR_UNKNOWN_MAP"]
    finally:
        R.rmp_esdf_release(ctx.handle, eid)
    for bad in (W.Primitive("sphere", np.array([0.0, 0, 0]), np.array([0.0])),
                W.Primitive("box", np.array([np.nan, 0, 0]), np.array([1.0, 1, 1]))):
        with pytest.raises(R.RmpError):
            R.rmp_esdf_upload(ctx.handle, [bad])


def test_many_states_per_launch(ctx):
    """More states than the launch has warps at once (warp-stride loop): 600000 states, a
    sample of 500 against the oracle, bit for bit in d and the gradient."""
    torch = torch_cuda()
    hm, prims = scene(60)
    pr = O.prims_array(prims)
    eid = R.rmp_esdf_upload(ctx.handle, prims)
    try:
        rng = np.random.default_rng(8)
        n = 600000
        states = np.concatenate([rng.uniform(0, 10, (n, 3)), rng.normal(0, 1, (n, 3))], 1)
        pg = R.make_params(W.PARAMS_STATIC_MAP, 10.0)
        po = O.make_params(W.PARAMS_STATIC_MAP, 10.0)
        st = torch.tensor(states, device="cuda")
        out = torch.empty((n, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        q = torch.empty((n, 4), dtype=torch.float64, device="cuda")
        R.rmp_esdf_eval_async(ctx.handle, eid, st, None, n, pg, ALPHA, BETA, out, q)
        torch.cuda.synchronize()
        qn = q.cpu().numpy()
        on = out.cpu().numpy()
        for i in rng.choice(n, 500, replace=False):
            ro, qo = O.esdf_eval(pr, states[i, :3], states[i, 3:], po)
            assert np.array_equal(qn[i], qo)
            g = R.result_from_bytes(on[i].tobytes())
            assert g["n_hits"] == ro["n_hits"] and g["n_active"] == ro["n_active"]
            assert np.allclose(g["sumA"], ro["sumA"], rtol=1e-12, atol=1e-300)
    finally:
        R.rmp_esdf_release(ctx.handle, eid)


def test_rollouts_step_for_step(ctx):
    """ESDF closed loop against the oracle's.  Each control step from the same state agrees
    to FP64 rounding (both sides evaluate the policy in FP64; the library exp and log1p
    differ in the last bits): short rollouts from the starts, and every step along the
    GPU's own 150-step trajectories, each from the state the GPU reached.  (Whole long
    rollouts are not compared state for state: the nearest obstacle changes discontinuously
    where two are equally far, so a last-bit difference there sends the two trajectories
    apart -- 1e-3 m after 150 steps, seen.)  In free space (attractor alone) whole
    rollouts are identical."""
    t = W.rollout_tasks(16, n_prims=200, size_range=(0.2, 0.6))
    mid = ctx.upload(t.map)
    om = O.OracleMap(t.map)
    pr = O.prims_array(t.prims)
    eid = R.rmp_esdf_upload(ctx.handle, t.prims)
    try:
        pg = R.make_params(t.params, t.max_range)
        po = O.make_params(t.params, t.max_range)
        robots = np.concatenate([t.starts, np.zeros_like(t.starts), t.goals], 1)
        for steps in (1, 7):
            rp = R.rollout_params(ALPHA, BETA, 0.01, 0.2, steps, 10, 1)
            rpo = O.rollout_params(ALPHA, BETA, 0.01, 0.2, steps, 10, 1)
            got = R.rmp_rollout_esdf(ctx.handle, mid, eid, robots, pg, rp)
            for b in range(len(robots)):
                o = O.esdf_rollout(om, pr, po, rpo, t.starts[b], np.zeros(3), t.goals[b])
                g = got[b]
                assert (g["status"], g["steps"]) == (o["status"], o["steps"]), b
                assert np.allclose(g["x"], o["x"], rtol=1e-12, atol=1e-12), b
                assert np.allclose(g["xdot"], o["xdot"], rtol=1e-10, atol=1e-10), b
        # step by step along the GPU's trajectories: one step from the same state each time
        rp1 = R.rollout_params(ALPHA, BETA, 0.01, 0.2, 1, 10, 1)
        rpo1 = O.rollout_params(ALPHA, BETA, 0.01, 0.2, 1, 10, 1)
        cur = robots.copy()
        n_moving = 0
        for n in range(150):
            got = R.rmp_rollout_esdf(ctx.handle, mid, eid, cur, pg, rp1)
            for b in range(len(cur)):
                o = O.esdf_rollout(om, pr, po, rpo1, cur[b, :3], cur[b, 3:6], cur[b, 6:])
                g = got[b]
                assert (g["status"], g["steps"]) == (o["status"], o["steps"]), (n, b)
                assert np.allclose(g["x"], o["x"], rtol=1e-13, atol=1e-13), (n, b)
                assert np.allclose(g["xdot"], o["xdot"], rtol=1e-11, atol=1e-11), (n, b)
                if g["status"] == R.RMP_ROLLOUT_TIMEOUT:      # one step taken, still going
                    cur[b, :3] = g["x"]
                    cur[b, 3:6] = g["xdot"]
                    n_moving += 1
        assert n_moving > 1000
        # free space: no obstacle, exactly the oracle's steps
        eid0 = R.rmp_esdf_upload(ctx.handle, [])
        try:
            rp = R.rollout_params(ALPHA, BETA, 0.01, 0.2, 300, 10, 1)
            rpo = O.rollout_params(ALPHA, BETA, 0.01, 0.2, 300, 10, 1)
            got = R.rmp_rollout_esdf(ctx.handle, mid, eid0, robots[:4], pg, rp)
            for b in range(4):
                o = O.esdf_rollout(om, O.prims_array([]), po, rpo, t.starts[b], np.zeros(3),
                                   t.goals[b])
                assert np.allclose(got[b]["x"], o["x"], rtol=1e-13, atol=1e-13)
        finally:
            R.rmp_esdf_release(ctx.handle, eid0)
    finally:
        R.rmp_esdf_release(ctx.handle, eid)
        R.rmp_map_release(ctx.handle, mid)
