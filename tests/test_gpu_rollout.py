"""GPU parity of the attractor combination (Eq. 1 with the goal attractor) and of the
closed-loop rollout against the CPU oracle: combined sums and f_c per state; rollouts in a
free map (where f_c = f_a in FP64 on both sides) step for step, including the step at which
a robot enters a wall, leaves the grid, reaches its goal or times out; and short rollouts
among obstacles within a tolerance that grows with the path."""
import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import (REL, REL_F, UNDERFLOW, _full, abs_sums, eig_tolerance, observed_f_bound,
                         torch_cuda)

pytestmark = pytest.mark.gpu

ALPHA, BETA = 10.0, 15.0          # Table I, static map


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = R.Context(0)
    yield c
    c.close()


def assert_combined_close(g, o, por):
    """The gpu_helpers tolerances applied to the combined sums: the obstacle part carries
    the per-ray FP32 error (1e-5 of sum |A_i| per entry, likewise sum |A_i f_i|); I and
    f_a are added in FP64 on both sides (1e-15 of the combined entry for that rounding)."""
    assert g["status"] == 0 and g["n_hits"] == o["n_hits"] and g["n_active"] == o["n_active"]
    A, Af = abs_sums(por)
    tolA = REL * A + 1e-15 * np.abs(o["sumA"]) + UNDERFLOW
    tolAf = REL * Af + 1e-15 * np.abs(o["sumAf"]) + UNDERFLOW
    assert np.all(np.abs(g["sumA"] - o["sumA"]) <= tolA)
    assert np.all(np.abs(g["sumAf"] - o["sumAf"]) <= tolAf)
    lam = o["eig"]
    dS = np.linalg.norm(_full(tolA), "fro")
    assert np.all(np.abs(g["eig"] - lam) <= eig_tolerance(lam, dS))
    assert g["rank"] == o["rank"] == 3 and lam[0] >= 1.0 - 1e-12
    b = observed_f_bound(g, o)
    assert b is not None                      # I in the metric keeps the sum well away from 0
    nf = np.linalg.norm(o["f"])
    assert np.linalg.norm(g["f"] - o["f"]) <= max(REL_F * nf, b) + 1e-300


def test_combined_eval_matches_oracle(ctx):
    torch = torch_cuda()
    for wl, n in ((W.dense_box_workload(n_states=6, jitter=True), 1024),
                  (W.hashed_workload(n_states=6, state_seed_index=51), 20000)):
        mid = ctx.upload(wl.map)
        om = O.OracleMap(wl.map)
        rng = np.random.default_rng(4)
        goals = np.stack([s.x + rng.uniform(-3, 3, 3) for s in wl.states])
        states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states])
        B = len(wl.states)
        pg = R.make_params(wl.params, wl.max_range)
        po = O.make_params(wl.params, wl.max_range)
        st = torch.tensor(states, device="cuda")
        gl = torch.tensor(goals, device="cuda")
        nr = torch.full((B,), n, dtype=torch.int32, device="cuda")
        ws = torch.empty(R.rmp_batch_workspace_bytes(B, n), dtype=torch.uint8, device="cuda")
        out = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        for mean in (False, True):
            R.rmp_combined_eval_batch_async(ctx.handle, mid, st, nr, B, n, pg, gl, ALPHA, BETA,
                                            ws, out, metric_mean=mean)
            torch.cuda.synchronize()
            for b, s in enumerate(wl.states):
                g = R.result_from_bytes(out[b].cpu().numpy().tobytes())
                ro = O.combined_eval(om, s.x, s.xdot, n, po, goals[b], ALPHA, BETA, metric_mean=mean)
                _, _, por = O.raycast_eval(om, s.x, s.xdot, n, po, want_hits=False)
                if mean:                    # the mean metric scales A_i (and A_i f_i), not f_i
                    por = por.copy()
                    por[:, 3:] /= n
                assert_combined_close(g, ro, por)
        R.rmp_map_release(ctx.handle, mid)


def _robots(starts, goals):
    return np.concatenate([np.asarray(starts, float), np.zeros((len(starts), 3)),
                           np.asarray(goals, float)], axis=1)


def test_free_and_wall_rollouts_step_for_step(ctx):
    """Without obstacle forces f_c = f_a on both sides, so GPU and oracle rollouts agree to
    rounding and stop at the same step for the same reason."""
    n = 64
    occ = np.zeros((n, n, n), np.uint8)
    occ[:, :, 40] = 1                                    # wall at x in [4.0, 4.1) m
    wall = W.DenseMap(occ, 0.1, np.zeros(3))
    empty = W.DenseMap(np.zeros((n, n, n), np.uint8), 0.1, np.zeros(3))
    quiet = dict(W.PARAMS_STATIC_MAP, eta_rep=0.0, eta_damp=0.0)
    starts = [[1.05, 3.2, 3.2], [1.05, 1.0, 2.0], [2.0, 2.0, 2.0], [3.3, 3.3, 3.3]]
    goals = [[1e6, 3.2, 3.2], [1.05, 5.0, 5.5], [2.0, 2.0, 2.0], [0.5, 6.0, 1.0]]
    for m in (wall, empty):
        mid = ctx.upload(m)
        om = O.OracleMap(m)
        for max_steps in (5, 3000):
            rp = R.rollout_params(ALPHA, BETA, 0.01, 0.05, max_steps, 10, 256)
            orp = O.rollout_params(ALPHA, BETA, 0.01, 0.05, max_steps, 10, 256)
            got = R.rmp_rollout(ctx.handle, mid, _robots(starts, goals), R.make_params(quiet, 3.0), rp)
            for g, s0, gl in zip(got, starts, goals):
                o = O.rollout(om, O.make_params(quiet, 3.0), orp, s0, np.zeros(3), gl)
                assert g["status"] == o["status"] and g["steps"] == o["steps"], (g, o)
                assert np.allclose(g["x"], o["x"], rtol=1e-12, atol=1e-12)
                assert np.allclose(g["xdot"], o["xdot"], rtol=1e-12, atol=1e-12)
                assert g["path_length"] == pytest.approx(o["path_length"], rel=1e-12, abs=1e-12)
                assert g["smooth_n"] == o["smooth_n"]
                assert g["smoothness"] == pytest.approx(o["smoothness"], abs=1e-9)
        R.rmp_map_release(ctx.handle, mid)
    assert got[2]["status"] == R.RMP_ROLLOUT_REACHED and got[2]["steps"] == 1


def test_short_rollouts_among_obstacles(ctx):
    wl = W.hashed_workload(n_states=6, state_seed_index=52)
    mid = ctx.upload(wl.map)
    om = O.OracleMap(wl.map)
    rng = np.random.default_rng(6)
    starts = [s.x for s in wl.states]
    goals = [s.x + rng.uniform(-5, 5, 3) for s in wl.states]
    steps = 25
    po = O.make_params(wl.params, wl.max_range)
    for mean in (False, True):
        rp = R.rollout_params(ALPHA, BETA, 0.01, 0.05, steps, 5, 1024, metric_mean=mean)
        orp = O.rollout_params(ALPHA, BETA, 0.01, 0.05, steps, 5, 1024, metric_mean=mean)
        got = R.rmp_rollout(ctx.handle, mid, _robots(starts, goals),
                            R.make_params(wl.params, wl.max_range), rp)
        for g, s0, gl in zip(got, starts, goals):
            o = O.rollout(om, po, orp, s0, np.zeros(3), gl)
            assert g["status"] == o["status"] and g["steps"] == o["steps"]
            tol = 1e-4 * o["path_length"] + 1e-9
            assert np.linalg.norm(g["x"] - o["x"]) <= tol, (g["x"], o["x"])
            assert g["path_length"] == pytest.approx(o["path_length"], rel=1e-4, abs=1e-9)
    R.rmp_map_release(ctx.handle, mid)


def test_rollout_argument_errors(ctx):
    wl = W.dense_box_workload()
    mid = ctx.upload(wl.map)
    p = R.make_params(wl.params, wl.max_range)
    robots = _robots([wl.states[0].x], [wl.states[0].x + 1.0])
    for bad in (R.rollout_params(ALPHA, BETA, 0.0, 0.1, 10, 5, 64),
                R.rollout_params(ALPHA, BETA, 0.01, 0.1, 0, 5, 64),
                R.rollout_params(ALPHA, BETA, 0.01, 0.1, 10, 5, 0)):
        with pytest.raises(R.RmpError):
            R.rmp_rollout(ctx.handle, mid, robots, p, bad)
    with pytest.raises(R.RmpError):
        R.rmp_rollout(ctx.handle, 9999, robots, p, R.rollout_params(ALPHA, BETA, 0.01, 0.1, 10, 5, 64))
    R.rmp_map_release(ctx.handle, mid)
