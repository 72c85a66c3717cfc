"""Pins of the oracle's attractor, combined policy (Eq. 1 with the attractor) and closed-loop
rollout step against closed forms and invariants: the soft-normalisation limits of the
attractor, the exact combination in an empty map (f_c = f_a), the normal equations of the
combination with obstacles, the discrete damped dynamics in free space (a geometric series),
and the step at which a robot without obstacle policy enters a wall, leaves the grid, reaches
its goal or times out."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import workloads as W

ALPHA, BETA = 10.0, 15.0          # Table I, static map: alpha_g, beta_g
C_SOFT = 0.2


def empty_dense(n=64, vs=0.1):
    return W.DenseMap(np.zeros((n, n, n), np.uint8), vs, np.zeros(3))


def test_attractor_limits():
    x = np.array([1.0, -2.0, 0.5])
    xd = np.array([0.3, 0.1, -0.7])
    # at the goal the spring term vanishes: only damping
    fa = O.attractor(x, xd, x, ALPHA, BETA, C_SOFT)
    assert np.array_equal(fa, -BETA * xd)
    # far away s is the unit vector to the goal
    g = x + 1e6 * np.array([0.6, 0.0, 0.8])
    fa = O.attractor(x, np.zeros(3), g, ALPHA, BETA, C_SOFT)
    assert np.allclose(fa, ALPHA * np.array([0.6, 0.0, 0.8]), rtol=1e-12, atol=0)
    # very close, |s(v)| -> |v| / (c ln 2)
    v = np.array([3e-10, -4e-10, 0.0])
    fa = O.attractor(np.zeros(3), np.zeros(3), v, ALPHA, BETA, C_SOFT)
    assert np.allclose(fa, ALPHA * v / (C_SOFT * math.log(2.0)), rtol=1e-8, atol=0)
    # s(v) is parallel to v and its length grows with |v|, staying below 1
    lens = []
    for z in (0.01, 0.1, 1.0, 5.0, 20.0):
        fa = O.attractor(x, np.zeros(3), x + z * np.array([0.0, 1.0, 0.0]), ALPHA, BETA, C_SOFT)
        assert fa[0] == 0.0 and fa[2] == 0.0 and fa[1] > 0.0
        lens.append(fa[1] / ALPHA)
    assert all(a < b for a, b in zip(lens, lens[1:])) and lens[-1] < 1.0


def test_combined_in_empty_map_is_the_attractor():
    om = O.OracleMap(empty_dense())
    p = O.make_params(W.PARAMS_STATIC_MAP, 5.0)
    x = np.array([3.2, 3.1, 3.3])
    xd = np.array([0.5, -0.2, 0.1])
    g = np.array([1.0, 5.0, 2.0])
    r = O.combined_eval(om, x, xd, 1024, p, g, ALPHA, BETA)
    fa = O.attractor(x, xd, g, ALPHA, BETA, p.c)
    assert r["n_hits"] == 0
    assert np.array_equal(r["sumA"], [1, 0, 0, 1, 0, 1]) and np.array_equal(r["sumAf"], fa)
    assert np.allclose(r["f"], fa, rtol=1e-14, atol=0) and r["rank"] == 3
    assert np.allclose(r["eig"], 1.0, rtol=1e-14)


def test_combined_solves_the_normal_equations():
    """With obstacles, sum A + I is positive definite, so f_c is the unique solution of
    (sum A + I) f_c = sum A f + f_a."""
    wl = W.dense_box_workload(n_states=4, jitter=True)
    om = O.OracleMap(wl.map)
    p = O.make_params(wl.params, wl.max_range)
    for s, mean in zip(wl.states, (False, True, False, True)):
        g = s.x + np.array([2.0, -1.0, 0.5])
        r = O.combined_eval(om, s.x, s.xdot, 1024, p, g, ALPHA, BETA, metric_mean=mean)
        obs = O.raycast_eval(om, s.x, s.xdot, 1024, p, want_hits=False, want_per_ray=False)[0]
        fa = O.attractor(s.x, s.xdot, g, ALPHA, BETA, p.c)
        scale = 1.0 / 1024 if mean else 1.0                 # the ray policies' mean or sum
        assert np.allclose(r["sumA"], scale * obs["sumA"] + np.array([1, 0, 0, 1, 0, 1]),
                           rtol=1e-15)
        assert np.allclose(r["sumAf"], scale * obs["sumAf"] + fa, rtol=1e-15)
        S = r["sumA"]
        M = np.array([[S[0], S[1], S[2]], [S[1], S[3], S[4]], [S[2], S[4], S[5]]])
        res = M @ r["f"] - r["sumAf"]
        assert np.linalg.norm(res) <= 1e-12 * (np.linalg.norm(M) * np.linalg.norm(r["f"]) +
                                                np.linalg.norm(r["sumAf"]))
        assert r["eig"][0] >= 1.0 - 1e-12 and r["rank"] == 3


def _free_motion(k, dt):
    """Velocity and position after k semi-implicit Euler steps of v' = v + (alpha - beta v) dt,
    x' = x + v' dt from rest: v_k = (alpha/beta)(1 - q^k), q = 1 - beta dt."""
    q = 1.0 - BETA * dt
    v = [(ALPHA / BETA) * (1.0 - q ** i) for i in range(1, k + 1)]
    return v[-1], dt * sum(v)


def test_free_space_dynamics_geometric_series():
    om = O.OracleMap(empty_dense(n=32))
    p = O.make_params(W.PARAMS_STATIC_MAP, 2.0)
    rp = O.rollout_params(ALPHA, BETA, 0.01, 0.1, 1000, 10, 256)
    x0 = np.array([0.45, 1.6, 1.6])
    goal = x0 + np.array([1e6, 0.0, 0.0])
    st = O.rollout(om, p, rp, x0, np.zeros(3), goal, steps=100)
    v, dx = _free_motion(100, 0.01)
    assert st["status"] == O.ROLL_RUNNING and st["steps"] == 100
    assert st["xdot"][0] == pytest.approx(v, rel=1e-12)
    assert st["x"][0] - x0[0] == pytest.approx(dx, rel=1e-12)
    assert st["x"][1] == x0[1] and st["x"][2] == x0[2] and st["xdot"][1] == 0.0
    assert st["path_length"] == pytest.approx(dx, rel=1e-12)
    assert st["smoothness"] > 1.0 - 1e-7 and st["smooth_n"] == 9


def test_terminal_events_at_predicted_steps():
    vs = 0.1
    n = 64
    occ = np.zeros((n, n, n), np.uint8)
    occ[:, :, 40] = 1                                   # wall: voxel column x = 40 (x in [4.0, 4.1) m)
    wall = W.DenseMap(occ, vs, np.zeros(3))
    quiet = dict(W.PARAMS_STATIC_MAP, eta_rep=0.0, eta_damp=0.0)   # no obstacle forces
    p = O.make_params(quiet, 3.0)
    x0 = np.array([1.05, 3.2, 3.2])
    goal = np.array([1e6, 3.2, 3.2])
    dt = 0.01
    rp = O.rollout_params(ALPHA, BETA, dt, 0.1, 100000, 10, 256)
    st = O.rollout(O.OracleMap(wall), p, rp, x0, np.zeros(3), goal)
    k_wall = next(k for k in range(1, 10000) if x0[0] + _free_motion(k, dt)[1] >= 4.0)
    assert st["status"] == O.ROLL_COLLIDED and st["steps"] == k_wall
    # the same run without the wall leaves the 6.4 m grid
    st = O.rollout(O.OracleMap(empty_dense(n=n)), p, rp, x0, np.zeros(3), goal)
    k_out = next(k for k in range(1, 10000) if x0[0] + _free_motion(k, dt)[1] >= 6.4)
    assert st["status"] == O.ROLL_LEFT_MAP and st["steps"] == k_out
    # a robot at rest on its goal reaches it in one step; a far goal times out
    st = O.rollout(O.OracleMap(empty_dense(n=n)), p, rp, x0, np.zeros(3), x0)
    assert st["status"] == O.ROLL_REACHED and st["steps"] == 1
    rp5 = O.rollout_params(ALPHA, BETA, dt, 0.1, 5, 10, 256)
    st = O.rollout(O.OracleMap(empty_dense(n=n)), p, rp5, x0, np.zeros(3), goal)
    assert st["status"] == O.ROLL_TIMEOUT and st["steps"] == 5


def test_straight_run_reaches_goal_on_the_line():
    om = O.OracleMap(empty_dense(n=64))
    p = O.make_params(W.PARAMS_STATIC_MAP, 3.0)
    rp = O.rollout_params(ALPHA, BETA, 0.01, 0.05, 3000, 10, 64)
    x0 = np.array([1.0, 1.0, 1.0])
    goal = np.array([5.0, 4.0, 1.0])
    st, path = O.rollout(om, p, rp, x0, np.zeros(3), goal, want_path=True)
    assert st["status"] == O.ROLL_REACHED
    u = (goal - x0) / np.linalg.norm(goal - x0)
    off = path - x0 - np.outer((path - x0) @ u, u)          # distance from the start-goal line
    assert np.abs(off).max() < 1e-9 and np.all(path[:, 2] == 1.0)
    assert st["smoothness"] > 1.0 - 1e-6
