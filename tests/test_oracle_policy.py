"""Pins for the oracle's obstacle policy (Sec. III-C), ray policy sum (Eq.
raytracing_policy) and resolve (Eq. 1).

Checked against: the paper's stated special values (w_r(0) = 1, w_r(r) = 0, zero metric
for rays pointing away from the velocity, rank-1 metric stretched along the obstacle
direction), limits of the soft normalisation, scaling laws of f_rep and f_damp,
numpy's pseudo-inverse and eigenvalues, exactly rounded sums (math.fsum), and the
closed form of a robot at the centre of a hollow sphere (1-D quadrature by scipy).
"""
import math

import numpy as np
import pytest

from paper_2301_08068_gb300 import workloads as W


def params(orc, **kw):
    d = dict(W.PARAMS_STATIC_MAP)
    d.update(kw)
    return orc.make_params(d, kw.get("max_range", 10.0))


def full(A6):
    a = np.asarray(A6, np.float64)
    return np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])


R_UNIT = np.array([0.6, -0.48, 0.64])            # unit vector away from the obstacle


# ----------------------------------------------------------------------------- per-ray policy
@pytest.mark.parametrize("w_mode", [0, 1])
def test_weight_endpoints_and_midpoint(orc, w_mode):
    """With c -> 0 the soft normalisation is a plain normalisation, so trace(A) = w_r(d)."""
    p = params(orc, c=1e-9, w_mode=w_mode)
    xdot = -5.0 * R_UNIT                      # head-on: moving towards the obstacle
    tr = {}
    for d in (0.0, 0.5 * p.r, 0.999999 * p.r):
        f, A = orc.ray_policy(p, R_UNIT, d, xdot, True, True)
        tr[d] = np.trace(full(A))
    assert abs(tr[0.0] - 1.0) < 1e-9                     # w_r(0) = 1
    mid = 0.25 if w_mode == 0 else 0.5                   # printed quadratic / cubic spline
    assert abs(tr[0.5 * p.r] - mid) < 1e-9
    assert tr[0.999999 * p.r] < 1e-10                    # -> w_r(r) = 0
    f, A = orc.ray_policy(p, R_UNIT, 1.5 * p.r, xdot, True, False)
    assert np.all(np.asarray(A) == 0.0)                  # 0 beyond the radius


def test_weight_flat_at_the_radius(orc):
    """The weight's slope vanishes at d = r (both readings); the cubic is also flat at 0."""
    for w_mode in (0, 1):
        p = params(orc, c=1e-9, w_mode=w_mode)
        xdot = -5.0 * R_UNIT
        h = 1e-4 * p.r
        w = lambda d: np.trace(full(orc.ray_policy(p, R_UNIT, d, xdot, True, True)[1]))
        assert abs(w(p.r - h) - w(p.r - 2 * h)) < 1e-7
        if w_mode == 1:
            assert abs(w(h) - w(0.0)) < 1e-7


@pytest.mark.parametrize("w_mode", [0, 1])
def test_weight_relative_accuracy_near_the_radius(orc, w_mode):
    """w_r(d) keeps its relative accuracy as d -> r: against the exact rational value of the
    printed quadratic (or the cubic) at the FP64 d and r, for 1 - d/r from 1e-1 to 1e-9.
    (c -> 0 and a head-on velocity make trace(A) = w_r(d) to ~1e-18.)"""
    from fractions import Fraction as Fr
    p = params(orc, c=1e-15, w_mode=w_mode)
    xdot = -5.0 * R_UNIT
    for k in range(1, 10):
        d = p.r * (1.0 - 10.0 ** -k)
        x = Fr(d) / Fr(p.r)
        exact = x * x - 2 * x + 1 if w_mode == 0 else 1 - 3 * x * x + 2 * x * x * x
        tr = np.trace(full(orc.ray_policy(p, R_UNIT, d, xdot, True, True)[1]))
        assert abs(Fr(tr) - exact) <= Fr(1, 10 ** 12) * exact, (k, tr, float(exact))


def test_metric_rank_one_along_obstacle_direction(orc):
    p = params(orc)
    rng = np.random.default_rng(3)
    for _ in range(20):
        xdot = rng.normal(size=3) * 2
        d = rng.uniform(0, p.r)
        f, A = orc.ray_policy(p, R_UNIT, d, xdot, bool(xdot @ -R_UNIT > 0), True)
        M = full(A)
        assert np.allclose(M, M.T)
        assert np.allclose(M @ R_UNIT, np.trace(M) * R_UNIT, atol=1e-12)
        assert np.linalg.eigvalsh(M).min() >= -1e-14


def test_zero_metric_when_moving_away(orc):
    p = params(orc)
    xdot = 3.0 * R_UNIT                            # moving away from the obstacle
    f, A = orc.ray_policy(p, R_UNIT, 0.7, xdot, False, True)
    assert np.all(np.asarray(A) == 0.0)
    f0, A0 = orc.ray_policy(p, R_UNIT, 0.7, np.zeros(3), False, True)
    assert np.all(np.asarray(A0) == 0.0) and np.allclose(f, f0)


def test_repulsive_term_halves_every_ln2_nu(orc):
    p = params(orc)
    d = p.nu_rep * math.log(2.0)
    f, _ = orc.ray_policy(p, R_UNIT, d, np.zeros(3), False, True)
    assert abs(f @ R_UNIT - p.eta_rep / 2) < 1e-12 * p.eta_rep
    assert np.allclose(np.cross(f, R_UNIT), 0, atol=1e-12)           # along r: repulsive
    f0, _ = orc.ray_policy(p, R_UNIT, 0.0, np.zeros(3), False, True)
    assert abs(f0 @ R_UNIT - p.eta_rep) < 1e-12 * p.eta_rep


def test_damping_quadratic_in_speed_and_inverse_in_distance(orc):
    p = params(orc, eta_rep=0.0)
    fd = lambda V, d: orc.ray_policy(p, R_UNIT, d, -V * R_UNIT, True, True)[0]
    assert np.allclose(fd(2.0, 0.9), 4.0 * fd(1.0, 0.9), rtol=1e-13)
    ratio = (fd(1.0, 0.0) @ R_UNIT) / (fd(1.0, p.nu_damp) @ R_UNIT)
    assert abs(ratio - (1.0 + p.eps) / p.eps) < 1e-9 * ratio
    # g_obs depends on the velocity's component along r only
    tang = np.cross(R_UNIT, [0, 0, 1.0])
    assert np.allclose(fd(1.0, 0.9), orc.ray_policy(p, R_UNIT, 0.9, -R_UNIT + 7 * tang, True, True)[0])


def test_soft_normalisation_limits(orc):
    """h(z) = z + c log(1 + exp(-2cz)) -> c ln 2 as z -> 0 and -> z as z -> inf."""
    for c in (0.2, 1.0):
        p = params(orc, eta_rep=0.0, c=c)
        for V, expect in ((1e-7, None), (300.0, 1.0)):
            f, A = orc.ray_policy(p, R_UNIT, 0.0, -V * R_UNIT, True, True)
            z = np.linalg.norm(f)                   # |f_damp| (f_rep = 0)
            tr = np.trace(full(A))                  # w = 1 at d = 0, so trace = |s|^2
            if expect is None:
                assert abs(math.sqrt(tr) - z / (c * math.log(2))) < 1e-6 * z / (c * math.log(2))
            else:
                assert abs(tr - 1.0) < 1e-6


def test_active32_decision(orc):
    u = np.array([0.6, -0.48, 0.64], np.float32)
    assert orc.active32(np.array([1.0, 0, 0]), u)
    assert not orc.active32(np.array([-1.0, 0, 0]), u)
    assert not orc.active32(np.zeros(3), u)


# ----------------------------------------------------------------------------- resolve
def random_psd(rng, rank):
    B = rng.normal(size=(3, rank))
    return B @ B.T


def six(M):
    return np.array([M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]])


@pytest.mark.parametrize("rank", [3, 2, 1])
def test_pinv_matches_numpy(orc, rank):
    rng = np.random.default_rng(rank)
    for _ in range(50):
        M = random_psd(rng, rank) * 10 ** rng.uniform(-3, 3)
        P, eig, rk = orc.pinv3(six(M))
        ref = np.linalg.pinv(M, rcond=1e-12, hermitian=True)
        assert np.allclose(full(P), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
        assert np.allclose(eig, np.linalg.eigvalsh(M), atol=1e-12 * np.abs(M).max())
        assert rk == rank


def test_pinv_closed_forms(orc):
    s = np.array([0.3, -1.2, 2.0])
    P, eig, rk = orc.pinv3(six(np.outer(s, s)))
    assert rk == 1 and np.allclose(full(P), np.outer(s, s) / np.dot(s, s) ** 2, rtol=1e-12)
    P, eig, rk = orc.pinv3(six(4.0 * np.eye(3)))
    assert rk == 3 and np.allclose(full(P), np.eye(3) / 4.0, rtol=1e-15)
    P, eig, rk = orc.pinv3(np.zeros(6))
    assert rk == 0 and np.all(P == 0)


# ----------------------------------------------------------------------------- sums
def test_map_eval_sums_equal_exactly_rounded_sums(orc):
    wl = W.dense_box_workload()
    om = orc.OracleMap(wl.map)
    p = orc.make_params(wl.params, wl.max_range)
    res, hits, per = orc.raycast_eval(om, wl.states[0].x, wl.states[0].xdot, wl.n_rays, p)
    A = per[:, 3:]
    Af = np.einsum("nij,nj->ni", np.stack([full(a) for a in A]), per[:, :3])
    for k in range(6):
        assert abs(res["sumA"][k] - math.fsum(A[:, k])) <= 1e-14 * np.abs(A[:, k]).sum()
    for k in range(3):
        assert abs(res["sumAf"][k] - math.fsum(Af[:, k])) <= 1e-14 * np.abs(Af[:, k]).sum()
    ref = np.linalg.pinv(full(res["sumA"]), rcond=1e-12, hermitian=True) @ res["sumAf"]
    assert np.allclose(res["f"], ref, rtol=1e-9)
    assert res["n_hits"] == int((hits["status"] == orc.HIT).sum())
    assert np.all(per[hits["status"] != orc.HIT] == 0)
    assert np.linalg.eigvalsh(full(res["sumA"])).min() >= -1e-12 * np.abs(res["sumA"]).max()


def test_concurrent_evaluations_equal_serial_ones(orc):
    """The all-cores CPU baseline runs the oracle on several host threads at once; its
    evaluation keeps no shared state, so each thread's result is the serial one bit for bit."""
    from concurrent.futures import ThreadPoolExecutor
    wl = W.hashed_workload(n_states=8)
    om = orc.OracleMap(wl.map)
    p = orc.make_params(wl.params, wl.max_range)

    def run(s):
        return orc.raycast_eval(om, s.x, s.xdot, 2048, p, want_hits=False, want_per_ray=False)[0]

    serial = [run(s) for s in wl.states]
    with ThreadPoolExecutor(4) as ex:
        threaded = list(ex.map(run, wl.states))
    for a, b in zip(serial, threaded):
        for k in ("sumA", "sumAf", "f", "eig"):
            assert np.array_equal(a[k], b[k]), k
        assert (a["n_hits"], a["n_active"], a["rank"]) == (b["n_hits"], b["n_active"], b["rank"])


def test_zero_velocity_gives_zero_policy(orc):
    wl = W.hashed_workload()
    om = orc.OracleMap(wl.map)
    p = orc.make_params(wl.params, wl.max_range)
    res, _, _ = orc.raycast_eval(om, wl.states[0].x, np.zeros(3), 4096, p)
    assert res["n_hits"] > 0 and res["n_active"] == 0
    assert np.all(res["sumA"] == 0) and np.all(res["f"] == 0) and res["rank"] == 0


def test_empty_map_gives_zero_policy(orc):
    hm = W.HashedMap(np.zeros((0, 3), np.int32), np.zeros((0, 512), np.float32), 0.1)
    p = params(orc)
    res, hits, _ = orc.raycast_eval(orc.OracleMap(hm), np.array([1.0, 2, 3]), np.array([1.0, 0, 0]),
                                    2048, p)
    assert res["n_hits"] == 0 and np.all(res["f"] == 0) and np.all(res["sumA"] == 0)
    assert np.all(hits["status"] == orc.MISS_RANGE)


def test_scan_permutation_invariance_and_skips(orc):
    sw = W.lidar_workload()
    p = orc.make_params(sw.params, sw.max_range)
    res, per = orc.scan_eval(sw.points, sw.x, sw.xdot, p)
    perm = np.random.default_rng(0).permutation(sw.points.shape[0])
    res2, _ = orc.scan_eval(sw.points[perm], sw.x, sw.xdot, p)
    assert np.allclose(res2["f"], res["f"], rtol=1e-12)
    assert np.allclose(res2["sumA"], res["sumA"], rtol=1e-12)
    finite = np.isfinite(sw.points).all(axis=1)
    rng_ = np.linalg.norm(sw.points.astype(np.float64), axis=1)
    expect = finite & (rng_ >= p.min_range) & (rng_ <= p.max_range)
    assert res["n_hits"] == int(expect.sum())
    assert np.all(per[~expect] == 0)
    # a point closer than min_range, or beyond max_range, changes nothing
    extra = np.array([[0.05, 0.0, 0.0], [40.0, 0.0, 0.0], [np.nan, 1.0, 1.0]], np.float32)
    res3, _ = orc.scan_eval(np.concatenate([sw.points, extra]), sw.x, sw.xdot, p)
    assert np.all(res3["f"] == res["f"]) and res3["n_hits"] == res["n_hits"]


# ----------------------------------------------------------------------------- closed form
def sphere_closed_form(p, R, V):
    """Robot at the centre of a hollow sphere of radius R < r, velocity V e.  With
    mu = cos(angle to e), only mu > 0 is active, |f_damp| = k V^2 mu^2 with
    k = eta_damp / (R/nu_damp + eps), alpha = |f_damp| / h(|f_damp|), beta = eta_rep
    exp(-R/nu_rep).  For directions spread evenly over the sphere,
      f = -e  int_0^1 alpha^2 (beta + k V^2 mu^2) mu dmu / int_0^1 alpha^2 mu^2 dmu,
      e^T (sum A) e = w_r(R) (n/2) int_0^1 alpha^2 mu^2 dmu."""
    from scipy.integrate import quad
    k = p.eta_damp / (R / p.nu_damp + p.eps)
    beta = p.eta_rep * math.exp(-R / p.nu_rep)
    h = lambda z: z + p.c * math.log1p(math.exp(-2 * p.c * z))
    alpha = lambda mu: (k * V * V * mu * mu) / h(k * V * V * mu * mu)
    num = quad(lambda mu: alpha(mu) ** 2 * (beta + k * V * V * mu * mu) * mu, 0, 1, epsabs=0, epsrel=1e-13)[0]
    den = quad(lambda mu: alpha(mu) ** 2 * mu * mu, 0, 1, epsabs=0, epsrel=1e-13)[0]
    return num / den, den


@pytest.mark.parametrize("n,tol", [(4096, 3e-3), (65536, 5e-4)])
@pytest.mark.parametrize("which", ["static", "lidar"])
def test_centred_sphere_closed_form(orc, n, tol, which):
    pytest.importorskip("scipy")
    base = W.PARAMS_STATIC_MAP if which == "static" else W.PARAMS_LIDAR
    p = orc.make_params(dict(base, min_range=0.0), 30.0)
    R = 0.6 * p.r
    V = 1.7
    e = np.array([0.36, 0.48, 0.8])
    pts = W.sphere_lattice_scan(n, R)
    res, _ = orc.scan_eval(pts, np.zeros(3), V * e, p)
    mag, den = sphere_closed_form(p, R, V)
    f = res["f"]
    assert abs(f @ e + mag) <= tol * mag                         # -mag along e
    assert np.linalg.norm(f - (f @ e) * e) <= tol * mag          # nothing transverse
    w = (1 - R / p.r) ** 2
    eAe = e @ full(res["sumA"]) @ e
    assert abs(eAe - w * n / 2 * den) <= tol * w * n / 2 * den   # pins w_r(R) too


def test_symmetric_room_pushes_back(orc):
    """Robot at the centre of a closed cubic room moving along +x: the policy decelerates
    along -x and the transverse parts stay small."""
    occ = np.zeros((41, 41, 41), np.uint8)
    occ[0, :, :] = occ[-1, :, :] = occ[:, 0, :] = occ[:, -1, :] = occ[:, :, 0] = occ[:, :, -1] = 1
    m = W.DenseMap(occ, 0.05, np.zeros(3))
    p = params(orc, max_range=5.0)
    x = np.array([20.5, 20.5, 20.5]) * 0.05
    res, hits, _ = orc.raycast_eval(orc.OracleMap(m), x, np.array([2.0, 0, 0]), 16384, p)
    assert res["n_hits"] == 16384
    f = res["f"]
    assert f[0] < 0 and abs(f[1]) < 0.02 * abs(f[0]) and abs(f[2]) < 0.02 * abs(f[0])
