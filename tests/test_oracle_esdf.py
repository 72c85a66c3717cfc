"""Pins for the oracle's ESDF policy (Sec. III-D): the exact distance to the closest obstacle
of a union of spheres and boxes, its gradient, and the obstacle policy evaluated on them.

Checked against: hand-computed distances and gradients, brute-force sampling of the
primitives' surfaces, finite differences of the distance, the unit rate of the distance
along its gradient, the map generator's own signed-distance code (written for building the
voxel maps), the union as a minimum of single-primitive queries, the policy's special cases
(moving away, out of radius, no obstacle: the attractor alone) and a rollout that must equal
the raycasting policy's in an empty scene."""
import numpy as np

from paper_2301_08068_gb300 import workloads as W


def prims(orc, *specs):
    return orc.prims_array([W.Primitive(k, np.asarray(c, float), np.asarray(s, float))
                            for k, c, s in specs])


def test_hand_values(orc):
    pr = prims(orc, ("sphere", [0, 0, 0], [1.0]), ("box", [5, 0, 0], [1, 2, 3]))
    d, g, i = orc.esdf_query(pr, [0, 3, 4])          # |(0,3,4)| - 1 = 4, away from the centre
    assert (d, i) == (4.0, 0) and np.allclose(g, [0, 0.6, 0.8], atol=1e-15)
    d, g, i = orc.esdf_query(pr, [9, 6, 0])          # box corner region: (3, 4, 0) outside
    assert (d, i) == (5.0, 1) and np.allclose(g, [0.6, 0.8, 0], atol=1e-15)
    d, g, i = orc.esdf_query(pr, [5.5, 0, 0])        # inside the box: distance 0, nearest face +x
    assert (d, i) == (0.0, 1) and np.array_equal(g, [1.0, 0, 0])
    d, g, i = orc.esdf_query(pr, [5, -1.5, 0.2])     # inside, nearest face -y (0.5 away)
    assert d == 0.0 and np.array_equal(g, [0, -1.0, 0])
    d, g, i = orc.esdf_query(pr[:0], [1, 2, 3])      # no obstacle
    assert d == np.inf and i == -1 and np.all(g == 0)


def _surface_samples(pr, n=20000):
    """Points on the surface of one primitive: a Fibonacci lattice of a sphere, a grid on
    each face of a box; with the largest distance from any surface point to its nearest
    sample (a bound on the sampling error)."""
    c, s = pr["center"], pr["size"]
    if pr["kind"] == 0:
        k = np.arange(n) + 0.5
        z = 1 - 2 * k / n
        phi = np.pi * (1 + 5 ** 0.5) * k
        rr = np.sqrt(1 - z * z)
        pts = c + s[0] * np.stack([rr * np.cos(phi), rr * np.sin(phi), z], 1)
        return pts, 2.5 * s[0] * np.sqrt(4 * np.pi / n)
    m = 60
    faces = []
    for a in range(3):
        b, e = [x for x in range(3) if x != a]
        u, v = np.meshgrid(np.linspace(-s[b], s[b], m), np.linspace(-s[e], s[e], m))
        for sg in (-1, 1):
            p = np.zeros((m * m, 3))
            p[:, a] = sg * s[a]
            p[:, b] = u.ravel()
            p[:, e] = v.ravel()
            faces.append(c + p)
    step = 2 * s.max() / (m - 1)
    return np.concatenate(faces), step


def test_distance_against_sampled_surfaces(orc):
    rng = np.random.default_rng(5)
    specs = [("sphere", rng.uniform(0, 6, 3), [rng.uniform(0.3, 1.5)]) for _ in range(4)]
    specs += [("box", rng.uniform(0, 6, 3), rng.uniform(0.2, 1.2, 3)) for _ in range(4)]
    pr = prims(orc, *specs)
    samples, gaps = zip(*(_surface_samples(p) for p in pr))
    allp = np.concatenate(samples)
    gap = max(gaps)
    pts = rng.uniform(-1, 7, (400, 3))
    n_out = 0
    for x in pts:
        d, g, i = orc.esdf_query(pr, x)
        inside = any(W.Primitive(k, np.asarray(c, float), np.asarray(s, float)).sdf(x) < 0
                     for k, c, s in specs)
        if inside:
            assert d == 0.0
            continue
        n_out += 1
        ds = np.min(np.linalg.norm(allp - x, axis=1))
        assert d <= ds + 1e-12                        # no sampled surface point is closer
        assert ds - d <= gap                          # and one is within the sampling gap
    assert n_out > 200


def test_gradient_is_the_distance_gradient(orc):
    """Away from the medial axis: central differences of d match the gradient, the gradient
    has unit length, and d grows at unit rate along it."""
    hs = W.hashed_scene((10.0, 10.0, 10.0), 0.1, 40, seed_index=31)[1]
    pr = orc.prims_array(hs)
    rng = np.random.default_rng(6)
    checked = 0
    for x in rng.uniform(0, 10, (600, 3)):
        d, g, i = orc.esdf_query(pr, x)
        if d < 0.05:
            continue
        # second-nearest primitive at least 0.05 farther: a unique nearest obstacle nearby
        dists = sorted(max(W.Primitive(p_.kind, p_.center, p_.size).sdf(x), 0) for p_ in hs)
        if dists[1] - dists[0] < 0.05:
            continue
        h = 1e-5
        fd = np.array([(orc.esdf_query(pr, x + h * e)[0] - orc.esdf_query(pr, x - h * e)[0])
                       / (2 * h) for e in np.eye(3)])
        assert np.abs(np.linalg.norm(g) - 1.0) < 1e-14
        assert np.allclose(fd, g, atol=2e-5), (x, fd, g)
        t = min(0.02, d / 2)
        assert abs(orc.esdf_query(pr, x + t * g)[0] - (d + t)) < 1e-12
        checked += 1
    assert checked > 200


def test_matches_the_map_generator_and_union(orc):
    """The scene's distance equals max(0, the map generator's signed distance) and the
    minimum over single-primitive queries, with the first minimising primitive reported."""
    hs = W.hashed_scene((10.0, 10.0, 10.0), 0.1, 40, seed_index=31)[1]
    pr = orc.prims_array(hs)
    rng = np.random.default_rng(7)
    pts = rng.uniform(0, 10, (300, 3))
    sdf = W.scene_sdf(hs, pts)
    for x, s in zip(pts, sdf):
        d, g, i = orc.esdf_query(pr, x)
        assert abs(d - max(s, 0.0)) <= 1e-12 * max(1.0, abs(s))
        singles = [orc.esdf_query(pr[j:j + 1], x)[0] for j in range(len(pr))]
        raw = [W.Primitive(p_.kind, p_.center, p_.size).sdf(x) for p_ in hs]
        assert d == min(singles)
        assert i == int(np.argmin(raw))


def _policy_params(orc, **kw):
    return orc.make_params(dict(W.PARAMS_STATIC_MAP, **kw), 10.0)


def test_policy_uses_the_query_as_one_ray(orc):
    """The obstacle part is the obstacle policy of Sec. III-C evaluated once, with d the
    distance, r the gradient, active iff xdot . r < 0: the same sums as the oracle's ray
    policy on that pair."""
    pr = prims(orc, ("sphere", [0, 0, 0], [1.0]))
    p = _policy_params(orc)
    x = np.array([0.0, 1.8, 0.6])
    xdot = np.array([0.3, -1.2, 0.1])
    res, q = orc.esdf_eval(pr, x, xdot, p)
    d, r = q[0], q[1:]
    f, A = orc.ray_policy(p, r, d, xdot, bool(xdot @ r < 0), d < p.r)
    assert np.array_equal(res["sumA"], np.asarray(A))
    Af = np.array([[A[0], A[1], A[2]], [A[1], A[3], A[4]], [A[2], A[4], A[5]]]) @ np.asarray(f)
    assert np.allclose(res["sumAf"], Af, rtol=1e-14)
    assert res["n_hits"] == 1 and res["n_active"] == 1 and res["rank"] == 1
    # rank one along r: the resolved force is f projected on r, pointing away (repulsive)
    assert np.allclose(np.cross(res["f"], r), 0, atol=1e-9 * np.linalg.norm(res["f"]))
    assert res["f"] @ r > 0


def test_policy_special_cases_reduce_to_the_attractor(orc):
    """Moving away from the obstacle, beyond the radius, or with no obstacle at all, the
    obstacle metric is 0 and Eq. (1) gives the attractor alone: f = f_a."""
    p = _policy_params(orc)
    sph = prims(orc, ("sphere", [0, 0, 0], [1.0]))
    goal = np.array([4.0, 5.0, 6.0])
    cases = [(sph, [0, 2.0, 0], [0, 0.7, 0.2]),       # moving away
             (sph, [0, 4.0, 0], [0, -2.0, 0]),        # d = 3 > r = 2.4
             (sph[:0], [1, 2, 3], [1, 1, 1])]         # no obstacle
    for pr, x, v in cases:
        res, _ = orc.esdf_eval(pr, x, v, p, goal=goal, alpha=10.0, beta=15.0)
        fa = orc.attractor(x, v, goal, 10.0, 15.0, p.c)
        assert np.allclose(res["f"], fa, rtol=1e-13, atol=1e-13)
        assert res["n_active"] == 0 and res["rank"] == 3


def test_rollout_equals_the_ray_rollout_in_an_empty_scene(orc):
    """With no obstacle both policies are the attractor alone: the ESDF rollout and the
    raycasting rollout in an empty map take identical steps."""
    hm = W.HashedMap(np.zeros((0, 3), np.int32), np.zeros((0, 512), np.float32), 0.1)
    om = orc.OracleMap(hm)
    p = _policy_params(orc)
    rp = orc.rollout_params(10.0, 15.0, 0.01, 0.2, 2000, 10, 64)
    x0, v0, goal = np.array([1.0, 1.0, 1.0]), np.array([0.5, 0.0, 0.0]), np.array([6.0, 4.0, 2.0])
    a = orc.esdf_rollout(om, prims(orc)[:0], p, rp, x0, v0, goal)
    b = orc.rollout(om, p, rp, x0, v0, goal)
    for k in ("x", "xdot"):
        assert np.array_equal(a[k], b[k])
    assert (a["status"], a["steps"]) == (b["status"], b["steps"])
    assert a["status"] == orc.ROLL_REACHED
