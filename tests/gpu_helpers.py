"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, run the
oracle on the same seeded inputs, and compare with the stated tolerances.

Tolerances (FP32 march and per-ray policy against the FP64 oracle; Sec. III-C and Eq. (1)):
  * hit records (status, voxel, steps, d, blocks): bit-exact -- both sides follow one fixed-point
    DDA specification and one FP32 recipe for d;
  * per-ray f_i: |f_gpu - f_orc| <= 1e-5 |f_orc| (Euclidean norms);
  * per-ray A_i on the map path: max|A_gpu - A_orc| <= 1e-5 max|A_orc| -- relative only (the
    2^-100 floor sits far below FP32's normal range against A's natural bound |A_ij| < 1, so
    it only excuses an FP32 underflow); the ray's direction and d are bit-identical on both
    sides, so nothing but the FP32 policy arithmetic differs.  Entries the oracle computes as
    exactly 0 (inactive rays, d >= r, misses) must be exactly 0;
  * per-point A_i of a LiDAR scan: the same relative bound plus `scan_abs_term`, derived from
    the one input the two sides do not share: the kernel forms the direction q/|q| and the
    range |q| in FP32, the oracle in FP64.  The term is the change of A_i over the box of
    (xdot.r, d) values those FP32 roundings allow, evaluated with the policy formulas;
  * sums: |sumA_gpu - sumA_orc| <= 1e-5 sum|A_i| per entry (plus the per-point terms of a
    scan), likewise for sum A f with |A_i f_i|;
  * eigenvalues of sum A: within the Frobenius norm of the entry bounds (Weyl) plus the error
    of the kernel's eigenvalue report (eig_tolerance): FP64 Rayleigh quotients of FP32
    Jacobi eigenvectors, accurate to r^2 / gap for an eigenvalue separated by gap from the
    others and to r inside a cluster, r = 4e-6 lambda_max bounding the residual of the
    FP32 eigenvectors (Jacobi stops at off-diagonal <= 1e-6 of the diagonal);
  * resolved f = (sum A)^+ sum A f: within max(1e-4 |f|, B), B the perturbation bound of
    the solve for the sums the kernel produced (checked above against their own tolerance):
    (|db| + |dS| |f|) / (lambda_k - |dS|) with dS, db twice the observed differences of the
    sums, plus the rotation of the kept eigenvectors (Davis-Kahan) below full rank,
    lambda_k the smallest kept eigenvalue.  For well-conditioned sums B is below 1e-4 |f|
    and the check is the stated 1e-4 relative; for ill-conditioned ones B is about
    cond(sum A) times the relative error of the sums, which the FP32 per-ray values set.
    Where an eigenvalue could cross the pseudo-inverse's 1e-12 lambda_max cut under that
    perturbation (every rank-deficient sum: FP32 per-ray values leave ~1e-8 lambda_max of
    noise where the FP64 oracle has ~1e-17), the rank and so f are not determined by the
    inputs at FP32 precision, and only the sums and eigenvalues are checked.
"""
import numpy as np

from paper_2301_08068_gb300 import rmp as R

REL = 1e-5          # per-ray and summed A, A f: the stated relative tolerance
REL_F = 1e-4        # resolved acceleration: the stated relative tolerance
UNDERFLOW = 2.0 ** -100


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def gpu_raycast(ctx: R.Context, map_id: int, x, xdot, n: int, params, want=True):
    torch = torch_cuda()
    hits = torch.empty(n * 24, dtype=torch.uint8, device="cuda") if want else None
    per = torch.empty(n * 9, dtype=torch.float32, device="cuda") if want else None
    res = R.rmp_raycast_eval(ctx.handle, map_id, x, xdot, n, params, hits=hits, per_ray=per)
    if not want:
        return res, None, None
    h = hits.cpu().numpy().view(R.HIT_DTYPE)
    p = per.cpu().numpy().reshape(n, 9).astype(np.float64)
    return res, h, p


def gpu_scan(ctx: R.Context, pts_np: np.ndarray, x, xdot, params):
    torch = torch_cuda()
    pts = torch.from_numpy(np.ascontiguousarray(pts_np, np.float32)).cuda()
    n = pts.shape[0]
    per = torch.empty(n * 9, dtype=torch.float32, device="cuda")
    res = R.rmp_scan_eval(ctx.handle, pts, x, xdot, params, per_ray=per)
    return res, per.cpu().numpy().reshape(n, 9).astype(np.float64)


def assert_hits_exact(g, o):
    assert np.array_equal(g["status"], o["status"]), np.nonzero(g["status"] != o["status"])[0][:10]
    assert np.array_equal(g["voxel"], o["voxel"])
    assert np.array_equal(g["steps"], o["steps"])
    assert np.array_equal(g["d"].view(np.uint32), o["d"].view(np.uint32))
    assert np.array_equal(g["blocks"], o["blocks"])


def _metric_scale(pd: dict, d, xr, active):
    """alpha = w_r(d) (z / h(z))^2 with z = |f_damp| = k_d (xdot.r)^2 (Sec. III-C): A_i =
    alpha r r^T.  Vectorised, FP64; used only to size the scan tolerance."""
    r, c = pd["r"], pd["c"]
    x = np.clip(d / r, 0.0, 1.0)
    w = (1.0 - x) ** 2 if pd.get("w_mode", 0) == 0 else 1.0 - 3.0 * x * x + 2.0 * x ** 3
    w = np.where(d < r, w, 0.0)
    kd = pd["eta_damp"] / (d / pd["nu_damp"] + pd["eps"])
    z = np.where(active, kd * xr * xr, 0.0)
    h = z + c * np.log1p(np.exp(-2.0 * c * z))
    return w * (z / h) ** 2


def scan_abs_term(points, x, xdot, pd: dict):
    """Per point, bounds on the change of f_i and of any entry of A_i over the (xdot.r, d)
    values that the kernel's FP32 direction and range can take: |dq| <= 2^-24 (|x| + |q|)
    from q = RN32(p - RN32(x)), the range within 2^-22 of |q| plus that, the direction
    q / d (correctly rounded divides of the rounded q by the rounded range) within
    1.5 2^-23 + 2 |dq| / d, so |d(xdot.r)| <= |xdot| (1.5 2^-23 + 2 |dq| / d).
    alpha is monotone in |xdot.r| and piecewise monotone in d, so its change is taken at
    the corners of that box; where |xdot.r| lies inside the box the activity decision may
    flip too.  Entries of r r^T are at most 1 in magnitude.  Returns (A term, f term)."""
    p = np.asarray(points, np.float64)
    x = np.asarray(x, np.float64)
    v = np.asarray(xdot, np.float64)
    q = p - x
    d = np.linalg.norm(q, axis=1)
    ok = np.isfinite(d) & (d > 0)
    d = np.where(ok, d, 1.0)
    u = q / d[:, None]
    xr = u @ v                                   # xdot . (direction to the point)
    dq = 2.0 ** -24 * (np.linalg.norm(x) + d)
    dd = dq + 2.0 ** -22 * d
    du = 1.5 * 2.0 ** -23 + 2.0 * dq / d
    dxr = np.linalg.norm(v) * du
    act = xr > 0
    base = _metric_scale(pd, d, np.abs(xr), act)
    worst = np.zeros_like(base)
    flip = np.abs(xr) <= dxr
    for sd in (-1.0, 1.0):
        dc = np.maximum(d + sd * dd, 1e-12)
        for sx in (-1.0, 1.0):
            xc = np.maximum(np.abs(xr) + sx * dxr, 0.0)
            worst = np.maximum(worst, np.abs(_metric_scale(pd, dc, xc, act) - base))
        on = _metric_scale(pd, dc, np.abs(xr) + dxr, np.ones_like(act))
        worst = np.where(flip, np.maximum(worst, np.maximum(on, base)), worst)
    a_term = np.where(ok, worst, 0.0)
    # f = (f_rep + k_d m) r: k_d at the shorter range, m = (xdot.r)^2 over the box, and
    # the direction error times |f|
    kd = pd["eta_damp"] / (np.maximum(d - dd, 1e-12) / pd["nu_damp"] + pd["eps"])
    frep = pd["eta_rep"] * np.exp(-(d - dd) / pd["nu_rep"])
    m_hi = (np.abs(xr) + dxr) ** 2
    f_hi = frep + kd * m_hi
    f_term = kd * (m_hi - xr * xr) + frep * (np.exp(dd / pd["nu_rep"]) - 1.0) + f_hi * du
    return a_term, np.where(ok, f_term, 0.0)


def assert_per_ray_close(g, o, abs_term=None):
    """Per-ray f_i and A_i (rows: f 3, A xx xy xz yy yz zz) against the oracle's; abs_term
    (scans only) is the pair (A term, f term) of scan_abs_term."""
    fg, fo = g[:, :3], o[:, :3]
    ag, ao = g[:, 3:], o[:, 3:]
    ef = np.linalg.norm(fg - fo, axis=1)
    nf = np.linalg.norm(fo, axis=1)
    ftol = REL * nf + UNDERFLOW
    if abs_term is not None:
        ftol = ftol + abs_term[1]
    assert np.all(ef <= ftol), (np.max(ef / np.maximum(nf, 1e-30)))
    ea = np.max(np.abs(ag - ao), axis=1)
    na = np.max(np.abs(ao), axis=1)
    tol = REL * na + UNDERFLOW
    if abs_term is not None:
        tol = tol + abs_term[0]
    bad = ea > tol
    assert not np.any(bad), ("A_i", int(np.argmax(bad)), float(np.max((ea - tol))),
                             float(np.max(ea / np.maximum(na, 1e-300))))
    assert np.all(ag[ao == 0.0] == 0.0)


def _full(a):
    return np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])


def abs_Af(per):
    """|A_i f_i| per ray (n x 3) from per-ray rows (f: 3, A: xx xy xz yy yz zz)."""
    f, a = per[:, :3], per[:, 3:]
    return np.abs(np.stack([a[:, 0] * f[:, 0] + a[:, 1] * f[:, 1] + a[:, 2] * f[:, 2],
                            a[:, 1] * f[:, 0] + a[:, 3] * f[:, 1] + a[:, 4] * f[:, 2],
                            a[:, 2] * f[:, 0] + a[:, 4] * f[:, 1] + a[:, 5] * f[:, 2]], axis=1))


def abs_sums(per_orc):
    """(sum |A_i| per entry (6), sum |A_i f_i| per entry (3)) of the oracle's per-ray rows."""
    return np.abs(per_orc[:, 3:]).sum(axis=0), abs_Af(per_orc).sum(axis=0)


def sum_tolerances(o, per_orc=None, abs_term=None, sums=None):
    """Entry bounds (6 for sum A, 3 for sum A f) of the summed values, from the oracle's
    per-ray rows or their abs_sums.  Without either, the oracle's largest summed entry
    stands in for sum |A_i| (a looser bound)."""
    if sums is not None and per_orc is None:
        return REL * sums[0] + UNDERFLOW, REL * sums[1] + UNDERFLOW
    if per_orc is not None:
        A, Af = abs_sums(per_orc)
        tolA = REL * A + UNDERFLOW
        tolAf = REL * Af + UNDERFLOW
        if abs_term is not None:
            # |d(A f)| <= |dA| |f| + |A| |df| per ray, entries of A at most |A_i|'s largest
            a_t, f_t = abs_term
            fmax = np.linalg.norm(per_orc[:, :3], axis=1)
            amax = np.abs(per_orc[:, 3:]).max(axis=1)
            tolA = tolA + a_t.sum()
            tolAf = tolAf + 3.0 * ((a_t * (fmax + f_t)) + amax * f_t).sum()
    else:
        tolA = np.full(6, REL * max(np.abs(o["sumA"]).max(), 1e-300))
        tolAf = np.full(3, REL * max(np.abs(o["sumAf"]).max(), 1e-300))
    return tolA, tolAf


def eig_tolerance(lam, dS):
    """Per-eigenvalue tolerance of the reported eigenvalues (ascending oracle values lam):
    dS (Weyl, from the sum entries) + min(r, r^2 / gap_i), r = 4e-6 max|lambda|."""
    lam = np.asarray(lam, np.float64)
    r = 4e-6 * np.max(np.abs(lam))
    tol = np.empty(3)
    for i in range(3):
        gap = min(abs(lam[i] - lam[j]) for j in range(3) if j != i)
        tol[i] = dS * (1.0 + 1e-9) + (min(r, r * r / gap) if gap > 0 else r) + 1e-300
    return tol


def f_bound(o, dS, db):
    """Perturbation bound of f = S^+ b when the sum matrix moves by at most dS (2-norm) and
    b by at most db, or None where the pseudo-inverse's rank decision (eigenvalues above
    1e-12 lambda_max) could change under that perturbation -- f is then not determined.
    Full rank: |df| <= (db + dS |f|) / (lambda_min - dS).  Lower rank: that on the kept
    eigenvalues plus the rotation of their eigenvectors (Davis-Kahan: angle <= dS / gap)."""
    lam = np.asarray(o["eig"], np.float64)
    lmax = np.max(np.abs(lam))
    if lmax <= 0 or o["rank"] == 0:
        return 0.0
    kept = lam[lam > 1e-12 * lmax]
    disc = lam[lam <= 1e-12 * lmax]
    lam_k = kept.min()
    if lam_k - dS <= 1e-12 * (lmax + dS):
        return None
    if disc.size and disc.max() + dS > 1e-12 * (lmax - dS):
        return None
    nf = np.linalg.norm(o["f"])
    bound = (db + dS * nf) / (lam_k - dS)
    if disc.size:
        gap = lam_k - disc.max()
        bound += 2.0 * dS / (gap - dS) * np.linalg.norm(o["sumAf"]) / (lam_k - dS)
    return bound


def observed_f_bound(g, o):
    """f_bound for the sums the kernel actually produced: twice the observed differences
    of sum A (Frobenius) and sum A f from the oracle's (a margin for second-order terms),
    plus the FP64 resolve's own rounding (1e-13 relative, far above FP64's 1e-16 times the
    few operations of the 3 x 3 solve)."""
    lam = np.abs(np.asarray(o["eig"], np.float64))
    dS = 2.0 * np.linalg.norm(_full(np.asarray(g["sumA"]) - o["sumA"]), "fro") + 1e-13 * lam.max()
    db = 2.0 * np.linalg.norm(np.asarray(g["sumAf"]) - o["sumAf"]) + \
        1e-13 * np.linalg.norm(o["sumAf"])
    return f_bound(o, dS, db)


def assert_result_close(g, o, per_orc=None, abs_term=None, sums=None):
    assert g["status"] == 0
    assert g["n_rays"] == o["n_rays"] and g["n_hits"] == o["n_hits"]
    assert g["n_active"] == o["n_active"]
    tolA, tolAf = sum_tolerances(o, per_orc, abs_term, sums)
    assert np.all(np.abs(g["sumA"] - o["sumA"]) <= tolA), (g["sumA"], o["sumA"], tolA)
    assert np.all(np.abs(g["sumAf"] - o["sumAf"]) <= tolAf), (g["sumAf"], o["sumAf"], tolAf)
    lam = o["eig"]
    dS = np.linalg.norm(_full(tolA), "fro")
    assert np.all(np.abs(g["eig"] - lam) <= eig_tolerance(lam, dS)), (g["eig"], lam, dS)
    b = observed_f_bound(g, o)
    if b is not None:
        nf = np.linalg.norm(o["f"])
        assert g["rank"] == o["rank"], (g["rank"], o["rank"])
        err = np.linalg.norm(g["f"] - o["f"])
        assert err <= max(REL_F * nf, b) + 1e-300, (g["f"], o["f"], err, REL_F * nf, b)
    if o["n_active"] == 0:
        assert np.all(g["f"] == 0.0) and np.all(g["sumA"] == 0.0)


def f_error_report(g, o):
    """(relative error of f, cond(sum A), the observed-sum bound relative to |f|) for the
    printed precision tables; NaN where f is not determined."""
    lam = np.asarray(o["eig"], np.float64)
    nf = max(np.linalg.norm(o["f"]), 1e-300)
    cond = (lam.max() / lam.min()) if lam.min() > 0 else np.inf
    b = observed_f_bound(g, o)
    return (float(np.linalg.norm(g["f"] - o["f"]) / nf), float(cond),
            float(b / nf) if b is not None else float("nan"))
