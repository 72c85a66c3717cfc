"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, run the
oracle on the same seeded inputs, and compare with the stated tolerances.

Tolerances (FP32 march and per-ray policy against the FP64 oracle):
  * hit records (status, voxel, steps, d, blocks): bit-exact -- both sides follow one fixed-point
    DDA specification and one FP32 recipe for d;
  * per-ray f_i: |f_gpu - f_orc| <= 1e-5 |f_orc| (Euclidean norms);
  * per-ray A_i: max|A_gpu - A_orc| <= 1e-5 max|A_orc| + 1e-6.  The absolute term is 1e-6
    of A's natural bound (A = w_r s s^T with w_r <= 1 and |s| < 1): it covers FP32 rounding
    of the scan directions (q/|q| to 1 ulp per component) that feeds xdot.r; entries the
    oracle computes as exactly 0 (inactive rays, d >= r, misses) must be exactly 0;
  * sums: |sumA_gpu - sumA_orc| <= 1e-5 sum|A_i| + 1e-6 n_active (per entry), likewise for
    sum A f with the per-ray |A_i f_i|;
  * resolved f: |f_gpu - f_orc| <= 1e-4 |f_orc| when cond(sum A) <= 1e4.
"""
import numpy as np

from paper_2301_08068_gb300 import rmp as R


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


def assert_per_ray_close(g, o):
    fg, fo = g[:, :3], o[:, :3]
    ag, ao = g[:, 3:], o[:, 3:]
    ef = np.linalg.norm(fg - fo, axis=1)
    nf = np.linalg.norm(fo, axis=1)
    assert np.all(ef <= 1e-5 * nf + 1e-30), (np.max(ef / np.maximum(nf, 1e-30)))
    ea = np.max(np.abs(ag - ao), axis=1)
    na = np.max(np.abs(ao), axis=1)
    assert np.all(ea <= 1e-5 * na + 1e-6), np.max(ea - 1e-5 * na)
    assert np.all(ag[ao == 0.0] == 0.0)


def _full(a):
    return np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])


def abs_Af(per):
    """|A_i f_i| per ray (n x 3) from per-ray rows (f: 3, A: xx xy xz yy yz zz)."""
    f, a = per[:, :3], per[:, 3:]
    return np.abs(np.stack([a[:, 0] * f[:, 0] + a[:, 1] * f[:, 1] + a[:, 2] * f[:, 2],
                            a[:, 1] * f[:, 0] + a[:, 3] * f[:, 1] + a[:, 4] * f[:, 2],
                            a[:, 2] * f[:, 0] + a[:, 4] * f[:, 1] + a[:, 5] * f[:, 2]], axis=1))


def assert_result_close(g, o, per_orc=None):
    assert g["status"] == 0
    assert g["n_rays"] == o["n_rays"] and g["n_hits"] == o["n_hits"]
    assert g["n_active"] == o["n_active"]
    if per_orc is not None:
        A = np.abs(per_orc[:, 3:]).sum(axis=0)
        Af = abs_Af(per_orc).sum(axis=0)
    else:
        A = np.full(6, np.abs(o["sumA"]).max())
        Af = np.full(3, np.abs(o["sumAf"]).max())
    tolA = 1e-5 * A + 1e-6 * max(o["n_active"], 1)
    tolAf = 1e-5 * Af + 1e-6 * max(o["n_active"], 1) * max(1.0, np.abs(per_orc[:, :3]).max()
                                                           if per_orc is not None else 1.0)
    assert np.all(np.abs(g["sumA"] - o["sumA"]) <= tolA), (g["sumA"], o["sumA"])
    assert np.all(np.abs(g["sumAf"] - o["sumAf"]) <= tolAf), (g["sumAf"], o["sumAf"])
    lam = o["eig"]
    lmax = np.max(np.abs(lam))
    assert np.all(np.abs(g["eig"] - lam) <= 1e-5 * lmax + 1e-6 * max(o["n_active"], 1))
    if lmax > 0 and lam[0] > 1e-4 * lmax:                 # cond(sum A) <= 1e4
        assert g["rank"] == o["rank"] == 3
        nf = np.linalg.norm(o["f"])
        assert np.linalg.norm(g["f"] - o["f"]) <= 1e-4 * nf, (g["f"], o["f"])
    if o["n_active"] == 0:
        assert np.all(g["f"] == 0.0) and np.all(g["sumA"] == 0.0)
