"""GPU tests of streamed LiDAR scans at OS-0 size (128 x 2048 = 262144 points): the scan
against the CPU oracle, and the copy/compute pipeline against direct evaluations (bitwise:
same kernel, same launch shape) with slot reuse and its error."""
import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import (assert_per_ray_close, assert_result_close, gpu_scan, scan_abs_term,
                         torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def os0():
    return W.lidar_workload(beams=128, columns=2048, fov_deg=90.0)


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = R.Context(0)
    yield c
    c.close()


def test_os0_scan_matches_oracle(ctx, os0):
    pg = R.make_params(os0.params, os0.max_range)
    po = O.make_params(os0.params, os0.max_range)
    assert os0.points.shape == (262144, 3)
    rg, pgr = gpu_scan(ctx, os0.points, os0.x, os0.xdot, pg)
    ro, por = O.scan_eval(os0.points, os0.x, os0.xdot, po)
    at = scan_abs_term(os0.points, os0.x, os0.xdot, os0.params)
    assert_per_ray_close(pgr, por, at)
    assert_result_close(rg, ro, por, at)


def test_pipeline_matches_direct_scans(ctx, os0):
    torch = torch_cuda()
    pg = R.make_params(os0.params, os0.max_range)
    rng = np.random.default_rng(8)
    scans = []
    for k in range(7):
        pts = os0.points.copy()
        pts[rng.integers(0, len(pts), 5000)] = np.nan          # dropouts differ per scan
        scans.append((torch.from_numpy(pts).pin_memory(), rng.normal(size=3)))
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    out = torch.empty(R.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    direct = []
    for pts, v in scans:
        st = torch.tensor(np.concatenate([os0.x, v]), dtype=torch.float64, device="cuda")
        R.rmp_scan_eval_async(ctx.handle, pts.cuda(), st, pg, ws, out)
        torch.cuda.synchronize()
        direct.append(R.result_from_bytes(out.cpu().numpy().tobytes()))
    with R.ScanPipeline(ctx, 262144, slots=3) as pipe:
        tickets = []
        for i, (pts, v) in enumerate(scans):
            tickets.append(pipe.submit(pts, os0.x, v, pg))
            if i >= 1:                                        # results trail submits by one
                got = pipe.wait(tickets[i - 1])
                for key in ("f", "sumA", "sumAf", "eig"):
                    assert np.array_equal(got[key], direct[i - 1][key]), (i - 1, key)
        got = pipe.wait(tickets[-1])
        assert np.array_equal(got["f"], direct[-1]["f"])
        with pytest.raises(R.RmpError):                       # slot reused 3 submits later
            pipe.wait(tickets[0])
        with pytest.raises(R.RmpError):
            pipe.wait(999)
    pts2 = scans[2][0].numpy()
    ro, por = O.scan_eval(pts2, os0.x, scans[2][1], O.make_params(os0.params, os0.max_range))
    assert_result_close(direct[2], ro, por, scan_abs_term(pts2, os0.x, scans[2][1], os0.params))
