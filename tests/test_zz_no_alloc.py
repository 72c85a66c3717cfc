"""The batched evaluation with the library's static device scratch
(rmp_raycast_eval_batch_static, through the C ABI) against the caller-workspace entry
point rmp_raycast_eval_batch_async on the same inputs, for two calls in a row, and its
rejection of batches larger than the static scratch.  Collected last on purpose: it must
pass after every other test has run in the same process, and alone."""
import numpy as np
import pytest

from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _results(out, B):
    return [R.result_from_bytes(out[b].cpu().numpy().tobytes()) for b in range(B)]


def test_static_scratch_batch_matches_workspace_batch():
    torch = torch_cuda()
    ctx = R.Context(0)
    try:
        wl = W.hashed_workload(n_states=6, state_seed_index=41)
        mid = ctx.upload(wl.map)
        pg = R.make_params(wl.params, wl.max_range)
        counts = np.array([65536, 4096, 1, 20000, 777, 65536], np.int32)
        B, mr = len(counts), int(counts.max())
        states = torch.tensor(np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states]),
                              device="cuda")
        nr = torch.tensor(counts, device="cuda")
        ws = torch.empty(R.rmp_batch_workspace_bytes(B, mr), dtype=torch.uint8, device="cuda")
        ref_out = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        R.rmp_raycast_eval_batch_async(ctx.handle, mid, states, nr, B, mr, pg, ws, ref_out)
        torch.cuda.synchronize()
        ref = _results(ref_out, B)
        for call in range(2):                       # two calls in a row
            out = torch.zeros((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
            R.rmp_raycast_eval_batch_static(ctx.handle, mid, states, nr, B, mr, pg, out)
            torch.cuda.synchronize()
            got = _results(out, B)
            for g, r in zip(got, ref):
                assert g["status"] == r["status"] == 0
                assert g["n_rays"] == r["n_rays"] and g["n_hits"] == r["n_hits"]
                assert g["n_active"] == r["n_active"] and g["rank"] == r["rank"]
                scale = max(np.abs(r["sumA"]).max(), 1e-30)
                assert np.all(np.abs(g["sumA"] - r["sumA"]) <= 1e-9 * scale)
                assert np.all(np.abs(g["sumAf"] - r["sumAf"]) <=
                              1e-9 * max(np.abs(r["sumAf"]).max(), 1e-30))
                nf = np.linalg.norm(r["f"])
                assert np.linalg.norm(g["f"] - r["f"]) <= 1e-9 * max(nf, 1e-30)
        # a batch whose workspace exceeds the static scratch is refused, not truncated
        big = torch.full((7,), 65536, dtype=torch.int32, device="cuda")
        st7 = torch.cat([states, states[:1]])
        out7 = torch.empty((7, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        with pytest.raises(R.RmpError) as e:
            R.rmp_raycast_eval_batch_static(ctx.handle, mid, st7, big, 7, 65536, pg, out7)
        assert e.value.status == R.STATUS_CODES["RMP_ERR_NO_MEMORY"]
    finally:
        ctx.close()
