"""The batched evaluation with the library's static device scratch
(rmp_raycast_eval_batch_static, through the C ABI) against the caller-workspace entry
point rmp_raycast_eval_batch_async on the same inputs -- bit for bit, since both run the
same kernels with the same fixed summation order -- for two calls in a row; one state
against the CPU oracle; no change of the device's free memory across a warm call; and the
size limit at its boundary (the largest accepted one-state batch, and one ray more).
Collected last on purpose: it must pass after every other test has run in the same process,
and alone."""
import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import assert_result_close, torch_cuda

pytestmark = pytest.mark.gpu

STATIC_BYTES = 4 << 20        # the library's static scratch per device
ONE_STATE_MAX = 406016        # largest max_rays of a one-state batch that fits it


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
        ref = ref_out.cpu().numpy().copy()
        out = torch.zeros((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        for call in range(2):                       # two calls in a row
            out.zero_()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            R.rmp_raycast_eval_batch_static(ctx.handle, mid, states, nr, B, mr, pg, out)
            torch.cuda.synchronize()
            if call == 1:                           # warm: the call allocates nothing
                assert torch.cuda.mem_get_info()[0] == free0
            got = out.cpu().numpy()
            for b in range(B):
                assert R.result_from_bytes(got[b].tobytes())["status"] == 0
                assert got[b].tobytes() == ref[b].tobytes(), (call, b)
        # one state against the oracle (4096 rays)
        s = wl.states[1]
        ro, _, por = O.raycast_eval(O.OracleMap(wl.map), s.x, s.xdot, 4096,
                                    O.make_params(wl.params, wl.max_range), want_hits=False)
        assert_result_close(R.result_from_bytes(got[1].tobytes()), ro, por)
        # the limit at its boundary: one state of up to ONE_STATE_MAX rays fits, one more
        # does not (the call checks max_rays, the size its workspace is laid out for)
        assert R.rmp_batch_workspace_bytes(1, ONE_STATE_MAX) <= STATIC_BYTES
        assert R.rmp_batch_workspace_bytes(1, ONE_STATE_MAX + 1) > STATIC_BYTES
        n1 = torch.tensor([1000], dtype=torch.int32, device="cuda")
        out1 = torch.zeros((1, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        R.rmp_raycast_eval_batch_static(ctx.handle, mid, states[:1], n1, 1, ONE_STATE_MAX, pg, out1)
        torch.cuda.synchronize()
        assert R.result_from_bytes(out1[0].cpu().numpy().tobytes())["n_rays"] == 1000
        with pytest.raises(R.RmpError) as e:
            R.rmp_raycast_eval_batch_static(ctx.handle, mid, states[:1], n1, 1,
                                            ONE_STATE_MAX + 1, pg, out1)
        assert e.value.status == R.STATUS_CODES["RMP_ERR_NO_MEMORY"]
        # a batch whose workspace exceeds the static scratch is refused, not truncated
        big = torch.full((7,), 65536, dtype=torch.int32, device="cuda")
        st7 = torch.cat([states, states[:1]])
        out7 = torch.empty((7, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
        with pytest.raises(R.RmpError) as e:
            R.rmp_raycast_eval_batch_static(ctx.handle, mid, st7, big, 7, 65536, pg, out7)
        assert e.value.status == R.STATUS_CODES["RMP_ERR_NO_MEMORY"]
    finally:
        ctx.close()
