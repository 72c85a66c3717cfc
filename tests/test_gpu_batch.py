"""GPU parity of the batched evaluation (persistent chunked kernel) against the CPU oracle,
state by state: hit records bit for bit, per-ray values and per-state sums within the
tolerances of gpu_helpers.  Covers uneven and ragged ray counts, zero-ray and invalid
states, both reductions, segmented rays, the split knob (which batches ignore), graph
capture and replay, the synchronous form and the autotuner."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import (abs_sums, assert_hits_exact, assert_per_ray_close, assert_result_close,
                         f_error_report, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = R.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def hashed(ctx):
    wl = W.hashed_workload(n_states=8, state_seed_index=21)
    return wl, ctx.upload(wl.map), O.OracleMap(wl.map)


@pytest.fixture(scope="module")
def dense(ctx):
    wl = W.dense_box_workload(n_states=6, jitter=True)
    return wl, ctx.upload(wl.map), O.OracleMap(wl.map)


def run_batch(ctx, mid, states, counts, params, max_rays=None, want=True):
    torch = torch_cuda()
    counts = np.asarray(counts, np.uint32)
    B = len(counts)
    mr = int(max_rays if max_rays is not None else max(1, counts.max()))
    st = torch.tensor(np.asarray(states, np.float64).reshape(B, 6), device="cuda")
    nr = torch.tensor(counts.astype(np.int32), device="cuda")
    ws = torch.empty(R.rmp_batch_workspace_bytes(B, mr), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    # zeroed: slots of invalid states and beyond a state's count are never written
    hits = torch.zeros(B * mr * 24, dtype=torch.uint8, device="cuda") if want else None
    per = torch.zeros(B * mr * 9, dtype=torch.float32, device="cuda") if want else None
    R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, B, mr, params, ws, out, hits=hits,
                                   per_ray=per)
    torch.cuda.synchronize()
    res = [R.result_from_bytes(out[b].cpu().numpy().tobytes()) for b in range(B)]
    if not want:
        return res, None, None, mr
    h = hits.cpu().numpy().view(R.HIT_DTYPE).reshape(B, mr)
    p = per.cpu().numpy().reshape(B, mr, 9).astype(np.float64)
    return res, h, p, mr


def check_batch(ctx, mid, om, wl_states, counts, pdict, max_range, max_rays=None):
    pg = R.make_params(pdict, max_range)
    po = O.make_params(pdict, max_range)
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl_states])
    res, h, p, mr = run_batch(ctx, mid, states, counts, pg, max_rays)
    for b, n in enumerate(counts):
        if n == 0:
            assert res[b]["status"] == 0 and res[b]["n_rays"] == 0 and res[b]["n_hits"] == 0
            assert np.all(res[b]["f"] == 0.0)
            continue
        s = wl_states[b]
        ro, ho, por = O.raycast_eval(om, s.x, s.xdot, int(n), po)
        assert_hits_exact(h[b, :n], ho)
        assert_per_ray_close(p[b, :n], por)
        assert_result_close(res[b], ro, por)
    return res


def test_batch_uneven_counts_hashed(ctx, hashed):
    wl, mid, om = hashed
    counts = [4096, 777, 65536, 1, 31, 20000, 0, 5000]
    check_batch(ctx, mid, om, wl.states, counts, wl.params, wl.max_range)


def test_batch_log_uniform_counts_fp64(ctx, hashed):
    """Uneven counts drawn log-uniform in [4096, 65536]; FP64 reduction."""
    wl, mid, om = hashed
    wu = W.hashed_workload(n_states=4, state_seed_index=22, uneven_rays=(4096, 65536))
    p = dict(wl.params, reduce_mode=1)
    check_batch(ctx, mid, om, wu.states, wu.n_rays, p, wl.max_range)


@pytest.mark.parametrize("lgs,split,cells", [(2, 0, -1), (1, 3, 0), (0, 1, -1), (0, 0, 0),
                                             (4, 0, -1)])
def test_batch_segments_and_split_dense(ctx, dense, lgs, split, cells):
    """Batches under fixed segment counts, split budgets and voxel-box settings (a segment
    setting above 4 segments per ray counts as 4 for batches, whose workspace is sized for
    4) keep hit records and results."""
    wl, mid, om = dense
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, lgs)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET, split)
    R.rmp_tune_set(ctx.handle, R.RMP_TUNE_CELL_SKIP, cells)
    try:
        check_batch(ctx, mid, om, wl.states, [1024, 4097, 1, 300, 2048, 999], wl.params,
                    wl.max_range)
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, -1)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET, -1)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_CELL_SKIP, -1)


def test_batch_matches_single_state_calls(ctx, hashed):
    """Each state's hits are identical to rmp_raycast_eval's, values within tolerance."""
    wl, mid, om = hashed
    torch = torch_cuda()
    pg = R.make_params(wl.params, wl.max_range)
    counts = [3000, 65536, 123]
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:3]])
    res, h, p, mr = run_batch(ctx, mid, states, counts, pg)
    for b, n in enumerate(counts):
        hits = torch.empty(n * 24, dtype=torch.uint8, device="cuda")
        r1 = R.rmp_raycast_eval(ctx.handle, mid, states[b, :3], states[b, 3:], n, pg, hits=hits)
        assert hits.cpu().numpy().tobytes() == h[b, :n].tobytes()
        assert r1["n_hits"] == res[b]["n_hits"] and r1["n_active"] == res[b]["n_active"]
        np.testing.assert_allclose(res[b]["sumA"], r1["sumA"], rtol=1e-9,
                                   atol=1e-9 * np.abs(r1["sumA"]).max())


def test_batch_deterministic_and_sync_form(ctx, hashed):
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    counts = [7000, 65536, 10, 4096, 33333]
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:5]])
    a = run_batch(ctx, mid, states, counts, pg, want=False)[0]
    b = run_batch(ctx, mid, states, counts, pg, want=False)[0]
    c = R.rmp_raycast_eval_batch(ctx.handle, mid, states, counts, pg)
    for x, y, z in zip(a, b, c):
        for key in ("f", "sumA", "sumAf", "eig"):
            assert np.array_equal(x[key], y[key]) and np.array_equal(x[key], z[key])


def test_batch_results_independent_of_order_and_company(ctx, hashed):
    """A state's result depends on that state alone: bitwise the same alone, in a batch, and
    in a permuted batch (segments per ray chosen per state, chunks and groups per state,
    fixed summation order)."""
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    counts = np.array([3000, 65536, 777, 20000, 4096, 12000, 1, 50000], np.uint32)
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:8]])
    base = run_batch(ctx, mid, states, counts, pg, want=False)[0]
    perm = np.random.default_rng(3).permutation(8)
    permuted = run_batch(ctx, mid, states[perm], counts[perm], pg, want=False)[0]
    keys = ("f", "sumA", "sumAf", "eig")
    for j, b in enumerate(perm):
        for key in keys:
            assert np.array_equal(permuted[j][key], base[b][key]), (b, key)
    for b in (0, 1, 6):
        alone = run_batch(ctx, mid, states[b:b + 1], counts[b:b + 1], pg, want=False)[0][0]
        for key in keys:
            assert np.array_equal(alone[key], base[b][key]), (b, key)


def test_batch_segment_thresholds(ctx, hashed):
    """Ray counts on both sides of the default per-state segment thresholds (4 segments
    while 4 n fits in the persistent launch's threads, 2 while 2 n does, else 1; 155648
    threads on a 152-SM part): every state matches the oracle, and its result is bitwise
    the same alone as in the mixed batch."""
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    po = O.make_params(wl.params, wl.max_range)
    counts = np.array([38912, 38913, 77824, 77825], np.uint32)
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:4]])
    mixed, h, p, _ = run_batch(ctx, mid, states, counts, pg)
    for b, n in enumerate(counts):
        s = wl.states[b]
        ro, ho, por = O.raycast_eval(om, s.x, s.xdot, int(n), po)
        assert_hits_exact(h[b, :n], ho)
        assert_result_close(mixed[b], ro, por)
        alone = run_batch(ctx, mid, states[b:b + 1], counts[b:b + 1], pg, want=False)[0][0]
        for key in ("f", "sumA", "sumAf", "eig"):
            assert np.array_equal(alone[key], mixed[b][key]), (n, key)


def test_batch_invalid_states_are_isolated(ctx, hashed):
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    po = O.make_params(wl.params, wl.max_range)
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:4]])
    states[1, 0] = np.nan
    counts = np.array([2000, 2000, 5000, 2000], np.uint32)
    res, h, p, mr = run_batch(ctx, mid, states, counts, pg, max_rays=4096)
    assert res[1]["status"] == R.RMP_ERR_INVALID_ARG
    assert res[2]["status"] == R.RMP_ERR_INVALID_ARG          # more rays than max_rays
    for b in (0, 3):
        s = wl.states[b]
        ro, ho, por = O.raycast_eval(om, s.x, s.xdot, 2000, po)
        assert_hits_exact(h[b, :2000], ho)
        assert_result_close(res[b], ro, por)


def test_batch_argument_errors(ctx, hashed):
    torch = torch_cuda()
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    st = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    nr = torch.ones(2, dtype=torch.int32, device="cuda")
    out = torch.empty((2, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    small = torch.empty(R.rmp_batch_workspace_bytes(2, 100) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, 2, 100, pg, small, out)
    ws = torch.empty(R.rmp_batch_workspace_bytes(2, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval_batch_async(ctx.handle, 12345, st, nr, 2, 100, pg, ws, out)
    with pytest.raises(R.RmpError):
        R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, 0, 100, pg, ws, out)


def test_batch_graph_capture_and_replay(ctx, hashed):
    """The async batch call captured in a CUDA graph and replayed with new states and counts
    gives bitwise the results of direct calls."""
    torch = torch_cuda()
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    B, mr = 6, 65536
    st = torch.zeros((B, 6), dtype=torch.float64, device="cuda")
    nr = torch.zeros(B, dtype=torch.int32, device="cuda")
    ws = torch.empty(R.rmp_batch_workspace_bytes(B, mr), dtype=torch.uint8, device="cuda")
    out = torch.zeros((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, B, mr, pg, ws, out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, B, mr, pg, ws, out)
    rng = np.random.default_rng(5)
    for rep in range(2):
        idx = rng.permutation(len(wl.states))[:B]
        states = np.stack([np.concatenate([wl.states[i].x, wl.states[i].xdot]) for i in idx])
        counts = rng.integers(0, mr + 1, B).astype(np.int32)
        st.copy_(torch.tensor(states, device="cuda"))
        nr.copy_(torch.tensor(counts, device="cuda"))
        g.replay()
        torch.cuda.synchronize()
        got = [R.result_from_bytes(out[b].cpu().numpy().tobytes()) for b in range(B)]
        ref = run_batch(ctx, mid, states, counts, pg, max_rays=mr, want=False)[0]
        for x, y in zip(got, ref):
            assert x["status"] == y["status"] == 0
            assert np.array_equal(x["f"], y["f"]) and np.array_equal(x["sumA"], y["sumA"])


def test_batch_autotuner(ctx, hashed):
    torch = torch_cuda()
    wl, mid, om = hashed
    pg = R.make_params(wl.params, wl.max_range)
    counts = np.array([4096, 65536, 9000, 30000], np.int32)
    B, mr = len(counts), int(counts.max())
    states = np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states[:B]])
    st = torch.tensor(states, device="cuda")
    nr = torch.tensor(counts, device="cuda")
    ws = torch.empty(R.rmp_batch_workspace_bytes(B, mr), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    try:
        times = R.rmp_batch_autotune(ctx.handle, mid, st, nr, B, mr, pg, ws, out, reps=3)
        assert len(times) == 9 and all(np.isfinite(t) and t > 0 for t in times)
        best = int(np.argmin(times))
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_BLOCK) == (64, 128, 256)[best // 3]
        assert R.rmp_tune_get(ctx.handle, R.RMP_TUNE_LG_SEGMENTS) == best % 3
        check_batch(ctx, mid, om, wl.states[:B], counts, wl.params, wl.max_range)
    finally:
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_BLOCK, 0)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_LG_SEGMENTS, -1)
        R.rmp_tune_set(ctx.handle, R.RMP_TUNE_SPLIT_BUDGET, -1)


def test_batch_precision_kahan_vs_fp64_per_state(ctx, hashed, capsys):
    """Config 4 in full: 256 states, rays log-uniform in [4096, 65536] (5.26 M rays), both
    reductions (compensated FP32, FP64).  Per state, the error of sum A, sum A f and the
    resolved f against the FP64 oracle (printed as a 256-row table with cond(sum A) and the
    perturbation bound of f), each within the tolerances of gpu_helpers."""
    from concurrent.futures import ThreadPoolExecutor
    wl, mid, om = hashed
    w4 = W.hashed_workload(n_states=256, uneven_rays=(4096, 65536))
    states, counts = w4.states, np.asarray(w4.n_rays, np.uint32)
    assert len(states) == 256 and int(counts.sum()) > 5_000_000
    po = O.make_params(wl.params, wl.max_range)
    sv = np.stack([np.concatenate([s.x, s.xdot]) for s in states])
    runs = {}
    for mode in (0, 1):
        pg = R.make_params(dict(wl.params, reduce_mode=mode), wl.max_range)
        runs[mode] = run_batch(ctx, mid, sv, counts, pg, want=False)[0]

    def oracle_state(b):
        s = states[b]
        ro, _, por = O.raycast_eval(om, s.x, s.xdot, int(counts[b]), po, want_hits=False)
        return ro, abs_sums(por)

    with ThreadPoolExecutor(os.cpu_count() or 4) as pool:
        orc = list(pool.map(oracle_state, range(len(states))))
    rows = []
    for b in range(len(states)):
        ro, sums = orc[b]
        row = [b, int(counts[b])]
        for mode in (0, 1):
            g = runs[mode][b]
            assert_result_close(g, ro, sums=sums)
            eA = np.abs(g["sumA"] - ro["sumA"]).max() / max(np.abs(ro["sumA"]).max(), 1e-300)
            eAf = np.abs(g["sumAf"] - ro["sumAf"]).max() / max(np.abs(ro["sumAf"]).max(), 1e-300)
            ef, cond, fb = f_error_report(g, ro)
            row += [eA, eAf, ef]
        row += [cond, fb]
        rows.append(row)
    a = np.array([r[2:8] for r in rows])
    with capsys.disabled():
        print("\nstate   rays | kahan32: sumA    sumAf   f       | fp64: sumA    sumAf   f       "
              "| cond(sumA) f bound  (relative to the FP64 oracle)")
        for r in rows:
            print("%5d %6d | %.1e %.1e %.1e | %.1e %.1e %.1e | %.1e %.1e" % tuple(r))
        print("max          | %.1e %.1e %.1e | %.1e %.1e %.1e |" % tuple(a.max(axis=0)))
        print("median       | %.1e %.1e %.1e | %.1e %.1e %.1e |" % tuple(np.median(a, axis=0)))
