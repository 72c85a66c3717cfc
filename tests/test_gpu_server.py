"""GPU tests of the continuous-batching request server: results against the CPU oracle,
the same request alone and inside a mixed stream (within the stated tolerances of the
oracle, and bitwise identical to each other), admission under a small device-memory
budget, error completion, and concurrent submitters."""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2301_08068_gb300 import rmp as R
from paper_2301_08068_gb300 import workloads as W

from gpu_helpers import assert_result_close, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch_cuda()
    ctx = R.Context(0)
    hw = W.hashed_workload(n_states=40, state_seed_index=31)
    dw = W.dense_box_workload(n_states=40, jitter=True, seed_index=0)
    maps = {"hashed": (hw, ctx.upload(hw.map), O.OracleMap(hw.map)),
            "dense": (dw, ctx.upload(dw.map), O.OracleMap(dw.map))}
    yield ctx, maps
    ctx.close()


def oracle_result(entry, i, n):
    wl, mid, om = entry
    s = wl.states[i]
    ro, _, por = O.raycast_eval(om, s.x, s.xdot, n, O.make_params(wl.params, wl.max_range),
                                want_hits=False)
    return ro, por


def submit(srv, entry, i, n):
    wl, mid, om = entry
    s = wl.states[i]
    return srv.submit(mid, s.x, s.xdot, n, R.make_params(wl.params, wl.max_range))


def close_to_each_other(a, b, por):
    """Two GPU results of one request: same counts, sums within the per-ray magnitude
    tolerance of gpu_helpers (each is within it of the oracle)."""
    assert a["n_hits"] == b["n_hits"] and a["n_active"] == b["n_active"] and a["rank"] == b["rank"]
    A = np.abs(por[:, 3:]).sum(axis=0)
    tol = 2e-5 * A + 2e-6 * max(a["n_active"], 1)
    assert np.all(np.abs(a["sumA"] - b["sumA"]) <= tol)


def test_server_results_match_oracle(env):
    ctx, maps = env
    rng = np.random.default_rng(1)
    jobs = []
    with R.Server(ctx, slots=4) as srv:
        for j in range(24):
            name = ("hashed", "dense")[j % 2]
            n = int(rng.integers(1, 20000))
            i = int(rng.integers(0, 40))
            jobs.append((name, i, n, submit(srv, maps[name], i, n)))
        for name, i, n, t in jobs:
            res, lat = srv.wait(t)
            assert lat > 0
            ro, por = oracle_result(maps[name], i, n)
            assert_result_close(res, ro, por)
        st = srv.stats()
    assert st["submitted"] == st["completed"] == 24 and st["rejected"] == 0
    assert st["batches"] <= 24 and st["batched_states"] == 24


def test_server_same_result_alone_and_in_mix(env):
    ctx, maps = env
    ro, por = oracle_result(maps["hashed"], 7, 5000)
    # one batch in flight at a time and every submission's arguments built beforehand, so
    # requests queue behind the running batch and share the next one
    with R.Server(ctx, slots=1) as srv:
        alone, _ = srv.wait(submit(srv, maps["hashed"], 7, 5000))
        rng = np.random.default_rng(2)
        params = {k: R.make_params(v[0].params, v[0].max_range) for k, v in maps.items()}
        plan = []
        for j in range(80):
            if j == 40:
                plan.append(("probe", "hashed", 7, 5000))
            name = ("hashed", "dense")[int(rng.integers(0, 2))]
            plan.append((name, name, int(rng.integers(0, 40)), int(rng.integers(1000, 60000))))
        tickets = []
        for tag, name, i, n in plan:
            wl, mid, _ = maps[name]
            tickets.append((tag, srv.submit(mid, wl.states[i].x, wl.states[i].xdot, n,
                                            params[name])))
        mixed = None
        for name, t in tickets:
            res, _ = srv.wait(t)
            assert res["status"] == 0
            if name == "probe":
                mixed = res
        st = srv.stats()
    assert st["batches"] < st["batched_states"]          # requests really shared batches
    assert_result_close(alone, ro, por)
    assert_result_close(mixed, ro, por)
    close_to_each_other(alone, mixed, por)
    for key in ("f", "sumA", "sumAf", "eig"):              # and in fact bitwise identical
        assert np.array_equal(alone[key], mixed[key]), key


def test_server_memory_budget_admission(env):
    ctx, maps = env
    need_one = R.rmp_batch_workspace_bytes(1, 30000)
    budget = int(need_one * 1.5) + (1 << 16)                # one 30000-ray batch at a time
    with R.Server(ctx, slots=4, mem_budget_bytes=budget, max_rays=262144) as srv:
        ts = [submit(srv, maps["hashed"], i, 30000) for i in range(6)]
        big = submit(srv, maps["hashed"], 0, 262144)        # can never fit the budget
        for i, t in enumerate(ts):
            res, _ = srv.wait(t)
            assert res["status"] == 0
        res, _ = srv.wait(big)
        assert res["status"] == R.STATUS_CODES["RMP_ERR_NO_MEMORY"]
        st = srv.stats()
    assert st["max_inflight"] == 1 and st["mem_high_water"] <= budget
    assert st["rejected"] == 1


def test_server_errors(env):
    ctx, maps = env
    wl, mid, om = maps["hashed"]
    p = R.make_params(wl.params, wl.max_range)
    with R.Server(ctx, slots=2, max_rays=100000) as srv:
        t = srv.submit(9999, wl.states[0].x, wl.states[0].xdot, 100, p)
        res, _ = srv.wait(t)
        assert res["status"] == R.STATUS_CODES["RMP_ERR_UNKNOWN_MAP"]
        with pytest.raises(R.RmpError):
            srv.submit(mid, wl.states[0].x, wl.states[0].xdot, 0, p)
        with pytest.raises(R.RmpError):
            srv.submit(mid, wl.states[0].x, wl.states[0].xdot, 100001, p)
        with pytest.raises(R.RmpError):
            srv.poll(123456)
        ok = srv.submit(mid, wl.states[1].x, wl.states[1].xdot, 1000, p)
        res, _ = srv.wait(ok)
        assert res["status"] == 0
        # a collected ticket is no longer valid: poll and wait fail at once, not NOT_READY
        with pytest.raises(R.RmpError):
            srv.poll(ok)
        with pytest.raises(R.RmpError):
            srv.wait(ok, 60000)


def test_server_concurrent_submitters(env):
    ctx, maps = env
    out = {}
    errors = []
    with R.Server(ctx, slots=4) as srv:
        def client(k):
            try:
                rng = np.random.default_rng(100 + k)
                mine = []
                for j in range(15):
                    name = ("hashed", "dense")[(j + k) % 2]
                    i, n = int(rng.integers(0, 40)), int(rng.integers(1, 8000))
                    mine.append((name, i, n, submit(srv, maps[name], i, n)))
                for name, i, n, t in mine:
                    out[t] = (name, i, n, srv.wait(t)[0])
            except Exception as e:                     # surfaced below
                errors.append(e)
        th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    assert not errors and len(out) == 60
    for name, i, n, res in list(out.values())[::6]:
        ro, por = oracle_result(maps[name], i, n)
        assert_result_close(res, ro, por)
