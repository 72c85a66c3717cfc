"""The served stream checked against the oracle request by request: three resident maps
(dense 128^3 at 0.05 m, hashed 40x40x10 m at 0.1 m, hashed 100x100x20 m at 0.2 m), Poisson
arrivals at 20000 requests/s fed to the continuous-batching server.  Every request of a
2000-request stream (1024..16384 rays, submitted as one burst) and a random 500 of the full two-second stream (1024..262144 rays,
about 40000 requests, in real time) must be within the gpu_helpers tolerances
of the oracle evaluated on its own.  The oracle runs on all host cores, one unchanged
single-threaded evaluation per thread."""
import os
import time
from concurrent.futures import ThreadPoolExecutor

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
    wls = W.served_workloads(64)
    mids = [ctx.upload(w.map) for w in wls]
    oms = [O.OracleMap(w.map) for w in wls]
    yield ctx, wls, mids, oms
    ctx.close()


def serve(ctx, wls, mids, duration, ray_lo, ray_hi, seed_index, limit=None, paced=True):
    """Submits the stream at its arrival times (or all at once when not `paced`); returns
    the requests and their results."""
    t_arr, maps, rays, vel = W.poisson_requests(3, 20000.0, duration, ray_lo, ray_hi,
                                                seed_index=seed_index)
    n = len(t_arr) if limit is None else min(limit, len(t_arr))
    reqs = [(int(maps[i]), wls[maps[i]].states[i % 64].x, vel[i], int(rays[i])) for i in range(n)]
    params = [R.make_params(w.params, w.max_range) for w in wls]
    with R.Server(ctx, slots=4, max_batch_states=256, max_rays=262144,
                  mem_budget_bytes=256 << 20) as srv:
        tickets = []
        t0 = time.perf_counter()
        for i, (m, x, v, r) in enumerate(reqs):
            while paced and time.perf_counter() - t0 < t_arr[i]:
                pass
            tickets.append(srv.submit(mids[m], x, v, r, params[m]))
        results = [srv.wait(t, 60000)[0] for t in tickets]
        st = srv.stats()
    assert st["completed"] == n and st["rejected"] == 0
    return reqs, results, st


def check(wls, oms, reqs, results, idx):
    def orc(i):
        m, x, v, r = reqs[i]
        ro, _, por = O.raycast_eval(oms[m], x, v, r, O.make_params(wls[m].params, wls[m].max_range),
                                    want_hits=False)
        return i, ro, por

    cores = len(os.sched_getaffinity(0))
    idx = list(idx)
    with ThreadPoolExecutor(cores) as ex:
        for c in range(0, len(idx), 4 * cores):          # bounded per-ray arrays in flight
            for i, ro, por in ex.map(orc, idx[c:c + 4 * cores]):
                assert results[i]["status"] == 0, i
                assert_result_close(results[i], ro, por)


def test_every_request_of_a_short_stream(env):
    ctx, wls, mids, oms = env
    reqs, results, st = serve(ctx, wls, mids, 0.2, 1024, 16384, seed_index=40, limit=2000,
                              paced=False)
    assert len(reqs) == 2000
    assert {m for m, _, _, _ in reqs} == {0, 1, 2}
    assert st["batched_states"] == len(reqs)
    check(wls, oms, reqs, results, range(len(reqs)))


def test_random_500_of_the_full_stream(env):
    ctx, wls, mids, oms = env
    reqs, results, _ = serve(ctx, wls, mids, 2.0, 1024, 262144, seed_index=4)
    assert len(reqs) > 30000
    idx = np.random.default_rng(5).choice(len(reqs), 500, replace=False)
    check(wls, oms, reqs, results, sorted(int(i) for i in idx))
