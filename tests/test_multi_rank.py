"""Host logic of the replicas-only multi-GPU bench path, on CPU with two gloo ranks: each
rank gets its own seeded states over the same replicated map, the per-step time is the
maximum over ranks, and the whole-job rate counts every rank's rays.  No GPU, no data-path
collective (the only collectives are the timing reductions)."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, lr, w = bench.dist_env()
        wl = bench.workload(r)
        ms = 1.0 + 0.5 * r                          # rank 1 is the slower one
        ms_max = bench.max_over_ranks(ms, "cpu", w)
        x0 = wl.states[0].x.tolist()
        keys = int(np.asarray(wl.map.keys).sum())
        q.put((r, lr, w, ms_max, x0, keys, bench.whole_job_rate(w, bench.N_RAYS, ms_max)))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:                          # reported to the parent
        q.put(("error", repr(e)))


def test_two_gloo_ranks_replicas_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[0] != "error" for o in out), out
    out.sort()
    (r0, lr0, w0, m0, x0, k0, v0), (r1, lr1, w1, m1, x1, k1, v1) = out
    assert (r0, r1, w0, w1, lr0, lr1) == (0, 1, 2, 2, 0, 1)
    assert m0 == m1 == 1.5                          # max over ranks on both
    assert k0 == k1                                 # the same map replica
    assert x0 != x1                                 # independent seeded states per rank
    assert v0 == v1 == pytest.approx(2 * 65536 / 1.5e-3 / 1e9)
