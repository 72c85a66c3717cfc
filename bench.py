#!/usr/bin/env python
"""Benchmark: raycast-RMP evaluation throughput on one GB300 (or N replicas).

Workload: hashed TSDF map (8^3 blocks, 0.1 m voxels over 40 x 40 x 10 m, 200 seeded boxes and
spheres, truncation 0.3 m), 65536 Halton rays per evaluation, max range 10 m, one robot
state per call (states cycle over 64 seeded free positions with N(0,1) velocities).  A step
is one full evaluation: Halton directions, exact DDA march, per-ray obstacle policy,
reduction and FP64 resolve (one fused kernel).

Printed JSON line (rank 0):
  value     whole-job rays/s (Grays/s): rays of all ranks / max over ranks of the mean
            per-step device time (CUDA events around each evaluation, inputs resident in HBM,
            L2 flushed by a 256 MiB write between timed steps, outside the events);
  e2e       the same metric through the public synchronous call rmp_raycast_eval with host
            x/xdot and a host result (the state goes to the device in the launch, the result
            comes back into pinned host memory, both inside the timed region), wall clock
            per call;
  roofline  algorithmic bytes per launch / mean kernel time against the measured HBM copy
            bandwidth; traffic from the committed ncu capture when it matches this kernel;
  cpu_baseline  the C oracle on a bounded sample: one evaluation per host thread at once,
            on every core of this host (and, beside it, on one core).
--impl reference times the oracle instead (rank 0 only, every host core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Grays/s and RMP evals/s at 65536 rays; served p50/p99 latency vs plain kernel"
UNIT = "Grays/s"
WORKLOAD = ("hashed TSDF 40x40x10 m at 0.1 m (8^3 blocks, 200 boxes/spheres, trunc 0.3 m), "
            "65536 Halton rays, max range 10 m, one state per call")
N_RAYS = 65536
N_STATES = 64
PREWARM_S = 0.3   # untimed evaluations while the clock sampler starts
FLUSH_BYTES = 256 << 20
PAPER_RATE = 65536 * 3000 / 1e9   # 65536 rays at up to 3 kHz (abstract), other hardware
# integer operations of one step of the plain exact DDA: two cross-multiplied t comparisons
# (two 32x32->64 products and a 64-bit compare each: 8), the range test (product, shift,
# compare: 3), the step itself (voxel index, boundary numerator: 3), the voxel address
# (block key, in-block offset: 4), the load's test and the loop branch (2)
INT_OPS_PER_STEP = 20
SM_COUNT = 152
INT_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and served sections (rank 0, N=1 only)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="length of the Poisson request stream of the served section")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def workload(rank: int):
    from paper_2301_08068_gb300 import workloads as W
    # every rank gets its own seeded states (independent work; the map is replicated)
    return W.hashed_workload(n_states=N_STATES, state_seed_index=1 + 1000 * rank)


def max_over_ranks(value: float, device, world: int) -> float:
    """Largest `value` over all ranks (identity on one rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, rays_per_rank_step: int, ms_max: float) -> float:
    """Whole-job Grays/s: every rank's rays over the slowest rank's time per step."""
    return world * rays_per_rank_step / (ms_max / 1e3) / 1e9


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_on_threads(om, p, states, n_rays: int, threads: int, evals: int, pool=None):
    """`evals` oracle evaluations of `n_rays` rays, state k % len(states) for evaluation k,
    spread over `threads` host threads: the oracle is the unchanged single-threaded C code
    (its evaluation keeps no global state and the ctypes call releases the GIL), run on
    independent states at once.  `pool` (a ThreadPoolExecutor of `threads` workers) is
    reused across calls when given.  Returns the wall time in seconds."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O

    def work(k):
        s = states[k % len(states)]
        O.raycast_eval(om, s.x, s.xdot, n_rays, p, want_hits=False, want_per_ray=False)

    own = pool is None
    if own:
        pool = ThreadPoolExecutor(threads)
    try:
        t0 = time.perf_counter()
        for f in [pool.submit(work, k) for k in range(evals)]:
            f.result()
        return time.perf_counter() - t0
    finally:
        if own:
            pool.shutdown()


def time_oracle(wl, seconds: float, max_evals: int):
    """Single-threaded oracle evaluations of the workload's states until `seconds` pass,
    with this process pinned to one core meanwhile (where the OS allows it)."""
    import oracle as O
    om = O.OracleMap(wl.map)
    p = O.make_params(wl.params, wl.max_range)
    try:
        cpus = os.sched_getaffinity(0)
        os.sched_setaffinity(0, {min(cpus)})
    except (AttributeError, OSError):
        cpus = None
    try:
        t0 = time.perf_counter()
        n = 0
        times = []
        while n < max_evals and (time.perf_counter() - t0 < seconds or n == 0):
            s = wl.states[n % len(wl.states)]
            t1 = time.perf_counter()
            O.raycast_eval(om, s.x, s.xdot, N_RAYS, p, want_hits=False, want_per_ray=False)
            times.append(time.perf_counter() - t1)
            n += 1
    finally:
        if cpus is not None:
            os.sched_setaffinity(0, cpus)
    return n, sum(times), times


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        import tempfile
        self.device = device
        self.proc = None
        # raw samples: RMP_BENCH_CLOCKS_DIR if set (to keep them), else a temporary folder
        folder = os.environ.get("RMP_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], float(parts[3])))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v == "Active"})
        loaded = [r[0] for r in rows if r[3] > 0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


LAUNCH_KEYS = ("block", "grid", "lg_segments", "ray_cells", "smem_bytes")


def code_only(text: str) -> str:
    """C++/CUDA source without comments, whitespace collapsed (string literals kept)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(launch: dict) -> str:
    """Identity of the measured launch: the device code (kernel source and its header,
    comments and layout aside) and the launch shape the host chose for it.  The committed
    DRAM traffic is used only while both are unchanged."""
    h = hashlib.sha256()
    for f in ("rmp_kernels.cu", "rmp_internal.h"):
        src = open(os.path.join(ROOT, "paper_2301_08068_gb300", "csrc", f)).read()
        h.update(code_only(src).encode())
    h.update(json.dumps([launch.get(k) for k in LAUNCH_KEYS]).encode())
    return h.hexdigest()[:16]


def strict_json(obj):
    """obj with every non-finite float replaced by None (the JSON line stays strict JSON)."""
    if isinstance(obj, float):
        return obj if np.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: strict_json(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [strict_json(v) for v in obj]
    return obj


def stratified_order(costs) -> list:
    """Indices of `costs` (a power-of-two count) such that every prefix samples the sorted
    costs evenly: position p holds the state of cost rank bitreverse(p)."""
    n = len(costs)
    bits = max(1, (n - 1).bit_length())
    assert n == 1 << bits
    ranked = list(np.argsort(np.asarray(costs), kind="stable"))
    rev = [int(format(p, "0%db" % bits)[::-1], 2) for p in range(n)]
    return [int(ranked[r]) for r in rev]


def committed_counters(src_hash: str) -> dict:
    """Per-launch counters of the raycast kernel from the committed ncu capture (DRAM bytes,
    L2 bytes, warp instructions), if it was taken on the current kernel source and launch
    shape; empty otherwise."""
    path = os.path.join(ROOT, "profiles", "raycast_hashed_65536_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return {}
    if d.get("kernel_launch_sha256_16") != src_hash:
        return {}
    return d


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def timed_device(fn, flush, reps: int):
    """Median CUDA-event time (ms) of fn() over `reps` runs, L2 flushed before each."""
    import torch
    for i in range(3):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for i in range(reps):
        flush.fill_(i & 0xFF)
        ev[i][0].record()
        fn()
        ev[i][1].record()
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def config1_section(ctx, flush) -> dict:
    """Config 1: dense uint8 grid 64^3 at 0.1 m with 20 boxes, 1024 Halton rays, max range
    5 m, one state per call (device-resident state and result, L2 flushed between calls),
    against the same kernel's floor: a one-ray evaluation."""
    import torch
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    wl = W.dense_box_workload(n_states=16, jitter=True)
    mid = ctx.upload(wl.map)
    p = R.make_params(wl.params, wl.max_range)
    st = torch.tensor(np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states]),
                      dtype=torch.float64, device="cuda")
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    out = torch.empty((16, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    n = wl.n_rays
    ev = []
    for i in range(400):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        R.rmp_raycast_eval_async(ctx.handle, mid, st[i % 16], n, p, ws, out[i % 16])
        b.record()
        ev.append((a, b))
    torch.cuda.synchronize()
    t = [x.elapsed_time(y) for x, y in ev[20:]]      # the first 20 calls warm up
    ms = float(np.mean(t))
    ms1 = timed_device(lambda: R.rmp_raycast_eval_async(ctx.handle, mid, st[0], 1, p, ws, out[0]),
                       flush, 200)
    R.rmp_map_release(ctx.handle, mid)
    return {"workload": "dense 64^3 at 0.1 m, 20 boxes, 1024 rays, max range 5 m",
            "us_per_eval": 1e3 * ms, "us_per_eval_p50": 1e3 * float(np.percentile(t, 50)),
            "Grays_per_s": n / ms / 1e6, "evals_per_s": 1e3 / ms,
            "floor_us_one_ray": 1e3 * ms1, "frac_of_floor": ms1 / ms}


def batch_section(ctx, mid, flush, per_state: bool = False) -> dict:
    """Batched evaluation: 256 states over the same hashed map with ray counts drawn
    log-uniform in [4096, 65536]; autotuned launch, captured once in a CUDA graph and
    replayed; against the plain single-state kernel called once per state; both
    reductions (compensated FP32, FP64).  per_state: also the per-state results of both
    reductions (for the precision report against the oracle)."""
    import torch
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    wl = W.hashed_workload(n_states=256, uneven_rays=(4096, 65536))
    counts = np.asarray(wl.n_rays, np.int32)
    B, mr = len(counts), int(counts.max())
    st = torch.tensor(np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states]),
                      dtype=torch.float64, device="cuda")
    nr = torch.tensor(counts, device="cuda")
    ws = torch.empty(R.rmp_batch_workspace_bytes(B, mr), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")
    knobs = [R.rmp_tune_get(ctx.handle, k) for k in (1, 2, 4)]
    res = {"workload": "256 states on the hashed 40x40x10 m map, rays log-uniform in "
                       "[4096, 65536] (total %d)" % int(counts.sum())}
    try:
        for mode, name in ((0, "kahan_fp32"), (1, "fp64")):
            p = R.make_params(dict(wl.params, reduce_mode=mode), wl.max_range)
            times = R.rmp_batch_autotune(ctx.handle, mid, st, nr, B, mr, p, ws, out, reps=3)
            tuned = {"block": R.rmp_tune_get(ctx.handle, 1),
                     "lg_segments": R.rmp_tune_get(ctx.handle, 2)}
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, B, mr, p, ws, out)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                R.rmp_raycast_eval_batch_async(ctx.handle, mid, st, nr, B, mr, p, ws, out)
            ms = timed_device(g.replay, flush, 20)
            res[name] = {"ms_per_batch": ms, "Grays_per_s": float(counts.sum()) / ms / 1e6,
                         "evals_per_s": B / ms * 1e3, "tuned": tuned,
                         "autotune_ms": [round(t, 4) for t in times]}
            if per_state:
                o = out.cpu().numpy()
                res.setdefault("_results", {})[name] = [R.result_from_bytes(o[b].tobytes())
                                                        for b in range(B)]
        # the plain single-state kernel, one launch per state, same states and counts
        R.rmp_tune_set(ctx.handle, 1, 0)
        R.rmp_tune_set(ctx.handle, 2, -1)
        R.rmp_tune_set(ctx.handle, 4, -1)
        p = R.make_params(wl.params, wl.max_range)
        wss = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
        R.rmp_workspace_init(wss)
        outs = torch.empty((B, R.RESULT_BYTES), dtype=torch.uint8, device="cuda")

        def loop():
            for b in range(B):
                R.rmp_raycast_eval_async(ctx.handle, mid, st[b], int(counts[b]), p, wss, outs[b])
        ms = timed_device(loop, flush, 5)
        res["plain_per_state"] = {"ms_per_batch": ms,
                                  "Grays_per_s": float(counts.sum()) / ms / 1e6,
                                  "evals_per_s": B / ms * 1e3}
        res["speedup_vs_plain"] = res["plain_per_state"]["ms_per_batch"] / \
            res["kahan_fp32"]["ms_per_batch"]
    finally:
        for k, v in zip((1, 2, 4), knobs):
            R.rmp_tune_set(ctx.handle, k, v)
    return res


def lidar_section(ctx, flush) -> dict:
    """LiDAR variant (config 3): a 64 x 1024 scan (65536 points, FP32, sensor frame), one
    fused launch per scan (per-point policy, reduction, FP64 resolve).  It is launch- and
    latency-bound, so it is reported against the same kernel's floor: a one-point scan."""
    import torch
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    sw = W.lidar_workload()
    p = R.make_params(sw.params, sw.max_range)
    pts = torch.from_numpy(np.ascontiguousarray(sw.points, np.float32)).cuda()
    st = torch.tensor(np.concatenate([sw.x, sw.xdot]), dtype=torch.float64, device="cuda")
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    R.rmp_workspace_init(ws)
    out = torch.empty(R.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ms = timed_device(lambda: R.rmp_scan_eval_async(ctx.handle, pts, st, p, ws, out), flush, 200)
    one = pts[:1].contiguous()
    ms1 = timed_device(lambda: R.rmp_scan_eval_async(ctx.handle, one, st, p, ws, out), flush, 200)
    n = int(pts.shape[0])
    return {"workload": "64 x 1024 scan (65536 points), Table I LiDAR params",
            "ms_per_scan": ms, "evals_per_s": 1e3 / ms, "Gpoints_per_s": n / ms / 1e6,
            "floor_ms_one_point": ms1, "frac_of_floor": ms1 / ms}


def lidar_stream_section(ctx) -> dict:
    """OS-0 sizing (128 x 2048 = 262144 points per scan, the paper's 20 Hz sensor-rate
    requirement): scans from pinned host memory through the copy/compute pipeline, each
    result read back, against copying then evaluating one scan at a time."""
    import torch
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    sw = W.lidar_workload(beams=128, columns=2048, fov_deg=90.0)
    p = R.make_params(sw.params, sw.max_range)
    rng = np.random.default_rng(11)
    scans = [(torch.from_numpy(sw.points.copy()).pin_memory(), rng.normal(size=3))
             for _ in range(8)]
    n_scans = 400
    with R.ScanPipeline(ctx, 262144, slots=2) as pipe:
        for i in range(8):
            pipe.wait(pipe.submit(scans[i][0], sw.x, scans[i][1], p))
        lat = []
        t0 = time.perf_counter()
        prev = None
        for i in range(n_scans):
            pts, v = scans[i % 8]
            ts = time.perf_counter()
            t = pipe.submit(pts, sw.x, v, p)
            if prev is not None:
                pipe.wait(prev[0])
                lat.append(time.perf_counter() - prev[1])
            prev = (t, ts)
        pipe.wait(prev[0])
        lat.append(time.perf_counter() - prev[1])
        span = time.perf_counter() - t0
    dev = torch.empty((262144, 3), dtype=torch.float32, device="cuda")
    t1 = time.perf_counter()
    for i in range(n_scans // 4):
        pts, v = scans[i % 8]
        dev.copy_(pts)
        R.rmp_scan_eval(ctx.handle, dev, sw.x, v, p)
    serial = (time.perf_counter() - t1) / (n_scans // 4)
    return {"workload": "128 x 2048 scan (262144 points, 3 MiB) per step, pinned host points, "
                        "2-slot pipeline; results read back",
            "scans_per_s": n_scans / span, "ms_per_scan": 1e3 * span / n_scans,
            "latency_p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "latency_p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "serial_copy_then_eval_ms": 1e3 * serial,
            "budget_ms_at_20Hz": 50.0}


def l2_probe(ctx) -> dict:
    """L2 read bandwidth: the library's probe kernel reads a 32 MiB buffer (resident in the
    129 MB L2) 200 times with 16-byte loads that bypass L1, on every SM; best of 5 launches
    by CUDA events.  GB/s = bytes read / time."""
    import torch
    from paper_2301_08068_gb300 import rmp as R
    buf = torch.ones(32 << 20, dtype=torch.uint8, device="cuda")
    chk = torch.zeros(4096, dtype=torch.int64, device="cuda")
    passes = 200
    for _ in range(2):
        R.rmp_probe_l2_read(ctx.handle, buf, passes, chk)
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R.rmp_probe_l2_read(ctx.handle, buf, passes, chk)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return {"GBps": buf.numel() * passes / (best / 1e3) / 1e9, "bytes": buf.numel(),
            "passes": passes,
            "probe": "rmp_probe_l2_read: 32 MiB read 200 times (ld.global.cg, 16 B per load)"}


def rollout_section(ctx) -> dict:
    """Closed loop (Sec. IV-A): 128 start/goal pairs across seeded 10 m maps, point robots
    driven by the raycasting policy combined with the goal attractor (Table I static-map
    gains), dt = 10 ms, up to 60 s; success (goal reached without collision) and path
    smoothness against the ray count N^2 (the paper's Fig. 6-7 sweep), with the time per
    control step of all 128 robots; both readings of the ray metric in the combination
    (sum as printed in Eq. raytracing_policy, mean as the text describes)."""
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    out = {"workload": "128 start/goal pairs per map (x 0.5-1.5 m -> 8.5-9.5 m), 10 m cube, "
                       "dt 10 ms, <= 6000 steps, goal tolerance 0.2 m, static-map params, "
                       "alpha_g 10, beta_g 15"}
    for n_prims, size in ((200, (0.2, 0.6)), (50, (0.2, 2.0))):
        t = W.rollout_tasks(128, n_prims=n_prims, size_range=size)
        mid = ctx.upload(t.map)
        p = R.make_params(t.params, t.max_range)
        robots = np.concatenate([t.starts, np.zeros_like(t.starts), t.goals], axis=1)
        # the ESDF single-query policy (Sec. III-D) on the same start/goal pairs
        eid = R.rmp_esdf_upload(ctx.handle, t.prims)
        rp = R.rollout_params(10.0, 15.0, 0.01, 0.2, 6000, 10, 1)
        t0 = time.perf_counter()
        res = R.rmp_rollout_esdf(ctx.handle, mid, eid, robots, p, rp)
        wall = time.perf_counter() - t0
        R.rmp_esdf_release(ctx.handle, eid)
        st = np.array([r["status"] for r in res])
        steps = np.array([r["steps"] for r in res])
        ok = st == R.RMP_ROLLOUT_REACHED
        out["%d_prims_%g-%gm_esdf" % (n_prims, size[0], size[1])] = {
            "policy": "ESDF single query (exact distance and gradient of the primitives)",
            "success": float(ok.mean()), "collided": float((st == R.RMP_ROLLOUT_COLLIDED).mean()),
            "timeout": float((st == R.RMP_ROLLOUT_TIMEOUT).mean()),
            "smoothness_success_mean": float(np.mean([r["smoothness"] for r, o in zip(res, ok)
                                                      if o])) if ok.any() else None,
            "steps_max": int(steps.max()), "wall_s": wall,
            "ms_per_control_step": 1e3 * wall / max(1, int(steps.max()))}
        for mean in (True, False):
            rows = []
            for side in (4, 8, 16, 32, 64):
                rp = R.rollout_params(10.0, 15.0, 0.01, 0.2, 6000, 10, side * side,
                                      metric_mean=mean)
                t0 = time.perf_counter()
                res = R.rmp_rollout(ctx.handle, mid, robots, p, rp)
                wall = time.perf_counter() - t0
                st = np.array([r["status"] for r in res])
                steps = np.array([r["steps"] for r in res])
                ok = st == R.RMP_ROLLOUT_REACHED
                rows.append({"rays": side * side, "success": float(ok.mean()),
                             "collided": float((st == R.RMP_ROLLOUT_COLLIDED).mean()),
                             "timeout": float((st == R.RMP_ROLLOUT_TIMEOUT).mean()),
                             "smoothness_success_mean":
                                 float(np.mean([r["smoothness"] for r, o in zip(res, ok) if o]))
                                 if ok.any() else None,
                             "steps_max": int(steps.max()), "wall_s": wall,
                             "ms_per_control_step": 1e3 * wall / max(1, int(steps.max())),
                             "robot_steps_per_s": float(steps.sum()) / wall})
            out["%d_prims_%g-%gm_%s" % (n_prims, size[0], size[1],
                                        "mean" if mean else "sum")] = rows
        R.rmp_map_release(ctx.handle, mid)
    return out


def serve_section(ctx, seconds: float) -> dict:
    """Served: a Poisson stream (20k requests/s) over three device-resident maps (dense
    128^3 at 0.05 m, hashed 40x40x10 m at 0.1 m, hashed 100x100x20 m at 0.2 m; max range
    10 m) with requests of 1024..262144 rays (log-uniform), fed in real time to the
    continuous-batching server (256 MiB device-memory budget), and the same stream served
    by the plain kernel one request at a time (FIFO); latency = completion - arrival."""
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    wls = W.served_workloads(64)
    mids = [ctx.upload(w.map) for w in wls]
    params = [R.make_params(w.params, w.max_range) for w in wls]
    t_arr, maps, rays, vel = W.poisson_requests(3, 20000.0, seconds, 1024, 262144)
    n = len(t_arr)
    reqs = []
    for i in range(n):
        w = wls[maps[i]]
        s = w.states[i % len(w.states)]
        reqs.append((int(maps[i]), s.x, vel[i], int(rays[i])))
    total_rays = float(np.sum(rays))

    def pct(lat):
        return {"p50_ms": float(np.percentile(lat, 50)) * 1e3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                "mean_ms": float(np.mean(lat)) * 1e3}

    out = {"workload": "Poisson 20000 req/s for %.2f s (%d requests, %.3g rays), 3 maps, "
                       "1024..262144 rays log-uniform" % (seconds, n, total_rays)}
    # warm both paths
    with R.Server(ctx, slots=4, max_batch_states=256, max_rays=262144,
                  mem_budget_bytes=256 << 20) as srv:
        for m in range(3):
            srv.wait(srv.submit(mids[m], wls[m].states[0].x, wls[m].states[0].xdot, 4096,
                                params[m]))
        import threading
        me = threading.get_native_id()
        cpu0 = thread_cpu_seconds(me)
        tickets = []
        t0 = time.perf_counter()
        for i, (m, x, v, r) in enumerate(reqs):
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            tickets.append(srv.submit(mids[m], x, v, r, params[m]))
        lat = []
        for t in tickets:
            res, l = srv.wait(t, 60000)
            assert res["status"] == 0
            lat.append(l)
        span = time.perf_counter() - t0
        cpu = thread_cpu_seconds(me) - cpu0
        st = srv.stats()
    out["served"] = dict(pct(lat), Grays_per_s=total_rays / span / 1e9, makespan_s=span,
                         batches=st["batches"], mean_batch=st["batched_states"] / max(1, st["batches"]),
                         max_inflight=st["max_inflight"], mem_high_water=st["mem_high_water"],
                         library_threads_cpu_per_s=cpu / span)
    # the plain kernel, one request at a time in arrival order
    for m in range(3):
        R.rmp_raycast_eval(ctx.handle, mids[m], wls[m].states[0].x, wls[m].states[0].xdot, 4096,
                           params[m])
    lat = []
    t0 = time.perf_counter()
    for i, (m, x, v, r) in enumerate(reqs):
        while time.perf_counter() - t0 < t_arr[i]:
            pass
        res = R.rmp_raycast_eval(ctx.handle, mids[m], x, v, r, params[m])
        lat.append(time.perf_counter() - t0 - t_arr[i])
    span = time.perf_counter() - t0
    out["plain_per_request"] = dict(pct(lat), Grays_per_s=total_rays / span / 1e9,
                                    makespan_s=span)
    out["load_sweep"] = load_sweep(ctx, mids, params, wls)
    ok = [r["rate_req_s"] for r in out["load_sweep"] if r["server"]["p99_ms"] < 1.0]
    out["max_rate_p99_under_1ms"] = max(ok) if ok else None
    for m in mids:
        R.rmp_map_release(ctx.handle, m)
    return out


def thread_cpu_seconds(exclude_tid: int) -> float:
    """CPU time (user + system) of this process's threads other than exclude_tid, from
    /proc (0 where /proc is unavailable)."""
    tot = 0.0
    tick = os.sysconf("SC_CLK_TCK") if hasattr(os, "sysconf") else 100
    try:
        for tid in os.listdir("/proc/self/task"):
            if int(tid) == exclude_tid:
                continue
            with open("/proc/self/task/%s/stat" % tid) as f:
                fields = f.read().rsplit(")", 1)[1].split()
            tot += (int(fields[11]) + int(fields[12])) / tick
    except (OSError, ValueError, IndexError):
        return 0.0
    return tot


def load_sweep(ctx, mids, params, wls, seconds: float = 0.25) -> list:
    """The served stream at several offered loads (Poisson, 5k..80k requests/s for
    `seconds` each, same maps and ray-count law): server against the plain kernel one
    request at a time (FIFO), p50/p99 latency, achieved Grays/s, mean batch size, and the
    CPU time the library's threads (server worker, CUDA callbacks) used per second."""
    import threading
    from paper_2301_08068_gb300 import rmp as R, workloads as W
    rows = []
    me = threading.get_native_id()
    for rate in (5000.0, 10000.0, 20000.0, 40000.0, 80000.0):
        t_arr, maps, rays, vel = W.poisson_requests(3, rate, seconds, 1024, 262144,
                                                    seed_index=40 + int(rate) // 1000)
        reqs = [(int(maps[i]), wls[maps[i]].states[i % len(wls[maps[i]].states)].x, vel[i],
                 int(rays[i])) for i in range(len(t_arr))]
        total = float(np.sum(rays))
        row = {"rate_req_s": rate, "requests": len(reqs), "offered_Grays_per_s": total / seconds / 1e9}
        with R.Server(ctx, slots=4, max_batch_states=256, max_rays=262144,
                      mem_budget_bytes=256 << 20) as srv:
            srv.wait(srv.submit(mids[1], wls[1].states[0].x, wls[1].states[0].xdot, 4096, params[1]))
            cpu0 = thread_cpu_seconds(me)
            t0 = time.perf_counter()
            tickets = []
            for i, (m, x, v, r) in enumerate(reqs):
                while time.perf_counter() - t0 < t_arr[i]:
                    pass
                tickets.append(srv.submit(mids[m], x, v, r, params[m]))
            lat = []
            for tk in tickets:
                res, l = srv.wait(tk, 60000)
                lat.append(l)
            span = time.perf_counter() - t0
            cpu = thread_cpu_seconds(me) - cpu0
            st = srv.stats()
        row["server"] = {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                         "Grays_per_s": total / span / 1e9,
                         "mean_batch": st["batched_states"] / max(1, st["batches"]),
                         "library_threads_cpu_per_s": cpu / span}
        lat = []
        t0 = time.perf_counter()
        for i, (m, x, v, r) in enumerate(reqs):
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            R.rmp_raycast_eval(ctx.handle, mids[m], x, v, r, params[m])
            lat.append(time.perf_counter() - t0 - t_arr[i])
        span = time.perf_counter() - t0
        row["plain"] = {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                        "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                        "Grays_per_s": total / span / 1e9}
        rows.append(row)
    return rows


def oracle_configs(cores: int, gpu_batch: dict) -> dict:
    """The oracle (unchanged single-threaded C) on configs 1, 3, 4 and 5, on one core and on
    every host core (one evaluation per thread at once), in rays (points) per second; and
    config 4's precision: each of the 256 states of the batch against the FP64 oracle, for
    both GPU reductions (gpu_batch: batch_section's per-state results)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O
    from paper_2301_08068_gb300 import workloads as W
    out = {}
    pool = ThreadPoolExecutor(cores)

    def rate(fn, items, rays_of, sample: str):
        t0 = time.perf_counter()
        fn(items[0])
        one = time.perf_counter() - t0
        t0 = time.perf_counter()
        res = list(pool.map(fn, items))
        wall = time.perf_counter() - t0
        n_all = float(sum(rays_of(i) for i in items))
        return {"single_thread_rays_per_s": rays_of(items[0]) / one,
                "all_cores_rays_per_s": n_all / wall, "cores": cores, "sample": sample}, res

    # config 1: dense 64^3, 1024 rays
    w1 = W.dense_box_workload(n_states=2 * cores, jitter=True)
    om1 = O.OracleMap(w1.map)
    p1 = O.make_params(w1.params, w1.max_range)
    out["config1"], _ = rate(lambda s: O.raycast_eval(om1, s.x, s.xdot, w1.n_rays, p1,
                                                      want_hits=False, want_per_ray=False),
                             w1.states, lambda s: w1.n_rays,
                             "%d states x 1024 rays" % len(w1.states))
    # config 3: 64 x 1024 scan
    sw = W.lidar_workload()
    p3 = O.make_params(sw.params, sw.max_range)
    out["config3"], _ = rate(lambda k: O.scan_eval(sw.points, sw.x, sw.xdot, p3,
                                                   want_per_ray=False),
                             list(range(cores)), lambda k: len(sw.points),
                             "%d scans of 65536 points" % cores)
    # config 4: all 256 states of the batch (5.26 M rays), and the precision per state
    w4 = W.hashed_workload(n_states=256, uneven_rays=(4096, 65536))
    om4 = O.OracleMap(w4.map)
    p4 = O.make_params(w4.params, w4.max_range)
    idx = list(range(256))
    out["config4"], orc = rate(lambda b: O.raycast_eval(om4, w4.states[b].x, w4.states[b].xdot,
                                                        int(w4.n_rays[b]), p4, want_hits=False,
                                                        want_per_ray=False)[0],
                               idx, lambda b: int(w4.n_rays[b]),
                               "the 256 states of the batch, %d rays" % int(np.sum(w4.n_rays)))
    if gpu_batch:
        prec = {}
        for name, res in gpu_batch.items():
            eA, ef, cond = [], [], []
            for g, o in zip(res, orc):
                eA.append(float(np.abs(g["sumA"] - o["sumA"]).max() /
                                max(np.abs(o["sumA"]).max(), 1e-300)))
                ef.append(float(np.linalg.norm(g["f"] - o["f"]) /
                                max(np.linalg.norm(o["f"]), 1e-300)))
                lam = o["eig"]
                cond.append(float(lam.max() / lam.min()) if lam.min() > 0 else float("inf"))
            worst = int(np.argmax(ef))
            prec[name] = {"sumA_rel_max": max(eA), "sumA_rel_median": float(np.median(eA)),
                          "f_rel_max": max(ef), "f_rel_median": float(np.median(ef)),
                          "f_rel_max_state": worst, "cond_of_worst_state": cond[worst],
                          "states": len(ef),
                          "f_rel_per_state": [float("%.3g" % e) for e in ef]}
        out["config4_precision"] = prec
    # config 5: a sample of the served stream's requests over the three maps
    wls = W.served_workloads(64)
    oms = [O.OracleMap(w.map) for w in wls]
    ps = [O.make_params(w.params, w.max_range) for w in wls]
    t_arr, maps, rays, vel = W.poisson_requests(3, 20000.0, 2.0, 1024, 262144)
    pick = list(range(0, len(maps), max(1, len(maps) // (4 * cores))))[:4 * cores]
    out["config5"], _ = rate(lambda i: O.raycast_eval(oms[maps[i]],
                                                      wls[maps[i]].states[i % 64].x, vel[i],
                                                      int(rays[i]), ps[maps[i]], want_hits=False,
                                                      want_per_ray=False),
                             pick, lambda i: int(rays[i]),
                             "%d requests of the served stream" % len(pick))
    pool.shutdown()
    return out


def run_reference(args):
    """The oracle on every core of this host, one evaluation per thread at once.  Each step
    evaluates a bounded sample of the workload -- the first m rays of one state per thread --
    with m sized so that warm-up plus timed steps take about --ref-seconds in total."""
    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    wl = workload(0)
    import oracle as O
    om = O.OracleMap(wl.map)
    p = O.make_params(wl.params, wl.max_range)
    s0 = wl.states[0]
    t = time.perf_counter()
    O.raycast_eval(om, s0.x, s0.xdot, 4096, p, want_hits=False, want_per_ray=False)
    per_ray = (time.perf_counter() - t) / 4096
    cores = host_cores()
    budget = args.ref_seconds / max(1, args.steps + args.warmup)   # wall seconds per step
    m = int(min(N_RAYS, max(256, budget / per_ray)) // 256 * 256)
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(cores)              # one pool for every step
    for i in range(args.warmup):
        st = [wl.states[(i * cores + c) % N_STATES] for c in range(cores)]
        oracle_on_threads(om, p, st, m, cores, cores, pool)
    times = []
    for i in range(args.steps):
        st = [wl.states[(i * cores + c) % N_STATES] for c in range(cores)]
        times.append(oracle_on_threads(om, p, st, m, cores, cores, pool))
    pool.shutdown()
    ms = 1e3 * sum(times) / len(times)
    value = cores * m / (ms / 1e3) / 1e9
    sample = ("each step: the first %d of the 65536 Halton rays of %d states of the workload, "
              "the single-threaded C oracle on %d host threads at once" % (m, cores, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_rays": N_RAYS, "states": N_STATES,
                   "rays_per_step_sample": m},
        "evals_per_s": value * 1e9 / N_RAYS,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample,
                         "host": {"cpu": host_cpu_model(), "nproc": os.cpu_count()}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(strict_json(line), allow_nan=False), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2301_08068_gb300 import rmp as R

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    wl = workload(rank)
    ctx = R.Context(local_rank)
    mid = ctx.upload(wl.map)
    params = R.make_params(wl.params, wl.max_range)
    states = torch.tensor(np.stack([np.concatenate([s.x, s.xdot]) for s in wl.states]),
                          dtype=torch.float64, device=dev)
    ws = torch.empty(R.rmp_workspace_bytes(), dtype=torch.uint8, device=dev)
    R.rmp_workspace_init(ws)
    outs = torch.empty((N_STATES, R.RESULT_BYTES), dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # algorithmic bytes per launch from the exact per-ray step and block counts
    hits = torch.empty(N_RAYS * 24, dtype=torch.uint8, device=dev)
    alg, steps_per_launch = [], []
    for i in range(N_STATES):
        R.rmp_raycast_eval_async(ctx.handle, mid, states[i], N_RAYS, params, ws, outs[i], hits=hits)
        h = hits.cpu().numpy().view(R.HIT_DTYPE)
        alg.append(float(((h["steps"].astype(np.int64) + 1) * 4).sum() +
                         16 * h["blocks"].astype(np.int64).sum()))
        steps_per_launch.append(float(h["steps"].astype(np.int64).sum()))
    launch = R.rmp_eval_launch_info(ctx.handle, mid, N_RAYS, params)
    grid = launch["grid"]
    alg_bytes = float(np.mean(alg)) + grid * 80 + 48 + 144

    # the states in an order stratified by their voxel-step counts (their cost): rank r of
    # the sorted counts goes to position bitreverse(r), so every prefix of the timed steps
    # (20 of the 64 states, say) spans the workload's range of costs evenly, and a short
    # run measures the same mix as a long one
    order = stratified_order(steps_per_launch)

    def step(i):
        j = order[i % N_STATES]
        R.rmp_raycast_eval_async(ctx.handle, mid, states[j], N_RAYS, params, ws, outs[j])

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the clock sampler starts (and settles) before the warm-up, so the warm-up steps, with
    # the same L2 flush between them as the timed ones, run right before the timed loop;
    # while it starts, untimed evaluations keep the GPU busy (an idle GPU needs more than a
    # few steps to come back to speed: 5 warm-up steps after 0.3 s idle measured 62.3 us,
    # 50 steps 59.2 us)
    clocks = ClockSampler(local_rank)
    clocks.start()
    t_end = time.perf_counter() + PREWARM_S
    n_pre = 0
    while time.perf_counter() < t_end:
        flush.fill_(n_pre & 0xFF)
        step(n_pre)
        n_pre += 1
        if n_pre % 32 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        step(i)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                 # evict L2 between timed evaluations
        ev[i][0].record()
        step(i)
        ev[i][1].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    per = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(per))
    ms_max = max_over_ranks(ms, dev, world)

    # check the results are real (finite, status ok) -- outside the timed region
    res = [R.result_from_bytes(outs[i].cpu().numpy().tobytes()) for i in range(N_STATES)]
    assert all(r["status"] == 0 and np.all(np.isfinite(r["f"])) for r in res)

    # the same evaluation with the per-ray outputs on (hit records 24 B and f, A 36 B per ray)
    hits_on = None
    if rank == 0 and world == 1 and not args.no_extra:
        per_ray = torch.empty(N_RAYS * 9, dtype=torch.float32, device=dev)
        evo = []
        for i in range(max(3, min(args.warmup, 50)) + 2000):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            j = order[i % N_STATES]
            R.rmp_raycast_eval_async(ctx.handle, mid, states[j], N_RAYS, params, ws,
                                     outs[j], hits=hits, per_ray=per_ray)
            b.record()
            evo.append((a, b))
        torch.cuda.synchronize()
        t_on = [a.elapsed_time(b) for a, b in evo[-2000:]]
        hits_on = {"outputs": "hit records and per-ray f, A (60 B per ray, 3.9 MB per launch)",
                   "ms_per_step": float(np.mean(t_on)),
                   "ms_per_step_p50": float(np.percentile(t_on, 50)),
                   "Grays_per_s": N_RAYS / float(np.mean(t_on)) / 1e6, "steps": 2000}

    # end to end through the public synchronous call with host buffers (after as many
    # untimed calls as there are warm-up steps, at least 200, so the host path is warm too)
    n_e2e = max(1, min(args.steps, 2000))
    for i in range(max(args.warmup, 200)):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        s = wl.states[order[i % N_STATES]]
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, N_RAYS, params)
    e2e_t = []
    for i in range(n_e2e):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        s = wl.states[order[i % N_STATES]]
        t = time.perf_counter()
        R.rmp_raycast_eval(ctx.handle, mid, s.x, s.xdot, N_RAYS, params)
        e2e_t.append(time.perf_counter() - t)
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    e2e_ms_max = max_over_ranks(e2e_ms, dev, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, secs, _ = time_oracle(wl, args.cpu_seconds, 200)
        one = n * N_RAYS / secs / 1e9
        import oracle as O
        cores = host_cores()
        # all cores: about cpu_seconds of CPU work in total, two evaluations per thread at least
        evals = max(2 * cores, int(round(args.cpu_seconds / (secs / n))))
        wall = oracle_on_threads(O.OracleMap(wl.map), O.make_params(wl.params, wl.max_range),
                                 wl.states, N_RAYS, cores, evals)
        cpu = {"value": evals * N_RAYS / wall / 1e9, "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": "%d full evaluations (65536 rays each) of the workload's states, the "
                         "single-threaded C oracle on %d host threads at once (independent "
                         "states), %.2f s wall" % (evals, cores, wall),
               "single_core": {"value": one, "unit": UNIT, "cores": 1,
                               "sample": "%d full evaluations, one thread pinned to one core, "
                                         "%.1f s" % (n, secs)},
               "host": {"cpu": host_cpu_model(), "nproc": os.cpu_count()}}

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["config1_dense"] = config1_section(ctx, flush)
        extra["lidar"] = lidar_section(ctx, flush)
        extra["lidar_stream_os0"] = lidar_stream_section(ctx)
        extra["batched"] = batch_section(ctx, mid, flush, per_state=cpu is not None)
        extra["served"] = serve_section(ctx, args.serve_seconds)
        extra["rollout"] = rollout_section(ctx)
    if cpu is not None:
        gb = extra.get("batched", {}).pop("_results", None)
        cpu["configs"] = oracle_configs(host_cores(), gb)

    src = kernel_source_hash(launch)
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (ms / 1e3) / 1e9
    # the kernel's bound: the serial integer DDA chain (INT_OPS_PER_STEP per voxel step)
    # against every SM's integer lanes at the sampled SM clock
    sm_mhz = clk.get("sm_mhz") or 2070.0
    alu_ops = float(np.mean(steps_per_launch)) * INT_OPS_PER_STEP
    alu_peak = SM_COUNT * INT_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    alu_achieved = alu_ops / (ms / 1e3) / 1e12
    counters = committed_counters(src)
    traffic = counters.get("dram_bytes_per_launch")
    l2 = l2_probe(ctx) if rank == 0 else None
    l2_bytes = counters.get("lts_bytes_per_launch")
    insts = counters.get("warp_inst_per_launch")
    if rank == 0:
        value = whole_job_rate(world, N_RAYS, ms_max)
        # compact scalars of the other configs (kept beside the workload description)
        summary = {"ms_per_step_p50": float(np.percentile(per, 50))}
        try:
            if "config1_dense" in extra:
                summary["c1_dense_1024_us_per_eval"] = extra["config1_dense"]["us_per_eval"]
            if "lidar" in extra:
                summary["c3_lidar_64x1024_us_per_scan"] = 1e3 * extra["lidar"]["ms_per_scan"]
            if "batched" in extra:
                b = extra["batched"]
                summary["c4_batch256_Grays_per_s"] = b["kahan_fp32"]["Grays_per_s"]
                summary["c4_batch256_ms"] = b["kahan_fp32"]["ms_per_batch"]
                summary["c4_batch256_fp64_Grays_per_s"] = b["fp64"]["Grays_per_s"]
            if cpu is not None and "config4_precision" in cpu.get("configs", {}):
                pr = cpu["configs"]["config4_precision"]
                summary["c4_f_rel_err_max_kahan32"] = pr["kahan_fp32"]["f_rel_max"]
                summary["c4_f_rel_err_median_kahan32"] = pr["kahan_fp32"]["f_rel_median"]
                summary["c4_sumA_rel_err_max_kahan32"] = pr["kahan_fp32"]["sumA_rel_max"]
            if "served" in extra:
                sv = extra["served"]
                summary["c5_served_p50_ms"] = sv["served"]["p50_ms"]
                summary["c5_served_p99_ms"] = sv["served"]["p99_ms"]
                summary["c5_served_Grays_per_s"] = sv["served"]["Grays_per_s"]
                summary["c5_plain_p50_ms"] = sv["plain_per_request"]["p50_ms"]
                summary["c5_max_rate_p99_under_1ms"] = sv.get("max_rate_p99_under_1ms")
            if "rollout" in extra:
                ro = extra["rollout"]
                summary["rollout_ray1024_success"] = ro["200_prims_0.2-0.6m_mean"][3]["success"]
                summary["rollout_esdf_success"] = ro["200_prims_0.2-0.6m_esdf"]["success"]
        except (KeyError, IndexError, TypeError):
            pass
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_rays": N_RAYS, "states": N_STATES,
                       "map_blocks": wl.map.n_blocks, "parallelism": "replicas x%d" % world,
                       "l2": "flushed between timed steps (256 MiB write outside the events)",
                       "state_order": "stratified by voxel-step count (every prefix of the "
                                      "timed steps spans the states' cost range)",
                       "prewarm": "untimed evaluations for %.1f s (%d) while the clock sampler "
                                  "starts, then the %d warm-up steps" % (PREWARM_S, n_pre,
                                                                          args.warmup),
                       "launch": launch, **summary},
            "evals_per_s": world * 1e3 / ms_max,
            "ms_per_step_p50": float(np.percentile(per, 50)),
            "ms_per_step_p99": float(np.percentile(per, 99)),
            "timed_wall_s": wall,
            "e2e": {"value": whole_job_rate(world, N_RAYS, e2e_ms_max), "unit": UNIT,
                    "h2d_bytes_per_step": 48, "d2h_bytes_per_step": R.RESULT_BYTES,
                    "ms_per_call": e2e_ms, "calls": n_e2e,
                    "path": "rmp_raycast_eval from Python, host x/xdot in and host result out: "
                            "the 48-byte state travels in the kernel launch's parameter block, "
                            "the kernel writes the 144-byte result into mapped pinned host "
                            "memory, the call returns after a stream synchronisation"},
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                         "unit": "Tops/s", "frac": alu_achieved / alu_peak, "traffic": traffic,
                         "peak_source": "%d SMs x %d int32 lanes x sampled SM clock %.0f MHz "
                                        "(derived)" % (SM_COUNT, INT_LANES_PER_SM, sm_mhz),
                         "algorithmic": "%d integer operations per voxel step of the plain "
                                        "exact DDA x %.0f voxel steps per launch (from the "
                                        "kernel's hit records)" %
                                        (INT_OPS_PER_STEP, float(np.mean(steps_per_launch))),
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind,
                                 "algorithmic_bytes_per_launch": alg_bytes,
                                 "dram_bytes_per_launch": traffic},
                         "l2": {"achieved": (l2_bytes / (ms / 1e3) / 1e9) if l2_bytes else None,
                                "peak": l2["GBps"] if l2 else None, "unit": "GB/s",
                                "frac": (l2_bytes / (ms / 1e3) / 1e9 / l2["GBps"])
                                        if (l2_bytes and l2) else None,
                                "bytes_per_launch": l2_bytes,
                                "bytes_source": "ncu lts__t_bytes.sum of the committed capture",
                                "probe": l2},
                         "issue": {"frac": (insts / (4 * SM_COUNT * sm_mhz * 1e6 * ms / 1e3))
                                           if insts else None,
                                   "warp_instructions_per_launch": insts,
                                   "schedulers": 4 * SM_COUNT,
                                   "what": "warp instructions (committed ncu capture) / "
                                           "(schedulers x cycles of the measured mean time)"},
                         "kernel": "raycast_rmp_kernel<hashed TSDF, grid layout, "
                                   "compensated FP32 reduction>",
                         "kernel_launch_sha256_16": src},
            "per_ray_outputs_on": hits_on,
            "cpu_baseline": cpu,
            "gpu_launches": args.steps,
            **extra,
            "clocks": clk,
            "paper_context": {"value": PAPER_RATE, "unit": UNIT,
                              "note": "65536 rays at up to 3 kHz (abstract), unnamed GPU of "
                                      "Jetson NX / MX150 / Titan Xp, different map"},
        }
        print(json.dumps(strict_json(line), allow_nan=False), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
