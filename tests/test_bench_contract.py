"""CPU checks of bench.py: the reference arm (the oracle on the host cores) prints one JSON
line with the keys the benchmark contract names, the whole-job rate arithmetic, and the
rule that the committed ncu traffic is reported only for the launch it was taken on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--ref-seconds", "2"],
                         capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "gpu_launches"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["gpu_launches"] == 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == bench.host_cores()
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_whole_job_rate():
    assert bench.whole_job_rate(1, 65536, 0.0685) == pytest.approx(65536 / 68.5e-6 / 1e9)
    assert bench.whole_job_rate(4, 65536, 0.0685) == pytest.approx(4 * 65536 / 68.5e-6 / 1e9)
    assert bench.max_over_ranks(3.5, None, 1) == 3.5


def test_traffic_only_for_the_captured_launch():
    d = json.load(open(os.path.join(ROOT, "profiles", "raycast_hashed_65536_traffic.json")))
    got = bench.committed_counters(d["kernel_launch_sha256_16"])
    assert got["dram_bytes_per_launch"] == d["dram_bytes_per_launch"]
    assert bench.committed_counters("0" * 16) == {}
    launch = {"block": 256, "grid": 256, "lg_segments": 0, "ray_cells": 1296, "smem_bytes": 16256}
    other = dict(launch, block=128, grid=512)
    assert bench.kernel_source_hash(launch) == bench.kernel_source_hash(dict(launch))
    assert bench.kernel_source_hash(launch) != bench.kernel_source_hash(other)
    # occupancy and SM count are not part of the identity
    assert bench.kernel_source_hash(launch) == bench.kernel_source_hash(
        dict(launch, ctas_per_sm=2, sm_count=152))


def test_launch_identity_ignores_comments_and_layout():
    a = 'int a = 1;  // note\n/* block\n comment */ const char* s = "x // y /* z */";\n'
    b = 'int a = 1;\nconst char* s = "x // y /* z */";'
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only('int a = 1;') != bench.code_only('int a = 2;')
    assert '"x // y /* z */"' in bench.code_only(a)          # string literals are code


def test_strict_json_and_stratified_order():
    """The JSON line never carries non-finite numbers; the timed states' order samples the
    sorted costs evenly in every prefix (bit-reversed ranks)."""
    d = bench.strict_json({"a": float("inf"), "b": [1.0, float("nan")], "c": {"d": 2.5}})
    assert d == {"a": None, "b": [1.0, None], "c": {"d": 2.5}}
    json.dumps(d, allow_nan=False)
    costs = [5.0, 1.0, 4.0, 2.0, 8.0, 7.0, 6.0, 3.0]
    order = bench.stratified_order(costs)
    assert sorted(order) == list(range(8))
    ranks = sorted(range(8), key=lambda i: costs[i])
    assert [ranks.index(i) for i in order] == [0, 4, 2, 6, 1, 5, 3, 7]
    with pytest.raises(AssertionError):
        bench.stratified_order([1.0, 2.0, 3.0])
