"""Host-only checks of the library's launch policy (csrc/rmp_policy.h): the direction-cell
count, segments per ray, threads per CTA and grid size, scan shape and voxel-box use, run
through a small C++ program built from the same header and compared with the rules as
stated here.  No GPU is needed."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
WAVE = 152 * 2 * 256          # one wave of 256-thread CTAs at 2 CTAs per SM on 152 SMs
MAX_GRID = 4096


@pytest.fixture(scope="module")
def policy(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("policy") / "launch_policy_check")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2301_08068_gb300", "csrc"),
                           "-I", CUDA_INC, os.path.join(ROOT, "tests", "launch_policy_check.cpp"),
                           "-o", exe])

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        return [tuple(int(v) for v in row.split()) for row in out if row.strip()]
    return run


def _cells_rule(n):
    """M = 2^a 3^b with 32 M <= n closest to n / 48 cells, near-square cells (3^b ~ pi 2^a),
    by the stated score; M = 1 when no candidate fits."""
    best, best_score = 1, math.inf
    lt = math.log2(max(n / 48.0, 1.0))
    for a in range(25):
        for b in range(16):
            m = (1 << a) * 3 ** b
            if 32 * m > n:
                break
            score = abs(a + b * math.log2(3) - lt) + 0.5 * abs(b * math.log2(3) - math.log2(math.pi) - a)
            if score < best_score - 1e-12:
                best, best_score = m, score
    return best


def test_direction_cells(policy):
    ns = [1, 31, 32, 63, 64, 100, 777, 1024, 4096, 20000, 65536, 262144, 1 << 20, (1 << 24) - 1]
    got = policy(["pick %d" % n for n in ns])
    for n, (m, q, r) in zip(ns, got):
        assert m == _cells_rule(n), n
        assert q * m + r == n and 0 <= r < m
        assert m == 1 or 32 * m <= n                  # every cell holds at least 32 rays
        a = (m & -m).bit_length() - 1                 # M is 2^a 3^b
        rest = m >> a
        while rest % 3 == 0:
            rest //= 3
        assert rest == 1


def test_segments_per_ray(policy):
    cases = []
    for n in (1, 4096, 19456, 19457, 38912, 38913, 65536, 1 << 20, 4864, 4865, 9728, 9729,
              2432, 2433):
        cases.append((-1, n, WAVE))
    cases += [(-1, 4096, 0), (0, 4096, WAVE), (1, 65536, WAVE), (2, 65536, WAVE)]
    got = policy(["segs %d %d %d" % c for c in cases])
    for (tune, n, wave), (lg,) in zip(cases, got):
        if tune >= 0 or wave == 0:
            assert lg == 7                            # left to the tuned value / count rule
            continue
        expect = 5
        while expect > 0 and (n << expect) > wave:
            expect -= 1
        assert lg == expect, (n, lg)
    # the thresholds on this part: 32 segments up to 2432 rays, 16 up to 4864, 8 up to 9728,
    # 4 up to 19456, 2 up to 38912, else 1
    assert [g[0] for g in got[:14]] == [5, 4, 2, 1, 1, 0, 0, 0, 4, 3, 3, 2, 5, 4]


def test_single_state_shape(policy):
    cases = [(0, t, WAVE) for t in (1, 4096, WAVE, WAVE + 1, 1 << 20, 1 << 24)]
    cases += [(0, 65536, 0), (64, 65536, WAVE), (128, 1, WAVE), (256, 1 << 24, WAVE)]
    got = policy(["shape %d %d %d" % c for c in cases])
    for (tune, threads, wave), (block, grid) in zip(cases, got):
        expect_block = tune if tune else (256 if 0 < wave and threads <= wave else 128)
        assert block == expect_block, (tune, threads)
        assert grid == max(1, min(MAX_GRID, -(-threads // block)))


def test_scan_shape(policy):
    cases = [(0, 152, n) for n in (1, 4096, 65536, 262144, 1 << 22)]
    cases += [(128, 152, 262144), (64, 152, 262144), (0, 0, 4096)]
    got = policy(["scan %d %d %d" % c for c in cases])
    for (tune, sms, n), (block, grid) in zip(cases, got):
        b = tune or 256
        assert block == b
        cap = (512 // b) * max(sms, 1)                # at most 512 threads per SM
        assert grid == max(1, min(cap, -(-n // b)))


def test_voxel_box_use(policy):
    cases = [(t, lg) for t in (-1, 0, 1) for lg in (0, 1, 2)]
    got = policy(["cells %d %d" % c for c in cases])
    for (tune, lg), (kept,) in zip(cases, got):
        assert kept == (1 if tune == 1 or (tune == -1 and lg == 2) else 0), (tune, lg)
