"""Host-only test of the request server's device-memory allocator (csrc/rmp_arena.h): a C++
program drives it with seeded random allocations and releases and checks, after every
operation, that live blocks never overlap and stay inside the region, that the used byte
count matches the live blocks, that a request fails only when no free range is large
enough, and that releasing everything coalesces the region back into one free range."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_08068_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include <algorithm>
#include "rmp_arena.h"
using rmp::Arena;
static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
struct Blk { size_t off, bytes; };
int main() {
  const size_t size = 1 << 20;
  Arena a(size);
  std::vector<Blk> live;
  for (int op = 0; op < 200000; ++op) {
    if (live.empty() || rnd() % 3 != 0) {
      const size_t want = 1 + rnd() % 40000;
      const size_t largest = a.largest_free();
      const size_t off = a.alloc(want);
      if (off == Arena::kFail) {
        if (Arena::round(want) <= largest) { std::printf("spurious failure\n"); return 1; }
      } else {
        if (off % 256 || off + Arena::round(want) > a.size()) { std::printf("bad block\n"); return 1; }
        live.push_back({off, want});
      }
    } else {
      const size_t i = rnd() % live.size();
      a.release(live[i].off, live[i].bytes);
      live[i] = live.back();
      live.pop_back();
    }
    std::vector<Blk> v = live;
    std::sort(v.begin(), v.end(), [](const Blk& x, const Blk& y) { return x.off < y.off; });
    size_t used = 0;
    for (size_t i = 0; i < v.size(); ++i) {
      used += Arena::round(v[i].bytes);
      if (i + 1 < v.size() && v[i].off + Arena::round(v[i].bytes) > v[i + 1].off) {
        std::printf("overlap\n");
        return 1;
      }
    }
    if (used != a.used()) { std::printf("used mismatch\n"); return 1; }
  }
  for (const Blk& b : live) a.release(b.off, b.bytes);
  if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != a.size()) {
    std::printf("not coalesced\n");
    return 1;
  }
  std::printf("ok %zu\n", a.high_water());
  return 0;
}
"""


def test_arena_allocator(tmp_path):
    src = tmp_path / "arena.cpp"
    src.write_text(PROG)
    exe = tmp_path / "arena"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("ok")
