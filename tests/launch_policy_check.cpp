// Runs the library's launch-policy functions (rmp_policy.h, host only) on commands read from
// stdin and prints one result line per command, for tests/test_launch_policy.py:
//   pick N              -> M Q R           (direction cells of N rays)
//   segs TUNE N WAVE    -> LG              (segments per ray of one state)
//   shape TUNE T WAVE   -> BLOCK GRID      (single-state launch of T threads)
//   scan TUNE SMS N     -> BLOCK GRID      (scan launch of N points)
//   cells TUNE LG       -> 1 if the voxel boxes stay on
#include <cstdio>
#include <cstring>

#include "rmp_policy.h"

int main() {
  char op[16];
  while (std::scanf("%15s", op) == 1) {
    rmp::EvalConsts k;
    std::memset(&k, 0, sizeof(k));
    rmp::Tuning t;
    if (!std::strcmp(op, "pick")) {
      unsigned n;
      if (std::scanf("%u", &n) != 1) return 2;
      rmp::pick_ray_cells(n, &k);
      std::printf("%u %u %u\n", k.perm_M, k.perm_Q, k.perm_R);
    } else if (!std::strcmp(op, "segs")) {
      int tune;
      unsigned n;
      unsigned long long wave;
      if (std::scanf("%d %u %llu", &tune, &n, &wave) != 3) return 2;
      t.lg_segs = tune;
      k.lg_segs = 7;                      // sentinel: untouched when the rule does not apply
      rmp::auto_segments(t, n, wave, &k);
      std::printf("%u\n", k.lg_segs);
    } else if (!std::strcmp(op, "shape")) {
      int tune;
      unsigned long long threads, wave;
      if (std::scanf("%d %llu %llu", &tune, &threads, &wave) != 3) return 2;
      t.block = tune;
      int block = 0, grid = 0;
      rmp::launch_shape(t, threads, wave, &block, &grid);
      std::printf("%d %d\n", block, grid);
    } else if (!std::strcmp(op, "scan")) {
      int tune, sms;
      unsigned long long n;
      if (std::scanf("%d %d %llu", &tune, &sms, &n) != 3) return 2;
      t.block = tune;
      int block = 0, grid = 0;
      rmp::scan_shape(t, sms, n, &block, &grid);
      std::printf("%d %d\n", block, grid);
    } else if (!std::strcmp(op, "cells")) {
      int tune;
      unsigned lg;
      if (std::scanf("%d %u", &tune, &lg) != 2) return 2;
      rmp::DevMap m;
      std::memset(&m, 0, sizeof(m));
      m.cells = reinterpret_cast<const uint32_t*>(&m);   // any non-null pointer
      k.lg_segs = lg;
      rmp::single_state_cells(tune, k, &m);
      std::printf("%d\n", m.cells != nullptr ? 1 : 0);
    } else {
      return 2;
    }
  }
  return 0;
}
