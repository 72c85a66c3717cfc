// rmp_policy.h -- launch policy of the evaluation kernels: host-only decisions taken from
// the ray count, the context's knobs and the measured occupancy (direction cells, segments
// per ray, threads per CTA, grid size, voxel-box use).  No CUDA calls, so the rules can be
// checked on a machine without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "rmp_internal.h"

namespace rmp {

// Launch knobs of a context (rmp_tune_set): -1 / 0 select the library's choice.
struct Tuning {
  // log2 segments per ray, ray order, split budget, threads per CTA, voxel boxes
  int lg_segs = -1, ray_order = 0, split = -1, block = 0, cells = -1;
};

// Coherent ray order: residue classes modulo M = 2^a 3^b are direction cells (see the
// kernel's ray_of_slot).  Cells hold >= 32 rays so a warp spans at most two of them, about
// n/48 cells, shaped close to square on the sphere (3^b ~ pi 2^a).
inline void pick_ray_cells(uint32_t n, EvalConsts* k) {
  // candidates M = 2^a 3^b with 32 M <= n, scored in log2 units with one logarithm per call:
  // |log2 M - log2(n / 48)| + 0.5 |log2(3^b / (pi 2^a))|
  const double L3 = 1.5849625007211562, LPI = 1.6514961294723187;   // log2 3, log2 pi
  const double lt = std::log2(std::max(n / 48.0, 1.0));
  uint64_t best = 1;
  double best_score = 1e300;
  for (int a = 0; a <= 24; ++a) {
    uint64_t m = 1ull << a;
    for (int b = 0; b <= 15 && m * 32ull <= n; ++b, m *= 3ull) {
      const double score = std::fabs(a + b * L3 - lt) + 0.5 * std::fabs(b * L3 - LPI - a);
      if (score < best_score) {
        best_score = score;
        best = m;
      }
    }
  }
  k->perm_M = (uint32_t)best;
  k->perm_Q = n / k->perm_M;
  k->perm_R = n % k->perm_M;
}

// Segments per ray of a single-state evaluation left to the library: as many (up to 32,
// kMaxSingleLgSegs) as keep the launch within one wave of 256-thread CTAs (`wave256`
// threads), since the evaluation lasts as long as its longest ray's serial march and
// segments shorten it while the extra threads still find free SMs (measured, L2 flushed:
// hashed map 1024 rays 33.0 / 26.6 / 22.0 / 19.9 us with 4 / 8 / 16 / 32 segments, 4096
// rays 33.5 / 26.7 / 23.7; dense 1024 rays 26.4 / 21.8 / 19.3 / 18.3; 16384 rays 54.3 us with 2 segments,
// 47.1 with 4; 32768 rays 65.5 with 1, 57.2 with 2; 65536 rays best with 1).  Without a
// wave size (0) the ray-count rule of make_consts stays.
constexpr uint32_t kMaxSingleLgSegs = 5;
inline void auto_segments(const Tuning& t, uint32_t n, uint64_t wave256, EvalConsts* k) {
  if (t.lg_segs >= 0 || wave256 == 0) return;
  uint32_t lg = kMaxSingleLgSegs;
  while (lg > 0 && ((uint64_t)n << lg) > wave256) --lg;
  k->lg_segs = lg;
}

// Voxel boxes in a single-state evaluation: as tuned, or (default) only with 4 or more
// segments per ray, where they pay (measured, 16384 rays: hashed 47.1 -> 44.6 us, dense 37.5 -> 36.6 us)
// -- with one segment per ray their extra dependent load lengthens the slowest warps
// (65536 rays: hashed 68.0 -> 71.2 us, dense 43.9 -> 49.4 us).
inline void single_state_cells(int tune_cells, const EvalConsts& k, DevMap* dm) {
  if (tune_cells == 1) return;
  if (tune_cells == 0 || k.lg_segs < 2) dm->cells = nullptr;
}

// n_threads: rays (or points) times segments per ray.  Threads per CTA: the tuned value, or
// (automatic) 256 when the whole launch fits in one wave of 256-thread CTAs (`wave256`
// threads; fewer CTAs stage the radius field and store partials: 65536 rays 69.7 -> 68.1 us
// hashed, 46.3 -> 43.8 us dense) and 128 otherwise (262144 rays: 132 against 135 us).
inline void launch_shape(const Tuning& t, uint64_t n_threads, uint64_t wave256, int* block,
                  int* grid) {
  int b = t.block;
  if (b == 0) b = (wave256 > 0 && n_threads <= wave256) ? 256 : 128;
  uint64_t g = (n_threads + b - 1) / b;
  if (g > (uint64_t)kMaxGrid) g = kMaxGrid;
  if (g < 1) g = 1;
  *block = b;
  *grid = (int)g;
}

// Scans: threads per CTA the tuned value or (automatic) 256, and at most 512 threads per
// SM, each thread striding over several points, so that large scans are reduced from few
// CTA partials (measured, L2 flushed: 4096 / 65536 / 262144 points 16.4 / 20.5 / 24.3 us
// with 128-thread CTAs and 4 per SM, 14.4 / 18.5 / 21.0 us with 256 and 2 per SM).
inline void scan_shape(const Tuning& t, int sm_count, uint64_t n, int* block, int* grid) {
  const int b = t.block != 0 ? t.block : 256;
  const uint64_t cap = (uint64_t)(512 / b) * (uint64_t)(sm_count > 0 ? sm_count : 1);
  uint64_t g = (n + b - 1) / b;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  *block = b;
  *grid = (int)g;
}

}  // namespace rmp
