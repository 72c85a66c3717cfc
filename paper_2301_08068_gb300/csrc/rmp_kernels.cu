// rmp_kernels.cu -- sm_103a kernels of librmp: the fused raycast-RMP evaluation, the
// LiDAR scan policy and the map-build kernels.
//
// One evaluation is ONE launch: each thread generates its ray's Halton direction in
// registers (Sec. III-E, Eq. halton), marches it with an exact fixed-point DDA through
// the occupancy bricks (Sec. III-F; free blocks are crossed box by box through the free
// radius field staged in shared memory, and the 8^3 brick of an occupied block is held
// in registers -- in the batch kernel in shared memory -- so steps inside it touch no
// global memory), evaluates the obstacle policy (Sec. III-C), and the block reduces the
// 9 unique terms of sum A_i and sum A_i f_i (Fig. 3's block reduce) with a compensated
// FP32 tree (or FP64).  The last CTA to finish sums the per-CTA partials in a fixed order
// in FP64 and resolves Eq. (1) (FP32 Jacobi eigenvectors refined by FP64 Rayleigh
// quotients, FP64 adjugate solve at full rank), so the result is deterministic.
//
// Bit-exact steps (Halton direction, DDA, hit distance, the FP32 decisions that gate a
// ray) use explicitly rounded intrinsics (__fmul_rn, __fmaf_rn, ...) so that no
// contraction or fast-math rewrite can change them.
#include "rmp_internal.h"

namespace rmp {
namespace {

// ------------------------------------------------------------------ Halton directions
// Radical inverse base 2 of i, rounded to FP32 (exact for i < 2^24).
__device__ __forceinline__ float halton2(uint32_t i) {
  return __fmul_rn(__uint2float_rn(__brev(i)), 2.3283064365386963e-10f);  // * 2^-32
}

// The 20 base-3 digits of i (< 3^20) reversed: H(i,3) * 3^20.
__device__ __forceinline__ uint32_t halton3_numerator(uint32_t i) {
  uint32_t num = 0;
#pragma unroll
  for (int k = 0; k < 20; ++k) {
    uint32_t q = i / 3u;
    num = num * 3u + (i - 3u * q);
    i = q;
  }
  return num;
}

// num / 3^20 correctly rounded to FP32 with integer arithmetic only (FP64 division is
// slow on this GPU): scale num by 2^s so the quotient has exactly 24 significant bits,
// divide, and round to nearest on the remainder (no ties: 3^20 is odd).
__device__ __forceinline__ float halton3_f32(uint32_t num) {
  if (num == 0) return 0.0f;
  constexpr unsigned long long M = 3486784401ull;
  int s = 55 - (32 - __clz(num));
  unsigned long long X = (unsigned long long)num << s;
  if (X < (M << 23)) {
    X <<= 1;
    ++s;
  }
  unsigned long long q = X / M;
  unsigned long long rem = X - q * M;
  if (2ull * rem > M) ++q;
  return __fmul_rn(__ull2float_rn(q), __int_as_float((127 - s) << 23));
}

// cos and sin of 2*pi*v by a fixed FP32 recipe: octant q = floor(8v), fraction t,
// reduced angle a = x * RN(pi/4) (x = t, or 1 - t in odd octants), Taylor series of
// sin (through a^11) and cos (through a^12) with RN(1/n!) coefficients by Horner's rule
// with fused multiply-adds, then the octant's symmetry.
__device__ __forceinline__ void sincos_turns(float v, float& c_out, float& s_out) {
  constexpr float kPi4 = 0.78539816339744830962f;
  constexpr float f2 = 1.0f / 2.0f, f3 = 1.0f / 6.0f, f4 = 1.0f / 24.0f, f5 = 1.0f / 120.0f,
                  f6 = 1.0f / 720.0f, f7 = 1.0f / 5040.0f, f8 = 1.0f / 40320.0f,
                  f9 = 1.0f / 362880.0f, f10 = 1.0f / 3628800.0f, f11 = 1.0f / 39916800.0f,
                  f12 = 1.0f / 479001600.0f;
  const float w = __fmul_rn(v, 8.0f);
  const int q = __float2int_rz(w);
  const float t = __fsub_rn(w, __int2float_rn(q));
  const float x = (q & 1) ? __fsub_rn(1.0f, t) : t;
  const float a = __fmul_rn(x, kPi4);
  const float a2 = __fmul_rn(a, a);
  float ps = -f11;
  ps = __fmaf_rn(ps, a2, f9);
  ps = __fmaf_rn(ps, a2, -f7);
  ps = __fmaf_rn(ps, a2, f5);
  ps = __fmaf_rn(ps, a2, -f3);
  const float sa = __fmaf_rn(__fmul_rn(a2, a), ps, a);
  float pc = f12;
  pc = __fmaf_rn(pc, a2, -f10);
  pc = __fmaf_rn(pc, a2, f8);
  pc = __fmaf_rn(pc, a2, -f6);
  pc = __fmaf_rn(pc, a2, f4);
  pc = __fmaf_rn(pc, a2, -f2);
  const float ca = __fmaf_rn(a2, pc, 1.0f);
  const int o = q & 7;
  // octant o: angle = o*pi/4 + (t pi/4); odd octants measure a from the next multiple
  const bool swap = ((o + 1) & 2) != 0;          // octants 1,2,5,6: cos <-> sin
  float c = swap ? sa : ca;
  float s = swap ? ca : sa;
  if (o >= 2 && o <= 5) c = -c;                  // cos < 0 in octants 2..5
  if (o >= 4) s = -s;                            // sin < 0 in octants 4..7
  c_out = c;
  s_out = s;
}

struct Ray {
  float dir[3];
  int D[3];
};

__device__ __forceinline__ Ray make_ray(uint32_t i) {
  const float u = halton2(i);
  const float v = halton3_f32(halton3_numerator(i));
  const float z = __fsub_rn(1.0f, __fmul_rn(2.0f, u));
  const float st = __fmul_rn(2.0f, __fsqrt_rn(__fmul_rn(u, __fsub_rn(1.0f, u))));
  float c, s;
  sincos_turns(v, c, s);
  Ray r;
  r.dir[0] = __fmul_rn(st, c);
  r.dir[1] = __fmul_rn(st, s);
  r.dir[2] = z;
#pragma unroll
  for (int a = 0; a < 3; ++a) r.D[a] = __float2int_rn(__fmul_rn(r.dir[a], 16777216.0f));
  return r;
}

// ------------------------------------------------------------------ map access
__device__ __forceinline__ int hash_lookup(const DevMap& m, int bx, int by, int bz) {
  const unsigned long long key = (unsigned long long)(uint32_t)(bx + kKeyBias) |
                                 ((unsigned long long)(uint32_t)(by + kKeyBias) << 21) |
                                 ((unsigned long long)(uint32_t)(bz + kKeyBias) << 42);
  uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> m.hash_shift);
  for (uint32_t probe = 0; probe <= m.cap_mask; ++probe) {   // bounded: table has empties
    const unsigned long long k = __ldg(&m.table[h].key);
    if (k == key) return (int)__ldg(&m.table[h].slot);
    if (k == kEmptyKey) return -1;
    h = (h + 1) & m.cap_mask;
  }
  return -1;
}

// A brick held in registers: 16 occupancy words, loaded with four 128-bit loads.
struct Brick {
  uint4 q0, q1, q2, q3;
};

__device__ __forceinline__ void load_brick(const uint4* src, Brick& br) {
  br.q0 = __ldg(src);
  br.q1 = __ldg(src + 1);
  br.q2 = __ldg(src + 2);
  br.q3 = __ldg(src + 3);
}

// Occupancy of voxel k in the register brick: word (ly>>2) + 2 lz picked by a select
// tree (no local memory), bit lx + 8 (ly & 3) -- bit p = lx + 8 ly + 64 lz of the brick.
// The same test on a brick staged in shared memory word-major, by bit index p: word q of
// the lane's brick at sb[32 q] (sb = the warp's 16 x 32 words + lane), so a warp's lanes
// never share a bank.
__device__ __forceinline__ bool smem_brick_bit(const uint32_t* sb, uint32_t p) {
  return (sb[32 * (p >> 5)] >> (p & 31u)) & 1u;
}

__device__ __forceinline__ void store_smem_brick(const uint4* src, uint32_t* sb) {
  const uint4 q0 = __ldg(src), q1 = __ldg(src + 1), q2 = __ldg(src + 2), q3 = __ldg(src + 3);
  sb[0] = q0.x;   sb[32] = q0.y;  sb[64] = q0.z;  sb[96] = q0.w;
  sb[128] = q1.x; sb[160] = q1.y; sb[192] = q1.z; sb[224] = q1.w;
  sb[256] = q2.x; sb[288] = q2.y; sb[320] = q2.z; sb[352] = q2.w;
  sb[384] = q3.x; sb[416] = q3.y; sb[448] = q3.z; sb[480] = q3.w;
}

__device__ __forceinline__ bool brick_bit(const Brick& b, int kx, int ky, int kz) {
  const int lx = kx & 7, ly = ky & 7, lz = kz & 7;
  const int wi = (ly >> 2) + 2 * lz;
  const uint4 q = (wi & 8) ? ((wi & 4) ? b.q3 : b.q2) : ((wi & 4) ? b.q1 : b.q0);
  const uint32_t w = (wi & 2) ? ((wi & 1) ? q.w : q.z) : ((wi & 1) ? q.y : q.x);
  return (w >> (lx + 8 * (ly & 3))) & 1u;
}

// Free radius v of block (bx,by,bz): 0 if it holds an occupied voxel (then *src points at
// its brick), else v >= 1 with every block within Chebyshev distance v - 1 free.  Grid
// layout: the 4-bit field `rad` (shared memory when it fits); outside the grid's bounding
// box the radius is the distance to the box.  Hash layout: 1 for free blocks.
template <int LAYOUT>
__device__ __forceinline__ int block_radius(const DevMap& m, const uint32_t* rad, int bx, int by,
                                            int bz, const uint4** src, uint32_t* bidx = nullptr) {
  if (LAYOUT == kLayoutGrid) {
    const int x = bx - m.gmin[0], y = by - m.gmin[1], z = bz - m.gmin[2];
    if ((unsigned)x >= (unsigned)m.gdim[0] || (unsigned)y >= (unsigned)m.gdim[1] ||
        (unsigned)z >= (unsigned)m.gdim[2]) {
      const int dx = max(max(-x, x - (m.gdim[0] - 1)), 0);
      const int dy = max(max(-y, y - (m.gdim[1] - 1)), 0);
      const int dz = max(max(-z, z - (m.gdim[2] - 1)), 0);
      return min(max(dx, max(dy, dz)), kMaxFreeRadius);
    }
    const uint32_t idx = (uint32_t)x + (uint32_t)m.gdim[0] * ((uint32_t)y + (uint32_t)m.gdim[1] * (uint32_t)z);
    const int v = (int)((rad[idx >> 3] >> ((idx & 7) * 4)) & 15u);
    *src = m.bricks + 4 * (size_t)idx;
    if (bidx) *bidx = idx;
    return v;
  } else {
    const int slot = hash_lookup(m, bx, by, bz);
    if (slot < 0) return 1;
    *src = m.bricks + 4 * (size_t)slot;
    return 0;
  }
}

// ------------------------------------------------------------------ exact DDA (raycast R)
// Fixed point: P in 2^-16 voxel units, D in 2^-24 units.  N_a = distance (in P units)
// to the next boundary of axis a; the ray reaches it at t_a = N_a / |D_a|.  Each
// iteration steps the axis with the smallest t_a (cross-multiplied exactly in 64 bits;
// ties go to the lowest axis); an axis with D_a = 0 has |D_a| = 0, N_a = 1 and so never
// wins.  A voxel is entered only if N_a 2^24 <= R_fx |D_a|, i.e. N_a <= L_a.
// Blocks without occupied voxels are crossed in one step of integer arithmetic that
// reproduces the voxel-by-voxel crossings exactly (skip_box).
constexpr int kSegContinues = 0;   // piece ended at its upper parameter bound

__device__ __forceinline__ int min_axis(const uint32_t n[3], const uint32_t a[3]) {
  const bool ylx = (unsigned long long)n[1] * a[0] < (unsigned long long)n[0] * a[1];
  const uint32_t nw = ylx ? n[1] : n[0];
  const uint32_t aw = ylx ? a[1] : a[0];
  const bool zlw = (unsigned long long)n[2] * aw < (unsigned long long)nw * a[2];
  return zlw ? 2 : (ylx ? 1 : 0);
}

__device__ __forceinline__ uint32_t sel3(const uint32_t v[3], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

__device__ __forceinline__ float sel3f(const float v[3], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

template <int KIND>
__device__ __forceinline__ bool outside(const DevMap& m, const int k[3]) {
  return KIND == RMP_MAP_DENSE_U8 &&
         ((unsigned)k[0] >= (unsigned)m.dims[0] || (unsigned)k[1] >= (unsigned)m.dims[1] ||
          (unsigned)k[2] >= (unsigned)m.dims[2]);
}

// The ray is in a free box: the blocks within Chebyshev distance R of its current block, or
// the voxels within R of its current voxel (clipped to the dense grid).  Advance the DDA state to the first voxel beyond the box
// exactly as single steps would: the box is left through the axis e whose face crossing
// F_e/|D_e| comes first (ties: lowest axis); every other axis b crosses its interior
// boundaries that come strictly before that time (or at the same time if b < e, the tie
// order).  If the face crossing is beyond the limit, the ray ends inside the box after
// every crossing within the limit; returns true then.
//
// Per axis b the crossing count is #{m >= 0 : (N_b + 2^16 m) |D_e| < F_e |D_b|} (<= for
// b < e), at most 8 (2R + 1) - 1.  It is estimated from 32-bit values in FP32 (error far
// below one crossing) and corrected once, up or down, with exact 64-bit comparisons.
template <int KIND>
__device__ __forceinline__ bool skip_box(const DevMap& m, int k[3], const int s[3], uint32_t N[3],
                                         const uint32_t A[3], const float rA[3], const uint32_t L[3],
                                         int R, bool voxel_box, uint32_t& steps, uint32_t& n_last,
                                         uint32_t& a_last) {
  uint32_t c[3], F[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = k[a] >> 3;
    // voxels left in the box along the step direction: a box of blocks within R blocks of
    // the current block, or (voxel_box) the voxels within R of the current voxel
    int ca = voxel_box ? R : (s[a] > 0 ? 8 * (b + R) + 7 - k[a] : k[a] - 8 * (b - R));
    if (KIND == RMP_MAP_DENSE_U8) {
      const int g = s[a] > 0 ? m.dims[a] - 1 - k[a] : k[a];
      ca = ca < g ? ca : g;
    }
    c[a] = (uint32_t)ca;
    F[a] = N[a] + (c[a] << 16);
  }
  const int e = min_axis(F, A);
  const uint32_t Fe = sel3(F, e), Ae = sel3(A, e), Le = sel3(L, e);
  if (Fe > Le) {
    uint32_t bn = 0, ba = 1;
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (A[a] != 0 && N[a] <= L[a]) {
        uint32_t cnt = ((L[a] - N[a]) >> 16) + 1;
        cnt = cnt < c[a] ? cnt : c[a];
        if (cnt > 0) {
          const uint32_t nl = N[a] + ((cnt - 1) << 16);
          if (!any || (unsigned long long)nl * ba > (unsigned long long)bn * A[a]) {
            bn = nl;
            ba = A[a];
          }
          any = true;
          k[a] += s[a] * (int)cnt;
          N[a] += cnt << 16;
          steps += cnt;
        }
      }
    }
    if (any) {
      n_last = bn;
      a_last = ba;
    }
    return true;
  }
  const float rAe = sel3f(rA, e) * (1.0f / 65536.0f);   // RN(1 / |D_e|) / 2^16
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == e || A[b] == 0) continue;
    const bool le = b < e;
    // est = (F_e |D_b| - N_b |D_e|) / (|D_e| 2^16): the numerator formed exactly in 64 bits
    // (-1 <= est <= 8 (2R + 1) < 2^8 and |D_e| <= 2^24, so |num| < 2^48) and converted from
    // two exact 24-bit halves with one rounding; est then carries a relative error below
    // 2^-22, an absolute one below 2^-14, and the count is floor(est) + 1 unless est lies
    // within 2^-12 of an integer, where exact comparisons decide (an FP32 estimate of
    // t_e |D_b| - N_b from the absolute numerators needed a band of 1/64, and then most
    // warps took the exact path for some lane)
    const long long num = (long long)((unsigned long long)Fe * A[b]) -
                          (long long)((unsigned long long)N[b] * Ae);
    const float est = __fmaf_rn(__int2float_rn((int)(num >> 24)), 16777216.0f,
                                __int2float_rn((int)(num & 0xFFFFFF))) * rAe;
    const float fl = floorf(est);
    const float fr = est - fl;
    int cnt;
    if (est < -0.000244140625f) {
      cnt = 0;
    } else if (fr > 0.000244140625f && fr < 0.999755859375f) {
      cnt = (int)fl + 1;
    } else {
      const unsigned long long X = (unsigned long long)Fe * A[b];
      cnt = est < 0.0f ? 0 : (int)est + 1;
      cnt = cnt < (int)c[b] + 1 ? cnt : (int)c[b] + 1;
      if (cnt > 0) {
        const unsigned long long y = (unsigned long long)(N[b] + ((uint32_t)(cnt - 1) << 16)) * Ae;
        if (!(le ? y <= X : y < X)) {
          cnt -= 1;
        } else {
          const unsigned long long y1 = y + ((unsigned long long)Ae << 16);
          if (le ? y1 <= X : y1 < X) cnt += 1;
        }
      } else {
        const unsigned long long y0 = (unsigned long long)N[b] * Ae;
        if (le ? y0 <= X : y0 < X) cnt = 1;
      }
    }
    k[b] += s[b] * cnt;
    N[b] += (uint32_t)cnt << 16;
    steps += (uint32_t)cnt;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == e) {
      k[a] += s[a] * (int)(c[a] + 1);
      N[a] = Fe + 65536u;
    }
  }
  steps += sel3(c, e) + 1;
  n_last = Fe;
  a_last = Ae;
  return false;
}

// Pieces of a ray.  The parameter range (0, R], R = R_fx / 2^24 voxel units, is cut at
// the points T_j = j R / 2^kGridLog (j = 0 .. 2^kGridLog); a piece covers (T_lo, T_hi]
// between two of them.  A crossing numerator n of axis a (t = n / |D_a|) satisfies
// t <= T_j iff n 2^(24 + kGridLog) <= j R_fx |D_a|, so a piece's start state (every
// crossing with t <= T_lo applied) and its limits L_a (the crossings with t <= T_hi are
// those with N_a <= L_a) are integer functions of j.  Pieces of one ray can be marched by
// different threads at once; the ray's result is the first piece (in t) that hit or left
// the map, else the last piece.  With R_fx <= 2^30 and |D_a| <= 2^24 every product stays
// below 2^62.
constexpr int kGridLog = 7;
constexpr int kBudgetOut = 4;      // march_run: iteration budget spent, state resumable

struct MarchState {
  int k[3];
  uint32_t N[3];
  uint32_t steps;           // steps from the ray's start voxel
  uint32_t n_last, a_last;  // entry numerator / |D| of the current voxel (0/1 at the start)
  int ax_last;              // axis of the last step (for map exits)
};

// Per-ray fixed-point constants: step signs, |D_a| and the start voxel's boundary distances.
struct RayFx {
  int k0[3], s[3];
  uint32_t A[3], N0[3];
};

__device__ __forceinline__ void ray_fx(const long long P[3], const int D[3], RayFx& r) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.k0[a] = (int)(P[a] >> 16);
    r.s[a] = D[a] > 0 ? 1 : -1;
    r.A[a] = (uint32_t)abs(D[a]);
    const long long lo = (long long)r.k0[a] << 16;
    r.N0[a] = D[a] > 0 ? (uint32_t)(lo + 65536 - P[a]) : (D[a] < 0 ? (uint32_t)(P[a] - lo) : 1u);
  }
}

__device__ __forceinline__ void limits_at(const RayFx& r, long long R_fx, uint32_t j, uint32_t L[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    L[a] = (uint32_t)(((unsigned long long)j * (unsigned long long)R_fx * r.A[a]) >> (24 + kGridLog));
}

// State after every crossing with t <= T_j: per axis the count of boundaries
// N0_a + 2^16 m (m >= 0) within the bound; the entry of the current voxel is the latest of
// the axes' last crossings.
__device__ __forceinline__ void state_at(const RayFx& r, long long R_fx, uint32_t j, MarchState& st) {
  uint32_t bn = 0, ba = 1;
  bool any = false;
  st.steps = 0;
  st.ax_last = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    st.k[a] = r.k0[a];
    st.N[a] = r.N0[a];
    if (j > 0 && r.A[a] != 0) {
      const unsigned long long X = (unsigned long long)j * (unsigned long long)R_fx * r.A[a];
      const unsigned long long Y = (unsigned long long)r.N0[a] << (24 + kGridLog);
      if (X >= Y) {
        const uint32_t cnt = (uint32_t)((X - Y) >> (40 + kGridLog)) + 1;
        const uint32_t nl = r.N0[a] + ((cnt - 1) << 16);
        if (!any || (unsigned long long)nl * ba > (unsigned long long)bn * r.A[a]) {
          bn = nl;
          ba = r.A[a];
        }
        any = true;
        st.k[a] += r.s[a] * (int)cnt;
        st.N[a] += cnt << 16;
        st.steps += cnt;
      }
    }
  }
  st.n_last = any ? bn : 0;
  st.a_last = any ? ba : 1;
}

// Crossings of every axis still within the limits L from state st: per axis the count of
// boundaries N_a + 2^16 m (m >= 0) with N_a + 2^16 m <= L_a (none where |D_a| = 0: then
// N_a = 1 > L_a = 0).  The march takes crossings in time order and a crossing is within the
// limit exactly when its time is at most the piece's end, so the piece reaches its limit
// exactly when st.steps has grown by this count.
__device__ __forceinline__ uint32_t crossings_within(const uint32_t N[3], const uint32_t L[3]) {
  uint32_t c = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) c += N[a] <= L[a] ? ((L[a] - N[a]) >> 16) + 1u : 0u;
  return c;
}

// March a piece from state st until a hit, a map exit, the limits L (returns `at_limit`) or
// `budget` block visits (returns kBudgetOut; st is then a state from which march_run
// continues exactly).  Each visit of the outer loop either crosses a free box of blocks
// (skip_box) or enters an occupied block, whose brick is staged in the lane's column of
// shared memory (`sb`: word q at sb[32 q], so a warp's lanes never share a bank) while the
// inner loop steps voxel by voxel, the order of the next crossings kept in the exact
// differences E_ab = N_a |D_b| - N_b |D_a|.  Per step the inner loop keeps only what the
// next step needs: the voxel, its brick bit index p = lx + 8 ly + 64 lz (brick word p / 32,
// bit p % 32), the crossing numerators and the number of crossings left before the limit;
// the step count and the entry crossing of the current voxel are brought up to date when
// the walk leaves the block.  WALK_UNROLL: unroll factor of the voxel walk (its 24
// iterations fully unrolled measured 57.4 -> 55.1 us for 65536 rays on the hashed map;
// the batch kernel, held to 64 registers, spills then and uses a factor of 2: 1.297 ->
// 1.290 ms against the compiler's 4, 1.43 ms with 6).
template <int KIND, int LAYOUT, bool CELLS, int WALK_UNROLL>
__device__ __forceinline__ int march_run(const DevMap& m, const uint32_t* bm, MarchState& st,
                                         const RayFx& r, const uint32_t L[3], int at_limit,
                                         uint32_t budget, uint32_t* sb) {
  if (outside<KIND>(m, st.k)) return RMP_RAY_MISS_EXIT;
  const uint32_t* A = r.A;
  const int* s = r.s;
  int* k = st.k;
  uint32_t* N = st.N;
  const float rA[3] = {__frcp_rn(__uint2float_rn(A[0])), __frcp_rn(__uint2float_rn(A[1])),
                       __frcp_rn(__uint2float_rn(A[2]))};
  const uint32_t lim_steps = st.steps + crossings_within(N, L);
  // brick-index change of one step along each axis
  const int d0 = s[0], d1 = 8 * s[1], d2 = 64 * s[2];
  const uint32_t guard = 8u * (kMaxRangeVoxels + 2);
  const uint32_t iters = budget < guard ? budget : guard;
  int status = budget < guard ? kBudgetOut : at_limit;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint4* src = nullptr;
    uint32_t bidx = 0;
    const int v = block_radius<LAYOUT>(m, bm, k[0] >> 3, k[1] >> 3, k[2] >> 3, &src, &bidx);
    // a free block is left through the box of free blocks around it; in an occupied block,
    // a voxel whose 2^3 cell lies at Chebyshev distance dv >= 2 from every occupied voxel
    // (grid layout's cell distances) is left through the free box of half-width dv - 1
    // voxels around it -- both in one exact step
    int R = v - 1;
    bool vox = false;
    if (CELLS && v == 0 && LAYOUT == kLayoutGrid && m.cells) {
      const uint32_t ci = (uint32_t)(((k[0] & 7) >> 1) | (((k[1] & 7) >> 1) << 2) |
                                     (((k[2] & 7) >> 1) << 4));
      const int dv = (int)((__ldg(m.cells + 8 * (size_t)bidx + (ci >> 3)) >> (4 * (ci & 7))) & 15u);
      R = dv - 1;
      vox = true;
    }
    if (R >= (vox ? 1 : 0)) {
      if (skip_box<KIND>(m, k, s, N, A, rA, L, R, vox, st.steps, st.n_last, st.a_last)) {
        status = at_limit;
        break;
      }
      if (outside<KIND>(m, k)) {
        // only the exit axis can have left the grid
        st.ax_last = ((unsigned)k[0] >= (unsigned)m.dims[0]) ? 0
                     : (((unsigned)k[1] >= (unsigned)m.dims[1]) ? 1 : 2);
        status = RMP_RAY_MISS_EXIT;
        break;
      }
      continue;
    }
    store_smem_brick(src, sb);
    uint32_t p = (uint32_t)((k[0] & 7) | ((k[1] & 7) << 3) | ((k[2] & 7) << 6));
    if (smem_brick_bit(sb, p)) {
      status = RMP_RAY_HIT;
      break;
    }
    // exact order of the next crossings: E_xy > 0 <=> t_y < t_x, etc.
    long long exy = (long long)N[0] * A[1] - (long long)N[1] * A[0];
    long long exz = (long long)N[0] * A[2] - (long long)N[2] * A[0];
    long long eyz = (long long)N[1] * A[2] - (long long)N[2] * A[1];
    const long long u0 = (long long)A[0] << 16, u1 = (long long)A[1] << 16,
                    u2 = (long long)A[2] << 16;
    const uint32_t rem0 = lim_steps - st.steps;   // crossings left within the limit
    uint32_t rem = rem0;
    int axl = 0;                                  // axis of the walk's latest step
    int fin = 0;
    // at most 21 interior steps and one exit step inside an 8^3 block
#pragma unroll WALK_UNROLL
    for (int j = 0; j < 24; ++j) {
      if (rem == 0u) {                                 // next crossing beyond the limit
        fin = 1;
        break;
      }
      const bool ylx = exy > 0;
      const bool zlw = ylx ? (eyz > 0) : (exz > 0);
      const int ax = zlw ? 2 : (ylx ? 1 : 0);
      --rem;
      axl = ax;
      bool crossed = false;
      if (ax == 0) {
        const int kn = k[0] + s[0];
        crossed = ((kn ^ k[0]) & ~7) != 0;
        k[0] = kn;
        N[0] += 65536u;
        p += d0;
        exy += u1;
        exz += u2;
      } else if (ax == 1) {
        const int kn = k[1] + s[1];
        crossed = ((kn ^ k[1]) & ~7) != 0;
        k[1] = kn;
        N[1] += 65536u;
        p += d1;
        exy -= u0;
        eyz += u2;
      } else {
        const int kn = k[2] + s[2];
        crossed = ((kn ^ k[2]) & ~7) != 0;
        k[2] = kn;
        N[2] += 65536u;
        p += d2;
        exz -= u0;
        eyz -= u1;
      }
      if (outside<KIND>(m, k)) {
        fin = 2;
        break;
      }
      if (crossed) break;
      if (smem_brick_bit(sb, p)) {
        fin = 3;
        break;
      }
    }
    if (rem != rem0) {                                 // the walk took steps
      st.steps += rem0 - rem;
      st.ax_last = axl;
      st.n_last = sel3(N, axl) - 65536u;
      st.a_last = sel3(A, axl);
    }
    if (fin) {
      status = fin == 1 ? at_limit : (fin == 2 ? RMP_RAY_MISS_EXIT : RMP_RAY_HIT);
      break;
    }
  }
  return status;
}

__device__ __forceinline__ bool piece_final(int status) {
  return status == RMP_RAY_HIT || status == RMP_RAY_MISS_EXIT;
}

__device__ __forceinline__ void shfl_state(MarchState& d, const MarchState& st, int src) {
  d.k[0] = __shfl_sync(0xffffffffu, st.k[0], src);
  d.k[1] = __shfl_sync(0xffffffffu, st.k[1], src);
  d.k[2] = __shfl_sync(0xffffffffu, st.k[2], src);
  d.N[0] = __shfl_sync(0xffffffffu, st.N[0], src);
  d.N[1] = __shfl_sync(0xffffffffu, st.N[1], src);
  d.N[2] = __shfl_sync(0xffffffffu, st.N[2], src);
  d.steps = __shfl_sync(0xffffffffu, st.steps, src);
  d.n_last = __shfl_sync(0xffffffffu, st.n_last, src);
  d.a_last = __shfl_sync(0xffffffffu, st.a_last, src);
  d.ax_last = __shfl_sync(0xffffffffu, st.ax_last, src);
}

// Smallest j >= j_min with T_j >= t (t = n / a > 0 the current entry parameter):
// n 2^(24 + kGridLog) <= j R_fx a.  FP32 estimate, then exact 64-bit corrections.
__device__ __forceinline__ uint32_t grid_index_at_or_after(uint32_t n, uint32_t a, long long R_fx,
                                                           uint32_t j_min) {
  if (n == 0) return j_min;
  const unsigned long long num = (unsigned long long)n << (24 + kGridLog);
  const unsigned long long den = (unsigned long long)R_fx * a;
  float e = __fdiv_rn(__ull2float_rn(num), __ull2float_rn(den));
  uint32_t j = e < 0.0f ? 0u : (e > 129.0f ? 129u : (uint32_t)ceilf(e));
  if ((unsigned long long)j * den < num) ++j;
  if (j > 0 && (unsigned long long)(j - 1) * den >= num) --j;
  return j > j_min ? j : j_min;
}

// Pieces that spent the first phase's budget are split over the warp's lanes: with u such
// pieces each gets h = 32 / u lanes.  Piece p (the owner lane's remaining range (t, T_hi],
// t its current entry parameter) is cut at grid points into up to h sub-pieces; the first
// continues from the owner's state, the others start from state_at.  The sub-pieces' first
// final result (else the last one's) becomes the owner's.  Both steps are
// warp-synchronous: every lane calls them with the same `unfinished` mask.
struct SplitPlan {
  uint32_t h;       // lanes per unfinished piece
  uint32_t p;       // this lane's rank among the unfinished lanes (if it owns one)
  uint32_t hq;      // sub-pieces of this lane's own piece
  bool mine;        // this lane owns an unfinished piece
};

// Number of sub-pieces of a piece whose remaining grid range is j0 .. j_hi.
__device__ __forceinline__ uint32_t sub_pieces(uint32_t j0, uint32_t j_hi, uint32_t h) {
  const uint32_t c = j_hi > j0 ? j_hi - j0 : 0u;
  return c < h ? (c > 0 ? c : 1u) : h;
}

// Give this lane its sub-piece: on return (st, r, L, at_limit) describe it and the result
// says whether the lane has one.
__device__ __forceinline__ bool split_setup(long long R_fx, const long long P[3], int D[3],
                                            uint32_t j_lo, uint32_t j_hi, int& at_limit,
                                            uint32_t unfinished, MarchState& st, RayFx& r,
                                            uint32_t L[3], SplitPlan& plan) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nu = __popc(unfinished);
  const uint32_t h = 32u / nu;
  plan.h = h;
  plan.mine = (unfinished >> lane) & 1u;
  plan.p = __popc(unfinished & ((1u << lane) - 1u));
  plan.hq = plan.mine ? sub_pieces(grid_index_at_or_after(st.n_last, st.a_last, R_fx, j_lo), j_hi, h)
                      : 1u;
  // the piece this lane works on: group gi = lane / h, sub-piece q
  const uint32_t gi = lane / h, q = lane - gi * h;
  const bool in_grp = gi < nu;
  const int owner = in_grp ? (int)(__fns(unfinished, 0, (int)gi + 1)) : (int)lane;
  MarchState o;
  shfl_state(o, st, owner);
  D[0] = __shfl_sync(0xffffffffu, D[0], owner);
  D[1] = __shfl_sync(0xffffffffu, D[1], owner);
  D[2] = __shfl_sync(0xffffffffu, D[2], owner);
  const uint32_t jl = __shfl_sync(0xffffffffu, j_lo, owner);
  const uint32_t jh = __shfl_sync(0xffffffffu, j_hi, owner);
  const int lim = __shfl_sync(0xffffffffu, at_limit, owner);
  const uint32_t j0 = grid_index_at_or_after(o.n_last, o.a_last, R_fx, jl);
  const uint32_t hq = sub_pieces(j0, jh, h);
  if (!in_grp || q >= hq) return false;
  ray_fx(P, D, r);
  const uint32_t c = jh - j0;
  const uint32_t b1 = q + 1 == hq ? jh : j0 + (c * (q + 1)) / hq;
  if (q > 0) state_at(r, R_fx, j0 + (c * q) / hq, st);
  else st = o;
  limits_at(r, R_fx, b1, L);
  at_limit = q + 1 == hq ? lim : kSegContinues;
  return true;
}

// Move each split piece's result to its owner lane; the other lanes get back their own
// result (own, own_status) from before the split.
__device__ __forceinline__ void split_combine(const SplitPlan& plan, bool worked, MarchState& st,
                                              int& status, const MarchState& own, int own_status) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t fin = __ballot_sync(0xffffffffu, worked && piece_final(status));
  const uint32_t gmask = (plan.hq >= 32 ? 0xffffffffu : ((1u << plan.hq) - 1u)) << (plan.p * plan.h);
  const uint32_t fb = fin & gmask;
  const int src = !plan.mine ? (int)lane
                             : (fb ? __ffs(fb) - 1 : (int)(plan.p * plan.h + plan.hq - 1));
  MarchState res;
  shfl_state(res, st, src);
  const int rs = __shfl_sync(0xffffffffu, status, src);
  st = plan.mine ? res : own;
  status = plan.mine ? rs : own_status;
}

// Distinct 8^3 blocks whose occupancy the march tested: the voxel path is monotone on
// each axis and blocks are convex, so this is 1 + the block changes along each axis up to
// the last tested voxel (for a map exit the voxel before the exit step; none if the ray
// starts outside the map).
__device__ __forceinline__ uint32_t blocks_tested(const int k0[3], const MarchState& o, int status,
                                                 const int s[3]) {
  int kf[3] = {o.k[0], o.k[1], o.k[2]};
  if (status == RMP_RAY_MISS_EXIT) {
    if (o.steps == 0) return 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a == o.ax_last) kf[a] -= s[a];
  }
  return 1u + (uint32_t)(abs((kf[0] >> 3) - (k0[0] >> 3)) + abs((kf[1] >> 3) - (k0[1] >> 3)) +
                         abs((kf[2] >> 3) - (k0[2] >> 3)));
}

__device__ __forceinline__ float entry_distance(uint32_t n, uint32_t a, float vs_f) {
  const float t = __fdiv_rn(__uint2float_rn(n), __uint2float_rn(a));
  return __fmul_rn(__fmul_rn(t, 256.0f), vs_f);
}

// ------------------------------------------------------------------ obstacle policy (Sec. III-C)
// u: unit direction towards the obstacle (r = -u points away), d: distance; the velocity
// is carried as an unevaluated FP32 pair vh + vl (= xdot to ~2^-48 relative).  Writes
// f_i (3), A_i (6 unique) and A_i f_i (3).  `active` and `in_radius` are the FP32
// decisions specified in the header; the values are FP32 except that xdot.r is a
// compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005)
// because f_damp amplifies its rounding error by eta_damp / eps at small d, and w_r uses
// (r - d) formed exactly instead of 1 - d/r, which cancels near the radius.
__device__ __forceinline__ float dot2(const float vh[3], const float vl[3], const float r[3]) {
  float p = __fmul_rn(vh[0], r[0]);
  float e = __fmaf_rn(vh[0], r[0], -p);
#pragma unroll
  for (int a = 1; a < 3; ++a) {
    const float h = __fmul_rn(vh[a], r[a]);
    const float eh = __fmaf_rn(vh[a], r[a], -h);
    const float t = __fadd_rn(p, h);
    const float bp = __fsub_rn(t, p);
    const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(t, bp)), __fsub_rn(h, bp));
    p = t;
    e = __fadd_rn(e, __fadd_rn(eh, es));
  }
  const float lo = vl[0] * r[0] + vl[1] * r[1] + vl[2] * r[2];
  return __fadd_rn(p, __fadd_rn(e, lo));
}

__device__ __forceinline__ void obstacle_policy(const EvalConsts& k, const float u[3], float d,
                                                const float vh[3], const float vl[3],
                                                bool active, bool in_radius, float f[3],
                                                float A[6], float af[3]) {
  const float r[3] = {-u[0], -u[1], -u[2]};
  const float frep = k.eta_rep * expf(-d * k.inv_nu_rep);
  const float xr = dot2(vh, vl, r);
  const float mm = active ? xr * xr : 0.0f;
  const float kd = __fdividef(k.eta_damp, d * k.inv_nu_damp + k.eps);
  const float z = kd * mm;                       // |f_damp| (|r| = 1)
  const float fr = frep + z;                     // f = (f_rep + |f_damp|) r
  f[0] = fr * r[0];
  f[1] = fr * r[1];
  f[2] = fr * r[2];
  float w = 0.0f;
  if (in_radius) {
    const float y = (__fsub_rn(k.r_hi, d) + k.r_lo) * k.inv_r;   // 1 - d/r
    const float x = d * k.inv_r;
    w = k.w_mode == 0 ? y * y : y * y * (1.0f + 2.0f * x);      // (1-x)^2 ; 1-3x^2+2x^3
  }
  const float h = z + k.c * log1pf(expf(-2.0f * k.c * z));
  const float sc = __fdividef(z, h);            // s(f_damp) = sc * r
  const float alpha = w * sc * sc;               // A = alpha r r^T
  A[0] = alpha * r[0] * r[0];
  A[1] = alpha * r[0] * r[1];
  A[2] = alpha * r[0] * r[2];
  A[3] = alpha * r[1] * r[1];
  A[4] = alpha * r[1] * r[2];
  A[5] = alpha * r[2] * r[2];
  const float rf = r[0] * f[0] + r[1] * f[1] + r[2] * f[2];
  const float g = alpha * rf;                    // A f = alpha (r.f) r
  af[0] = g * r[0];
  af[1] = g * r[1];
  af[2] = g * r[2];
}

__device__ __forceinline__ bool active32(const float v[3], const float u[3]) {
  const float dot = __fmaf_rn(v[2], u[2], __fmaf_rn(v[1], u[1], __fmul_rn(v[0], u[0])));
  return dot > 0.0f;
}

// ------------------------------------------------------------------ reduction
// Compensated FP32 accumulator: (s, c) with s + c the running sum; additions use the
// error-free TwoSum so the tree keeps about twice FP32's precision.
struct Acc32 {
  float s[9], c[9];
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void acc_add(Acc32& acc, const float v[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    float s, e;
    two_sum(acc.s[q], v[q], s, e);
    acc.s[q] = s;
    acc.c[q] = __fadd_rn(acc.c[q], e);
  }
}

__device__ __forceinline__ void acc_merge(Acc32& acc, float s2, float c2, int q) {
  float s, e;
  two_sum(acc.s[q], s2, s, e);
  acc.s[q] = s;
  acc.c[q] = __fadd_rn(__fadd_rn(acc.c[q], c2), e);
}

struct Acc64 {
  double s[9];
};

// Sums of one CTA handed from the block reduction to grid_finish: the 9 terms (FP64 value
// v, and for the compensated reduction also the unevaluated FP32 pair s + c it came from)
// and the hit and active counts.  In shared memory, written by lanes 0-10 of warp 0 (lane
// q < 9: term q; lanes 9, 10: the counts), which are the lanes that read them again.
struct CtaSums {
  double v[9];
  float s[9], c[9];
  unsigned u[2];
};

__device__ __forceinline__ void merge1(float& s, float& c, float s2, float c2) {
  float t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), e);
}

// Block-level reduction of the per-thread accumulators and counts: a shuffle tree per warp,
// then lane q of warp 0 merges term q of the warps in warp order (all terms at once, not one
// thread walking them).  Called by every thread.
template <int RED>
struct BlockReduce;

template <>
struct BlockReduce<RMP_REDUCE_KAHAN32> {
  using Acc = Acc32;
  __device__ static void init(Acc& a) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a.s[q] = a.c[q] = 0.0f;
  }
  __device__ static void add(Acc& a, const float v[9]) { acc_add(a, v); }
  __device__ static void reduce(Acc& a, unsigned nh, unsigned na, CtaSums& out) {
    __shared__ float sh[32][18];
    __shared__ unsigned shu[32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const float s2 = __shfl_down_sync(0xffffffffu, a.s[q], off);
        const float c2 = __shfl_down_sync(0xffffffffu, a.c[q], off);
        acc_merge(a, s2, c2, q);
      }
    }
    nh = __reduce_add_sync(0xffffffffu, nh);
    na = __reduce_add_sync(0xffffffffu, na);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        sh[warp][q] = a.s[q];
        sh[warp][9 + q] = a.c[q];
      }
      shu[warp][0] = nh;
      shu[warp][1] = na;
    }
    __syncthreads();
    if (warp == 0) {
      if (lane < 9) {
        float s = sh[0][lane], c = sh[0][9 + lane];
        for (int w = 1; w < nw; ++w) merge1(s, c, sh[w][lane], sh[w][9 + lane]);
        out.s[lane] = s;
        out.c[lane] = c;
        out.v[lane] = (double)s + (double)c;
      } else if (lane < 11) {
        unsigned t = 0;
        for (int w = 0; w < nw; ++w) t += shu[w][lane - 9];
        out.u[lane - 9] = t;
      }
    }
  }
};

template <>
struct BlockReduce<RMP_REDUCE_FP64> {
  using Acc = Acc64;
  __device__ static void init(Acc& a) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a.s[q] = 0.0;
  }
  __device__ static void add(Acc& a, const float v[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a.s[q] += (double)v[q];
  }
  __device__ static void reduce(Acc& a, unsigned nh, unsigned na, CtaSums& out) {
    __shared__ double sh[32][9];
    __shared__ unsigned shu[32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < 9; ++q) a.s[q] += __shfl_down_sync(0xffffffffu, a.s[q], off);
    nh = __reduce_add_sync(0xffffffffu, nh);
    na = __reduce_add_sync(0xffffffffu, na);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) sh[warp][q] = a.s[q];
      shu[warp][0] = nh;
      shu[warp][1] = na;
    }
    __syncthreads();
    if (warp == 0) {
      if (lane < 9) {
        double s = sh[0][lane];
        for (int w = 1; w < nw; ++w) s += sh[w][lane];
        out.v[lane] = s;
      } else if (lane < 11) {
        unsigned t = 0;
        for (int w = 0; w < nw; ++w) t += shu[w][lane - 9];
        out.u[lane - 9] = t;
      }
    }
  }
};

// ------------------------------------------------------------------ FP64 resolve (Eq. 1)
// f = (sum A)^+ (sum A f) with eigenvalues <= 1e-12 lambda_max treated as zero.  FP64
// division and square root cost hundreds of cycles each on this GPU and every FP64
// instruction of a warp occupies the FP64 pipe for tens of cycles whatever the number of
// active lanes (measured: the resolve's stages take about 64 cycles per FP64 instruction),
// so the FP64 arithmetic is kept to what the result needs and the work is split:
//   eigenvectors by cyclic Jacobi rotations in FP32 (the matrix scaled by a power of two
//   and narrowed to FP32 by integer operations on its bit patterns), and, in another warp
//   (or another lane of the same warp), the FP64 adjugate solve adj(S) b / det(S);
//   lanes 0-2: each eigenvalue as the FP64 Rayleigh quotient v^T S v / v^T v of its FP32
//   eigenvector (second-order accurate, ~1e-14 lambda_max), with 1 / v^T v = 2 - v^T v to
//   first order (v^T v = 1 + O(1e-7)); the eigenvector components widened to FP64 by bit
//   packing (exact);
//   lane 0: the eigenvalues sorted and the rank decided by comparing order-preserving
//   integer keys of the FP64 values; full rank uses the adjugate solution, a deficient
//   rank projects b on the kept eigenvectors; writes f, eig, rank into r.

// S / 2^(E - 1023) narrowed to FP32 by truncation, E the largest biased exponent of the six
// entries (so the largest lies in [1, 2)); entries with a zero or subnormal exponent, or
// below 2^-126 of the largest, become 0.  Integer operations only.
__device__ __forceinline__ void narrow_scaled(const double* S, float a[6]) {
  int hi[6];
  unsigned lo[6];
  int emax = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    hi[q] = __double2hiint(S[q]);
    lo[q] = (unsigned)__double2loint(S[q]);
    emax = max(emax, (hi[q] >> 20) & 0x7FF);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int e = (hi[q] >> 20) & 0x7FF;
    const int fe = e - emax + 127;
    const unsigned mant = ((unsigned)(hi[q] & 0xFFFFF) << 3) | (lo[q] >> 29);
    const unsigned bits = ((unsigned)hi[q] & 0x80000000u) | ((unsigned)fe << 23) | mant;
    a[q] = (e != 0 && fe > 0) ? __uint_as_float(bits) : 0.0f;
  }
}

// An FP32 value widened to FP64 exactly by packing its bits (zero and subnormal inputs give
// zero; the eigenvector components this serves are normal or zero).
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return e == 0 ? 0.0 : __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// Integer key with the order of the (non-NaN) double x.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}

// Eigenvectors (columns of W) of the symmetric S by FP32 Jacobi sweeps.  One thread.
__device__ __forceinline__ void jacobi_f32(const double* S, float W[3][3]) {
  float sa[6];
  narrow_scaled(S, sa);
  float a00 = sa[0], a01 = sa[1], a02 = sa[2], a11 = sa[3], a12 = sa[4], a22 = sa[5];
  for (int sweep = 0; sweep < 6; ++sweep) {
    const float off = fabsf(a01) + fabsf(a02) + fabsf(a12);
    const float dia = fabsf(a00) + fabsf(a11) + fabsf(a22);
    if (!(off > 1e-6f * dia)) break;              // FP32 accuracy; FP64 refines below
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      float app, aqq, apq, apo, aqo;
      if (pq == 0) { app = a00; aqq = a11; apq = a01; apo = a02; aqo = a12; }
      else if (pq == 1) { app = a00; aqq = a22; apq = a02; apo = a01; aqo = a12; }
      else { app = a11; aqq = a22; apq = a12; apo = a01; aqo = a02; }
      if (apq == 0.0f) continue;
      const float tau = __fdividef(aqq - app, 2.0f * apq);
      const float at = fabsf(tau);
      const float root = at < 1e18f ? (1.0f + at * at) * rsqrtf(1.0f + at * at) : at;
      const float tt = copysignf(__fdividef(1.0f, at + root), tau);
      const float c = rsqrtf(1.0f + tt * tt), sn = tt * c;
      const float npp = app - tt * apq, nqq = aqq + tt * apq;
      const float npo = c * apo - sn * aqo, nqo = sn * apo + c * aqo;
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      if (pq == 0) { a00 = npp; a11 = nqq; a01 = 0.f; a02 = npo; a12 = nqo; }
      else if (pq == 1) { a00 = npp; a22 = nqq; a02 = 0.f; a01 = npo; a12 = nqo; }
      else { a11 = npp; a22 = nqq; a12 = 0.f; a01 = npo; a02 = nqo; }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float vp = W[i][p], vq = W[i][q];
        W[i][p] = c * vp - sn * vq;
        W[i][q] = sn * vp + c * vq;
      }
    }
  }
}

// 1 / x in FP64 for a positive x, by Newton's iteration for the reciprocal, r <- r + r (1 - m r),
// on the mantissa m in [1, 2): two steps from the FP32 reciprocal of m truncated to FP32
// (relative error 2^-22.4 -> 2^-44.8 -> below the FP64 rounding of the steps, about one ulp),
// the exponent applied by integer operations.  Four FP64 instructions instead of a division's
// sequence; subnormal, infinite or NaN x, and results outside the normal range, take the
// division.
__device__ __forceinline__ double recip_pos(double x) {
  const long long bx = __double_as_longlong(x);
  const int ex = (int)((bx >> 52) & 0x7FF);
  const double m = __longlong_as_double((bx & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  const float mf = __uint_as_float(0x3F800000u | (unsigned)((bx >> 29) & 0x7FFFFF));
  double r = widen(__frcp_rn(mf));                        // in [0.5, 1]
  double e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  const long long br = __double_as_longlong(r);
  const int er = (int)((br >> 52) & 0x7FF) - (ex - 1023);
  if (ex == 0 || ex == 2047 || er <= 0 || er >= 2047) return 1.0 / x;
  return __longlong_as_double((br & 0x000FFFFFFFFFFFFFll) | ((long long)er << 52));
}

// FP64 solve adj(S) b / det(S); ok = det > 0.  One thread.
__device__ __forceinline__ void adjugate_solve(const double* S, const double* b, double& fa0,
                                               double& fa1, double& fa2, int& ok) {
  const double c00 = S[3] * S[5] - S[4] * S[4], c01 = S[2] * S[4] - S[1] * S[5],
               c02 = S[1] * S[4] - S[2] * S[3], c11 = S[0] * S[5] - S[2] * S[2],
               c12 = S[1] * S[2] - S[0] * S[4], c22 = S[0] * S[3] - S[1] * S[1];
  const double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  ok = det > 0.0;
  if (det > 0.0) {
    const double inv = recip_pos(det);
    fa0 = (c00 * b[0] + c01 * b[1] + c02 * b[2]) * inv;
    fa1 = (c01 * b[0] + c11 * b[1] + c12 * b[2]) * inv;
    fa2 = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
  }
}

// Sorted eigenpairs and rank from the FP32 eigenvectors W (valid in lane 0): lanes 0-2 take
// the FP64 Rayleigh quotients; lane 0 sorts, decides the rank, writes eig and rank into r and
// keeps in es what a rank-deficient projection needs.  Called by all 32 lanes of one warp;
// only lane 0's r and es are set.
struct EigenSet {
  float c[3][3];   // eigenvector i (ascending eigenvalues) in c[i]
  float dv[3];     // its v^T v - 1
  bool keep[3];    // eigenvalue above the rank threshold
};

// v^T v - 1 for an FP32 vector with v^T v = 1 + O(1e-7), in FP32 error-free arithmetic:
// the squares split exactly into product and FMA error, the three products summed by TwoSum,
// the sum minus 1 exact (Sterbenz), the small terms added last (error ~1e-15).
__device__ __forceinline__ float norm2_minus_one(float v0, float v1, float v2) {
  const float p0 = __fmul_rn(v0, v0), p1 = __fmul_rn(v1, v1), p2 = __fmul_rn(v2, v2);
  const float e0 = __fmaf_rn(v0, v0, -p0), e1 = __fmaf_rn(v1, v1, -p1), e2 = __fmaf_rn(v2, v2, -p2);
  float s1, r1, s2, r2;
  two_sum(p0, p1, s1, r1);
  two_sum(s1, p2, s2, r2);
  return __fadd_rn(__fsub_rn(s2, 1.0f), __fadd_rn(__fadd_rn(r1, r2), __fadd_rn(__fadd_rn(e0, e1), e2)));
}

__device__ __forceinline__ void resolve_eigen(const double* S, const float (&W)[3][3],
                                              rmp_result_t& r, EigenSet& es) {
  const int t = threadIdx.x & 31;
  float V[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = __shfl_sync(0xffffffffu, W[i][j], 0);
  // lanes 0-8: lane 3 i + c takes component c of eigenvector i (column i of V): its term
  // v_c (S v)_c in FP64; lane 3 i adds the three terms and applies 1 / v^T v = 1 - (v^T v - 1)
  // to first order.  Seven FP64 instructions per warp (every FP64 instruction holds the
  // pipe about 64 cycles whatever the active lanes).
  const int iv = t < 9 ? t / 3 : 0, c = t < 9 ? t - 3 * iv : 0;
  const float w0 = iv == 0 ? V[0][0] : (iv == 1 ? V[0][1] : V[0][2]);
  const float w1 = iv == 0 ? V[1][0] : (iv == 1 ? V[1][1] : V[1][2]);
  const float w2 = iv == 0 ? V[2][0] : (iv == 1 ? V[2][1] : V[2][2]);
  double term = 0.0;
  if (t < 9) {
    const double sc0 = c == 0 ? S[0] : (c == 1 ? S[1] : S[2]);
    const double sc1 = c == 0 ? S[1] : (c == 1 ? S[3] : S[4]);
    const double sc2 = c == 0 ? S[2] : (c == 1 ? S[4] : S[5]);
    const double u = sc0 * widen(w0) + sc1 * widen(w1) + sc2 * widen(w2);
    term = widen(c == 0 ? w0 : (c == 1 ? w1 : w2)) * u;
  }
  const double t1 = __shfl_down_sync(0xffffffffu, term, 1);
  const double t2 = __shfl_down_sync(0xffffffffu, term, 2);
  const float dv_t = norm2_minus_one(w0, w1, w2);
  double lam_t = (term + t1) + t2;
  lam_t = fma(-lam_t, widen(dv_t), lam_t);
  double lam[3];
  float dv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lam[i] = __shfl_sync(0xffffffffu, lam_t, 3 * i);
    dv[i] = __shfl_sync(0xffffffffu, dv_t, 3 * i);
  }
  if (t != 0) return;
  // ascending eigenpairs by a 3-element sorting network on the values' integer keys
  double e0 = lam[0], e1 = lam[1], e2 = lam[2];
  float d0 = dv[0], d1 = dv[1], d2 = dv[2];
  long long q0 = order_key(e0), q1 = order_key(e1), q2 = order_key(e2);
  float c0[3] = {V[0][0], V[1][0], V[2][0]}, c1[3] = {V[0][1], V[1][1], V[2][1]},
        c2[3] = {V[0][2], V[1][2], V[2][2]};
  auto swap01 = [&]() {
    const double te = e0;
    const float td = d0;
    const long long tq = q0;
    e0 = e1; d0 = d1; q0 = q1; e1 = te; d1 = td; q1 = tq;
#pragma unroll
    for (int i = 0; i < 3; ++i) { const float tc = c0[i]; c0[i] = c1[i]; c1[i] = tc; }
  };
  if (q1 < q0) swap01();
  if (q2 < q1) {
    const double te = e1;
    const float td = d1;
    const long long tq = q1;
    e1 = e2; d1 = d2; q1 = q2; e2 = te; d2 = td; q2 = tq;
#pragma unroll
    for (int i = 0; i < 3; ++i) { const float tc = c1[i]; c1[i] = c2[i]; c2[i] = tc; }
  }
  if (q1 < q0) swap01();
  // kept: lambda_max > 1e-300 and lambda > 1e-12 lambda_max
  const long long thr = order_key(1e-12 * e2);
  const bool live = q2 > order_key(1e-300);
  es.keep[0] = live && q0 > thr;
  es.keep[1] = live && q1 > thr;
  es.keep[2] = live && q2 > thr;
  r.eig[0] = e0;
  r.eig[1] = e1;
  r.eig[2] = e2;
  r.rank = (es.keep[0] ? 1u : 0u) + (es.keep[1] ? 1u : 0u) + (es.keep[2] ? 1u : 0u);
  es.dv[0] = d0;
  es.dv[1] = d1;
  es.dv[2] = d2;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    es.c[0][i] = c0[i];
    es.c[1][i] = c1[i];
    es.c[2][i] = c2[i];
  }
}

// f into r from the rank (resolve_eigen) and the adjugate solution: full rank takes the
// adjugate, a deficient rank projects b on the kept eigenvectors.  Lane 0 of the warp that
// ran resolve_eigen.
__device__ __forceinline__ void resolve_f(const double* b, const EigenSet& es, double fa0,
                                          double fa1, double fa2, int ok, rmp_result_t& r) {
  r.f[0] = r.f[1] = r.f[2] = 0.0;
  if (r.rank == 3 && ok) {
    r.f[0] = fa0;
    r.f[1] = fa1;
    r.f[2] = fa2;
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!es.keep[i]) continue;
    const float* c = es.c[i];
    const double proj = (c[0] * b[0] + c[1] * b[1] + c[2] * b[2]) / (r.eig[i] * (1.0 + widen(es.dv[i])));
    r.f[0] += proj * c[0];
    r.f[1] += proj * c[1];
    r.f[2] += proj * c[2];
  }
}

// One warp: lane 0 runs the Jacobi sweeps, lane 1 the adjugate solve (the two branches
// of one warp run one after the other).  Called by all 32 lanes of one warp.
__device__ void resolve_pinv(const double* S, const double* b, rmp_result_t& r) {
  const int t = threadIdx.x & 31;
  float W[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  double fa0 = 0.0, fa1 = 0.0, fa2 = 0.0;
  int ok = 0;
  if (t == 0) jacobi_f32(S, W);
  else if (t == 1) adjugate_solve(S, b, fa0, fa1, fa2, ok);
  fa0 = __shfl_sync(0xffffffffu, fa0, 1);
  fa1 = __shfl_sync(0xffffffffu, fa1, 1);
  fa2 = __shfl_sync(0xffffffffu, fa2, 1);
  ok = __shfl_sync(0xffffffffu, ok, 1);
  EigenSet es;
  resolve_eigen(S, W, r, es);
  if (t == 0) resolve_f(b, es, fa0, fa1, fa2, ok, r);
}

// Two warps of a CTA (threads 0-63): warp 0 runs the Jacobi sweeps and the Rayleigh
// quotients while warp 1 runs the adjugate solve; they meet at named barrier 1 only for
// the choice of f.  Called by threads 0-63 of a CTA of at least 64 threads; S, b and r in
// shared memory.
__device__ void resolve_pinv_cta(const double* S, const double* b, rmp_result_t& r) {
  __shared__ double fa_sh[3];
  __shared__ int ok_sh;
  const int t = threadIdx.x;
  if (t >= 32) {
    if (t == 32) {
      double fa0 = 0.0, fa1 = 0.0, fa2 = 0.0;
      int ok = 0;
      adjugate_solve(S, b, fa0, fa1, fa2, ok);
      fa_sh[0] = fa0;
      fa_sh[1] = fa1;
      fa_sh[2] = fa2;
      ok_sh = ok;
    }
    __syncwarp();
    asm volatile("bar.sync 1, 64;" ::: "memory");
    return;
  }
  float W[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  if (t == 0) jacobi_f32(S, W);
  EigenSet es;
  resolve_eigen(S, W, r, es);
  __syncwarp();
  asm volatile("bar.sync 1, 64;" ::: "memory");
  if (t == 0) resolve_f(b, es, fa_sh[0], fa_sh[1], fa_sh[2], ok_sh, r);
}

// A partial in the workspace (80 bytes, one per CTA): the compensated reduction stores each
// term as its FP32 pair (s, c), the FP64 reduction as a double (CtaPartial); both end with
// the hit and active counts.  Bit 31 of the hit count flags a CTA whose map staging timed
// out (counts stay below 2^25).  An empty slot holds 0xFF in every byte, a pattern no
// stored field takes: FP32 and FP64 arithmetic on this GPU returns its canonical NaNs
// (sign bit clear), never the all-ones word, and the counts stay far below 2^31.
struct CtaPartial32 {
  float s[9], c[9];
  unsigned n_hits, n_active;
};
static_assert(sizeof(CtaPartial32) == sizeof(CtaPartial) && sizeof(CtaPartial) == 80,
              "partials are five 16-byte words");
constexpr uint32_t kSlotTimeoutFlag = 0x80000000u;
constexpr uint64_t kFinishWaitNs = 10000000000ull;   // CTA 0 waits at most 10 s for a slot

// Slots are written with relaxed stores at GPU scope (each field one single-copy-atomic
// access) and read back with relaxed 64-bit loads, so a reader sees every field either
// empty or complete.
__device__ __forceinline__ void st_relaxed32(void* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed64(void* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void load_slot(const CtaPartial* p, uint32_t w[20]) {
  const unsigned long long* q = reinterpret_cast<const unsigned long long*>(p);
  unsigned long long v[10];
#pragma unroll
  for (int i = 0; i < 5; ++i)
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];"
                 : "=l"(v[2 * i]), "=l"(v[2 * i + 1])
                 : "l"(q + 2 * i)
                 : "memory");
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    w[2 * i] = (uint32_t)v[i];
    w[2 * i + 1] = (uint32_t)(v[i] >> 32);
  }
}
__device__ __forceinline__ void empty_slot(CtaPartial* p) {
  uint4* q = reinterpret_cast<uint4*>(p);
  const uint4 e = make_uint4(~0u, ~0u, ~0u, ~0u);
#pragma unroll
  for (int i = 0; i < 5; ++i) q[i] = e;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Storing a CTA's sums in its slot, lanes 0-10 of warp 0 one field each; the words of a
// CTA's own sums as its slot would hold them; whether a slot's words are all written; and
// starting a thread's accumulator from the words of a partial / merging one into it.
template <int RED>
struct PartialIO;

template <>
struct PartialIO<RMP_REDUCE_KAHAN32> {
  __device__ static void store(CtaPartial* slot, const CtaSums& cs, int t, uint32_t flag) {
    CtaPartial32* p = reinterpret_cast<CtaPartial32*>(slot);
    if (t < 9) {
      st_relaxed32(&p->s[t], __float_as_uint(cs.s[t]));
      st_relaxed32(&p->c[t], __float_as_uint(cs.c[t]));
    } else if (t == 9) {
      st_relaxed32(&p->n_hits, cs.u[0] | flag);
    } else if (t == 10) {
      st_relaxed32(&p->n_active, cs.u[1]);
    }
  }
  __device__ static void words(const CtaSums& cs, uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      w[q] = __float_as_uint(cs.s[q]);
      w[9 + q] = __float_as_uint(cs.c[q]);
    }
    w[18] = cs.u[0];
    w[19] = cs.u[1];
  }
  __device__ static bool ready(const uint32_t w[20]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 20; ++i) ok = ok && w[i] != ~0u;
    return ok;
  }
  __device__ static void set(Acc32& a, const uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      a.s[q] = __uint_as_float(w[q]);
      a.c[q] = __uint_as_float(w[9 + q]);
    }
  }
  __device__ static void merge(Acc32& a, const uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) merge1(a.s[q], a.c[q], __uint_as_float(w[q]), __uint_as_float(w[9 + q]));
  }
};

template <>
struct PartialIO<RMP_REDUCE_FP64> {
  __device__ static void store(CtaPartial* slot, const CtaSums& cs, int t, uint32_t flag) {
    if (t < 9) st_relaxed64(&slot->v[t], (unsigned long long)__double_as_longlong(cs.v[t]));
    else if (t == 9) st_relaxed32(&slot->n_hits, cs.u[0] | flag);
    else if (t == 10) st_relaxed32(&slot->n_active, cs.u[1]);
  }
  __device__ static void words(const CtaSums& cs, uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(cs.v[q]);
      w[2 * q] = (uint32_t)b;
      w[2 * q + 1] = (uint32_t)(b >> 32);
    }
    w[18] = cs.u[0];
    w[19] = cs.u[1];
  }
  __device__ static bool ready(const uint32_t w[20]) {
    bool ok = w[18] != ~0u && w[19] != ~0u;
#pragma unroll
    for (int q = 0; q < 9; ++q) ok = ok && (w[2 * q] & w[2 * q + 1]) != ~0u;
    return ok;
  }
  __device__ static double word_pair(const uint32_t w[20], int q) {
    return __hiloint2double((int)w[2 * q + 1], (int)w[2 * q]);
  }
  __device__ static void set(Acc64& a, const uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a.s[q] = word_pair(w, q);
  }
  __device__ static void merge(Acc64& a, const uint32_t w[20]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a.s[q] += word_pair(w, q);
  }
};

// CTA 0's wait, one warp at a time: every lane with a pending slot (`ok` false) loads it
// until all of its fields are written (then its words are in w).  The warp polls as a
// whole -- it leaves the loop when every lane is done, lanes never spin on their own --
// because lanes that finished while others of their warp still spin stall for microseconds
// (measured).  Returns false when the wait passed `deadline` (global timer, ns).  Called by
// all lanes of the warp.
template <int RED>
__device__ __forceinline__ bool wait_slots(const CtaPartial* p, bool ok, uint32_t w[20],
                                           unsigned long long deadline) {
  while (!__all_sync(0xffffffffu, ok)) {
    if (!ok) {
      load_slot(p, w);
      ok = PartialIO<RED>::ready(w);
    }
    if (__any_sync(0xffffffffu, global_ns() > deadline)) return false;
  }
  return true;
}

// Grid completion, deterministic, with the partial sums streamed to CTA 0: lanes 0-10 of
// warp 0 of every other CTA store its sums in its slot and the CTA exits (no atomics, no
// fence); CTA 0, once its own rays are done, takes the slots as they fill -- thread t slot
// t, then t + blockDim, ... in order, merging each into its accumulator and emptying the
// slot -- then reduces the threads (BlockReduce) and resolves.  The summation order is
// fixed by slot index, whatever the order of arrival, and the partials of CTAs that
// finished early are read while the slowest still march: after the last partial only its
// load, the block reduction and the resolve remain.  CTA 0 never waits on a CTA that
// waits on it, so the wait ends once every CTA has run; it is bounded all the same
// (kFinishWaitNs), and a wait that expires reports RMP_ERR_TIMEOUT and marks the workspace
// poisoned (every later evaluation on it reports RMP_ERR_TIMEOUT until it is
// re-initialised).  A grid of one CTA resolves its own sums.  Called by all threads of
// every CTA after BlockReduce::reduce.
template <int RED>
__device__ void grid_finish(const CtaSums& cta, WsHeader* ws, CtaPartial* parts,
                            rmp_result_t* out, uint32_t n_rays, int status) {
  __shared__ CtaSums gsum;
  __shared__ int poison_sh;
  const int G = gridDim.x;
  const CtaSums* tot = &cta;
  int st = status;
  if (G > 1) {
    if (blockIdx.x != 0) {
      if (threadIdx.x < 32)
        PartialIO<RED>::store(parts + blockIdx.x, cta, threadIdx.x,
                              status == RMP_ERR_TIMEOUT ? kSlotTimeoutFlag : 0u);
      return;
    }
    if (threadIdx.x == 0) poison_sh = ws->poisoned ? 1 : 0;
    __syncthreads();
    const bool poisoned = poison_sh != 0;
    typename BlockReduce<RED>::Acc acc;
    BlockReduce<RED>::init(acc);
    unsigned nh = 0, na = 0, flags = 0;
    bool expired = false;
    const unsigned long long deadline = global_ns() + kFinishWaitNs;
    // warp-uniform trip count: lane l of the warp takes slot base + l
    for (int base = threadIdx.x & ~31; base < G && !poisoned; base += blockDim.x) {
      const int i = base + (int)(threadIdx.x & 31);
      uint32_t w[20];
      if (i == 0) PartialIO<RED>::words(cta, w);
      if (!wait_slots<RED>(parts + i, i == 0 || i >= G, w, deadline)) {
        expired = true;
        break;
      }
      if (i >= G) continue;
      if (i > 0) empty_slot(parts + i);
      if (i == (int)threadIdx.x) PartialIO<RED>::set(acc, w);
      else PartialIO<RED>::merge(acc, w);
      flags |= w[18] & kSlotTimeoutFlag;
      nh += w[18] & ~kSlotTimeoutFlag;
      na += w[19];
    }
    BlockReduce<RED>::reduce(acc, nh, na, gsum);
    const int any_expired = __syncthreads_or(expired);
    const int any_flag = __syncthreads_or(flags != 0);
    if (poisoned || any_expired) {
      if (threadIdx.x == 0) ws->poisoned = 1;
      st = RMP_ERR_TIMEOUT;
    } else if (any_flag) {
      st = RMP_ERR_TIMEOUT;
    }
    tot = &gsum;
  }
  __shared__ rmp_result_t r;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) r.A[q] = tot->v[q];
    for (int q = 0; q < 3; ++q) r.Af[q] = tot->v[6 + q];
    r.n_rays = n_rays;
    r.n_hits = tot->u[0];
    r.n_active = tot->u[1];
    r.status = st;
    r.reserved = 0;
  }
  __syncthreads();
  if (threadIdx.x < 64) resolve_pinv_cta(r.A, r.Af, r);
  if (threadIdx.x == 0) *out = r;
}

// Per-CTA state: quantised position (FP64, threads 0-2 one axis each) and the velocity
// as an FP32 pair (threads 3-5).
struct CtaState {
  long long P[3];
  float v[3];     // RN32(xdot)
  float vl[3];    // RN32(xdot - v)
  float xf[3];
  int bad[3];
};

// Component i of (x, xdot): from device memory, or, with a null pointer, from the copy the
// launch carries in its constants (selected with constant offsets, no local-memory array).
__device__ __forceinline__ double state_at(const double* state, const EvalConsts& k, int i) {
  if (state) return state[i];
  double v = k.x0[0];
#pragma unroll
  for (int j = 1; j < 6; ++j) v = i == j ? k.x0[j] : v;
  return v;
}

// Which state component (0-2 x, 3-5 xdot) thread t sets up, or -1: x on threads 0-2 and
// xdot on threads 32-34, two warps, so that the FP64 work of each runs in parallel.
__device__ __forceinline__ int state_component(unsigned t) {
  return t < 3 ? (int)t : ((t >= 32 && t < 35) ? (int)t - 29 : -1);
}

__device__ __forceinline__ void split_velocity(double x, CtaState& cs, int a) {
  cs.v[a] = __double2float_rn(x);
  cs.vl[a] = __double2float_rn(__dsub_rn(x, (double)cs.v[a]));
}

// Coherent ray order: thread slot j -> ray index.  Ray indices i with the same residue
// i mod M (M = 2^a 3^b) share the first a binary digits of H(i,2) and the first b ternary
// digits of H(i,3), so they point into one cell of the sphere; slots enumerate residue
// classes one after the other, so a warp covers at most two cells.  Q = n / M, R = n % M:
// classes r < R hold Q + 1 rays, the others Q.  M = 1 is the identity.
__device__ __forceinline__ uint32_t ray_of_slot(uint32_t j, const EvalConsts& k) {
  const uint32_t big = k.perm_R * (k.perm_Q + 1);
  uint32_t r, q;
  if (j < big) {
    r = j / (k.perm_Q + 1);
    q = j - r * (k.perm_Q + 1);
  } else {
    const uint32_t jj = j - big;
    const uint32_t t = jj / k.perm_Q;
    r = k.perm_R + t;
    q = jj - t * k.perm_Q;
  }
  return r + k.perm_M * q;
}

// ------------------------------------------------------------------ shared-memory staging
// The free-radius field is copied into shared memory by one TMA bulk copy (cp.async.bulk,
// completion counted on an mbarrier) issued at kernel entry, so it overlaps the state
// set-up and ray generation.  The wait is bounded: on expiry the CTA reports a timeout
// (after waiting, again bounded, for the copy to land) instead of hanging.
constexpr uint32_t kWaitSpins = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bulk_load_begin(uint64_t* bar, void* dst, const void* src,
                                                uint32_t bytes) {
  const uint32_t b = smem_u32(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}

// true once phase 0 of the barrier completed; false if the bounded wait expired
__device__ __forceinline__ bool bulk_load_wait(uint64_t* bar) {
  const uint32_t b = smem_u32(bar);
  for (uint32_t i = 0; i < kWaitSpins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ------------------------------------------------------------------ per-ray march and outputs
// One thread's segment `seg` (of S = 2^lg_segs) of the ray `ray` from position P: march the
// piece (phase 0: split_budget block visits; pieces still running are then split over the
// warp and finished, phase 1), then combine the ray's S segments -- adjacent lanes -- into
// the first final one (lowest index), else the last one.  Warp-synchronous: every lane of
// the warp calls it (work = false for lanes without a segment).  Returns the ray's status;
// mo is its final state (valid in every lane of the ray's segment group).  sb: the lane's
// shared-memory brick column.  NOSPLIT: no phase 1 (the split budget is ignored);
// WALK_UNROLL: see march_run.
template <int KIND, int LAYOUT, bool CELLS, bool NOSPLIT = false, int WALK_UNROLL = 24>
__device__ __forceinline__ int march_ray(const DevMap& m, const uint32_t* bm, const EvalConsts& k,
                                         const long long P[3], const Ray& ray, uint32_t seg,
                                         uint32_t lgS, bool work, MarchState& mo, uint32_t* sb) {
  const uint32_t S = 1u << lgS;
  const uint32_t lane = threadIdx.x & 31;
  // this lane's piece: segment seg of the ray, grid points j_lo .. j_hi
  const uint32_t j_lo = seg << (kGridLog - lgS), j_hi = (seg + 1) << (kGridLog - lgS);
  const int at_limit = seg == S - 1 ? RMP_RAY_MISS_RANGE : kSegContinues;
  MarchState so;
  int sstat = kSegContinues;
  RayFx r;
  uint32_t L[3];
  int lim = at_limit;
  int D[3] = {ray.D[0], ray.D[1], ray.D[2]};
  ray_fx(P, D, r);
  state_at(r, k.R_fx, j_lo, so);
  limits_at(r, k.R_fx, j_hi, L);
  const bool work0 = work;
  SplitPlan plan;
  bool split = false;
  MarchState own;
  int own_stat = kSegContinues;
  for (int phase = 0; phase < (NOSPLIT ? 1 : 2); ++phase) {
    if (work)
      sstat = march_run<KIND, LAYOUT, CELLS, WALK_UNROLL>(m, bm, so, r, L, lim,
                                                 (phase == 0 && !NOSPLIT) ? k.split_budget : 0xffffffffu, sb);
    if (NOSPLIT) break;
    if (phase == 1) break;
    const uint32_t unfinished = __ballot_sync(0xffffffffu, work && sstat == kBudgetOut);
    if (!unfinished) break;
    split = true;
    own = so;
    own_stat = sstat;
    work = split_setup(k.R_fx, P, D, j_lo, j_hi, lim, unfinished, so, r, L, plan);
    if (!work) sstat = kSegContinues;
  }
  if (split) split_combine(plan, work, so, sstat, own, own_stat);
  const bool fin = work0 && piece_final(sstat);
  const uint32_t ballot = __ballot_sync(0xffffffffu, fin);
  const uint32_t grp0 = lane & ~(S - 1);
  const uint32_t gmask = (S == 32 ? 0xffffffffu : ((1u << S) - 1u)) << grp0;
  const uint32_t fb = ballot & gmask;
  const int src = fb ? (__ffs(fb) - 1) : (int)(grp0 + S - 1);
  shfl_state(mo, so, src);
  return __shfl_sync(0xffffffffu, sstat, src);
}

// The ray's obstacle policy (Sec. III-C) from its final state: vals = A_i (6) and A_i f_i
// (3), all zero unless it hit; counts hits and active rays; writes the optional hit record
// and per-ray (f_i, A_i).
__device__ __forceinline__ void ray_outputs(const DevMap& m, const EvalConsts& k,
                                            const long long P[3], const Ray& ray,
                                            const MarchState& mo, int mstat, const float v[3],
                                            const float vl[3], rmp_ray_hit_t* hit, float* per,
                                            float vals[9], unsigned& n_hit, unsigned& n_act) {
  const float d = mo.n_last == 0 ? 0.0f : entry_distance(mo.n_last, mo.a_last, m.vs_f);
  float f[3] = {0.f, 0.f, 0.f}, A[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, af[3] = {0.f, 0.f, 0.f};
  if (mstat == RMP_RAY_HIT) {
    const bool act = active32(v, ray.dir);
    const bool inr = d < k.r_up;
    n_hit += 1;
    n_act += (act && inr) ? 1u : 0u;
    obstacle_policy(k, ray.dir, d, v, vl, act, inr, f, A, af);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) vals[q] = A[q];
  vals[6] = af[0];
  vals[7] = af[1];
  vals[8] = af[2];
  if (hit) {
    const int k0[3] = {(int)(P[0] >> 16), (int)(P[1] >> 16), (int)(P[2] >> 16)};
    const int sg[3] = {ray.D[0] > 0 ? 1 : -1, ray.D[1] > 0 ? 1 : -1, ray.D[2] > 0 ? 1 : -1};
    rmp_ray_hit_t h;
    h.voxel[0] = mo.k[0];
    h.voxel[1] = mo.k[1];
    h.voxel[2] = mo.k[2];
    h.steps = mo.steps;
    h.d = d;
    h.status = (uint8_t)mstat;
    h.pad = 0;
    h.blocks = (uint16_t)blocks_tested(k0, mo, mstat, sg);
    *hit = h;
  }
  if (per) {
    per[0] = f[0]; per[1] = f[1]; per[2] = f[2];
    per[3] = A[0]; per[4] = A[1]; per[5] = A[2]; per[6] = A[3]; per[7] = A[4]; per[8] = A[5];
  }
}

// ------------------------------------------------------------------ fused raycast kernel
// Thread g of the launch handles segment g % S of the ray in slot g / S; the S segments of a
// ray sit in adjacent lanes, and the ray's result is the first segment (lowest index) that
// hit or left the map, else the last one -- found with a warp ballot and moved to the
// ray's first lane by shuffles.  That lane evaluates the policy and writes the outputs.
template <int KIND, int LAYOUT, int RED, bool CELLS>
__global__ void __launch_bounds__(256) raycast_rmp_kernel(DevMap m, EvalConsts k,
                                                          const double* __restrict__ state,
                                                          WsHeader* ws, CtaPartial* parts,
                                                          rmp_result_t* out, rmp_ray_hit_t* hits,
                                                          float* per_ray) {
  extern __shared__ uint4 smem_radius[];
  __shared__ CtaState cs;
  __shared__ __align__(8) uint64_t bm_bar;
  __shared__ int bm_timeout;
  const uint32_t bm_bytes = m.radius_words * 4u;
  const bool staged = LAYOUT == kLayoutGrid && bm_bytes <= kMaxSmemRadiusBytes;
  const uint32_t* bm = staged ? reinterpret_cast<const uint32_t*>(smem_radius) : m.radius;
  if (threadIdx.x == 0) {
    bm_timeout = 0;
    if (staged) bulk_load_begin(&bm_bar, smem_radius, m.radius, bm_bytes);
  }
  // state component of this thread: x on threads 0-2, xdot on threads 32-34 (another warp,
  // so the two FP64 chains below run side by side instead of one after the other), loaded
  // before the first ray is generated so that the ray's arithmetic covers the load
  const int comp = state_component(threadIdx.x);
  const double sv = comp >= 0 ? state_at(state, k, comp) : 0.0;
  typename BlockReduce<RED>::Acc acc;
  BlockReduce<RED>::init(acc);
  unsigned n_hit = 0, n_act = 0;
  const uint32_t lgS = k.lg_segs, S = 1u << lgS;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t total = k.n_rays << lgS;
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
  // the first ray is generated while the radius copy and the state loads are in flight
  uint32_t ray_idx = ray_of_slot(base + lane < total ? (base + lane) >> lgS : 0, k);
  Ray ray = make_ray(ray_idx + k.halton_offset);
  if (comp >= 0 && comp < 3) {
    const double o = KIND != RMP_MAP_DENSE_U8 ? 0.0
                     : (comp == 0 ? m.origin[0] : (comp == 1 ? m.origin[1] : m.origin[2]));
    const double q = __dmul_rn(__ddiv_rn(__dsub_rn(sv, o), m.vs), 65536.0);
    // |voxel| < 2^22 keeps block keys and fixed-point products in range; NaN fails too
    const int bad = !(fabs(q) < 274877906944.0);
    cs.bad[comp] = bad;
    cs.P[comp] = bad ? 0 : __double2ll_rn(q);
  } else if (comp >= 3) {
    split_velocity(sv, cs, comp - 3);
  }
  __syncthreads();                                  // state ready, barrier initialised
  if (staged && !bulk_load_wait(&bm_bar)) bm_timeout = 1;
  __syncthreads();
  const bool bad = (cs.bad[0] | cs.bad[1] | cs.bad[2] | bm_timeout) != 0;
  bool first = true;
  // this lane's column of its warp's staged brick words, after the radius field: one
  // shared load per voxel test instead of a select tree over 16 registers (measured, 65536
  // rays on the hashed map: 68.8 -> 65.8 us)
  uint32_t* sbr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem_radius) +
                                              (staged ? bm_bytes : 0u)) +
                  (threadIdx.x >> 5) * (kSmemBrickBytes / 4) + (threadIdx.x & 31);
  // warp-uniform trip count: every lane takes part in each ballot / shuffle
  for (; base < total; base += stride) {
    const uint32_t g = base + lane;
    const bool active = g < total;
    const uint32_t seg = g & (S - 1);
    if (!first) {
      ray_idx = ray_of_slot(active ? (g >> lgS) : 0, k);
      ray = make_ray(ray_idx + k.halton_offset);
    }
    first = false;
    const long long P[3] = {cs.P[0], cs.P[1], cs.P[2]};
    MarchState mo;
    const int mstat = march_ray<KIND, LAYOUT, CELLS>(m, bm, k, P, ray, seg, lgS,
                                                           active && !bad, mo, sbr);
    if (!active || bad || seg != 0) continue;
    float vals[9];
    ray_outputs(m, k, P, ray, mo, mstat, cs.v, cs.vl, hits ? hits + ray_idx : nullptr,
                per_ray ? per_ray + 9 * (size_t)ray_idx : nullptr, vals, n_hit, n_act);
    if (mstat == RMP_RAY_HIT) BlockReduce<RED>::add(acc, vals);
  }
  if (staged && bm_timeout) bulk_load_wait(&bm_bar);   // let a late copy land before exit
  __shared__ CtaSums sums;
  BlockReduce<RED>::reduce(acc, n_hit, n_act, sums);
  const int status = bm_timeout ? RMP_ERR_TIMEOUT
                     : ((cs.bad[0] | cs.bad[1] | cs.bad[2]) ? RMP_ERR_INVALID_ARG : RMP_OK);
  grid_finish<RED>(sums, ws, parts, out, k.n_rays, status);
}

// ------------------------------------------------------------------ batched evaluation
// Device form of the host's direction-cell choice, one warp per state: M = 2^a 3^b <=
// n / 32 minimising |log M - log(n / 48)| + 0.5 |log(3^b / (pi 2^a))| (cells close to
// square on the sphere).  The score is piecewise linear in b with its steeper kink where
// M = n / 48, so for a given a only the b next to that kink, b = 0 and the largest b the
// bound allows need checking; lane a checks those, the warp keeps the best (lowest a on
// ties).  Only the work schedule and the summation grouping depend on the choice.
__device__ __forceinline__ uint32_t pick_cells_warp(uint32_t n) {
  const uint32_t lane = threadIdx.x & 31;
  const float L3 = 1.5849625f, LPI = 1.6514961f;   // log2(3), log2(pi)
  const float lt = __log2f(fmaxf((float)n * (1.0f / 48.0f), 1.0f));
  const float lm = __log2f((float)n * (1.0f / 32.0f));
  float best_score = 3.0e38f;
  uint32_t best = 1;
  const int a = (int)lane;
  if (a <= 24 && (32ull << a) <= n) {
    const int bk = (int)floorf((lt - (float)a) / L3);
    const int bm = (int)floorf((lm - (float)a) / L3) + 1;
    const int cand[4] = {0, bk, bk + 1, bm};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int bb = cand[i] < 0 ? 0 : (cand[i] > 15 ? 15 : cand[i]);
      unsigned long long mm = 1ull << a;
      for (int j = 0; j < bb; ++j) mm *= 3ull;
      while (bb > 0 && mm * 32ull > n) {          // largest feasible b <= the candidate
        mm /= 3ull;
        --bb;
      }
      const float score = fabsf((float)a + (float)bb * L3 - lt) +
                          0.5f * fabsf((float)bb * L3 - LPI - (float)a);
      if (score < best_score) {
        best_score = score;
        best = (uint32_t)mm;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, best_score, off);
    const uint32_t m2 = __shfl_down_sync(0xffffffffu, best, off);
    if (s2 < best_score) {                          // strict: the lower lane wins ties
      best_score = s2;
      best = m2;
    }
  }
  return __shfl_sync(0xffffffffu, best, 0);
}

__device__ __forceinline__ uint32_t ray_of_slot_p(uint32_t j, uint32_t M, uint32_t Q, uint32_t R) {
  const uint32_t big = R * (Q + 1);
  uint32_t r, q;
  if (j < big) {
    r = j / (Q + 1);
    q = j - r * (Q + 1);
  } else {
    const uint32_t jj = j - big;
    const uint32_t t = jj / Q;
    r = R + t;
    q = jj - t * Q;
  }
  return r + M * q;
}

// Per-state set-up of a batch (one CTA of 1024 threads).  Phase A, one warp per state:
// validate the ray count, quantise the position (lanes 0-2, FP64), split the velocity
// (lanes 3-5), choose the direction cells, count chunks and groups.  Phase B, one thread
// per state: exclusive block scans assign consecutive chunk and group ranges.  Then the
// tickets and the work counter are cleared and every state without chunks (no rays, or
// invalid) gets its result here.
__global__ void __launch_bounds__(1024) batch_prep_kernel(
    const double* __restrict__ states, const uint32_t* __restrict__ n_rays, uint32_t n_states,
    uint32_t max_rays, DevMap m, EvalConsts k, BatchHeader* hdr, BatchState* bs,
    uint32_t* sticket, uint32_t* gticket, rmp_result_t* out) {
  __shared__ uint32_t s_chunks[1024], s_groups[1024];
  __shared__ uint32_t wsum_c[32], wsum_g[32];
  __shared__ uint32_t carry_c, carry_g;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) {
    carry_c = 0;
    carry_g = 0;
  }
  for (uint32_t base = 0; base < n_states; base += blockDim.x) {
    const uint32_t tile = min(blockDim.x, n_states - base);
    for (uint32_t j = warp; j < tile; j += nwarps) {
      const uint32_t b = base + j;
      const uint32_t n = n_rays[b];
      const double* x = states + 6 * (size_t)b;
      long long Pa = 0;
      int bad_a = 0;
      float va = 0.f, vla = 0.f;
      if (lane < 3) {
        const double o = m.kind != RMP_MAP_DENSE_U8 ? 0.0
                         : (lane == 0 ? m.origin[0] : (lane == 1 ? m.origin[1] : m.origin[2]));
        const double q = __dmul_rn(__ddiv_rn(__dsub_rn(x[lane], o), m.vs), 65536.0);
        bad_a = !(fabs(q) < 274877906944.0);
        Pa = bad_a ? 0 : __double2ll_rn(q);
      } else if (lane < 6) {
        const double v = x[lane];
        va = __double2float_rn(v);
        vla = __double2float_rn(__dsub_rn(v, (double)va));
      }
      const bool bad = (__ballot_sync(0xffffffffu, bad_a != 0) != 0) || n > max_rays;
      const uint32_t M = n >= 32 ? pick_cells_warp(n) : 1u;
      BatchState* sp = bs + b;
      if (lane < 3) sp->P[lane] = Pa;
      else if (lane < 6) {
        sp->v[lane - 3] = va;
        sp->vl[lane - 3] = vla;
      }
      if (lane == 0) {
        // segments per ray: the launch's fixed choice, or the most (up to 4) whose threads
        // the persistent launch holds at once -- either way a function of the state and
        // the launch shape alone, so the result does not depend on the other states of
        // the batch or their order (one state alone, measured: 8192 rays 64.2 -> 53.8 us
        // with 4 segments instead of 2, 32768 rays 81.1 -> 63.8 us with 4 instead of 1,
        // 65536 rays 85.4 -> 77.8 us with 2)
        uint32_t lg = k.lg_segs;
        if (lg > 2u) {
          if (k.seg_threads > 0u) {
            lg = 2u;
            while (lg > 0u && ((unsigned long long)n << lg) > k.seg_threads) --lg;
          } else {
            lg = n <= 4096u ? 2u : (n <= 16384u ? 1u : 0u);
          }
        }
        const uint32_t chunks = (!bad && n > 0) ? ((n << lg) + 31) / 32 : 0u;
        sp->n_rays = n;
        sp->status = bad ? RMP_ERR_INVALID_ARG : RMP_OK;
        sp->n_chunks = chunks;
        sp->perm_M = M;
        sp->perm_Q = n / M;
        sp->lg_segs = lg;
        s_chunks[j] = chunks;
        s_groups[j] = (chunks + kBatchGroup - 1) / kBatchGroup;
      }
    }
    __syncthreads();
    const uint32_t chunks = tid < tile ? s_chunks[tid] : 0u;
    const uint32_t groups = tid < tile ? s_groups[tid] : 0u;
    uint32_t ic = chunks, ig = groups;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t c2 = __shfl_up_sync(0xffffffffu, ic, off);
      const uint32_t g2 = __shfl_up_sync(0xffffffffu, ig, off);
      if (lane >= (uint32_t)off) {
        ic += c2;
        ig += g2;
      }
    }
    if (lane == 31) {
      wsum_c[warp] = ic;
      wsum_g[warp] = ig;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t wc = lane < nwarps ? wsum_c[lane] : 0u;
      uint32_t wg = lane < nwarps ? wsum_g[lane] : 0u;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t c2 = __shfl_up_sync(0xffffffffu, wc, off);
        const uint32_t g2 = __shfl_up_sync(0xffffffffu, wg, off);
        if (lane >= (uint32_t)off) {
          wc += c2;
          wg += g2;
        }
      }
      wsum_c[lane] = wc;   // inclusive over warps
      wsum_g[lane] = wg;
    }
    __syncthreads();
    const uint32_t pre_c = carry_c + (warp ? wsum_c[warp - 1] : 0u) + ic - chunks;
    const uint32_t pre_g = carry_g + (warp ? wsum_g[warp - 1] : 0u) + ig - groups;
    if (tid < tile) {
      const uint32_t b = base + tid;
      bs[b].chunk0 = pre_c;
      bs[b].group0 = pre_g;
      sticket[b] = 0;
      if (chunks == 0) {
        rmp_result_t r;
        memset(&r, 0, sizeof(r));
        r.n_rays = bs[b].n_rays;
        r.status = bs[b].status;
        out[b] = r;
      }
    }
    __syncthreads();
    if (tid == blockDim.x - 1) {
      carry_c = pre_c + chunks;
      carry_g = pre_g + groups;
    }
    __syncthreads();
  }
  for (uint32_t i = tid; i < carry_g; i += blockDim.x) gticket[i] = 0;
  if (tid == 0) {
    hdr->next_chunk = 0;
    hdr->total_chunks = carry_c;
    hdr->n_states = n_states;
  }
}

// Sum of a partial over the lanes of a warp (lane i holds p_i; lanes without one hold 0):
// FP64 shuffle tree in a fixed order, result in lane 0.
__device__ __forceinline__ void warp_sum_partial(double v[9], unsigned& h, unsigned& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  h = __reduce_add_sync(0xffffffffu, h);
  a = __reduce_add_sync(0xffffffffu, a);
}

__device__ __forceinline__ void load_partial(const CtaPartial* p, double v[9], unsigned& h,
                                             unsigned& a) {
#pragma unroll
  for (int q = 0; q < 9; ++q) v[q] = __ldcg(&p->v[q]);
  h = __ldcg(&p->n_hits);
  a = __ldcg(&p->n_active);
}

// Attractor policy (Sec. III-B, Eq. attractorPolicy) combined by Eq. (1): its metric I is
// added to sum A and f_a = alpha s(goal - x) - beta xdot to sum A f, in FP64 -- after
// dividing the ray sums by the ray count when the ray policies' mean is asked for.
__device__ __forceinline__ void add_attractor(const EvalConsts& k, const double* st,
                                              const double* goal, uint32_t n_rays, double tv[9]) {
  if (k.att_mean && n_rays > 0)
#pragma unroll
    for (int i = 0; i < 9; ++i) tv[i] = tv[i] / (double)n_rays;
  const double v0 = goal[0] - st[0], v1 = goal[1] - st[1], v2 = goal[2] - st[2];
  const double z = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  const double h = z + k.c64 * log1p(exp(-2.0 * k.c64 * z));
  tv[0] += 1.0;
  tv[3] += 1.0;
  tv[5] += 1.0;
  tv[6] += k.att_alpha * (v0 / h) - k.att_beta * st[3];
  tv[7] += k.att_alpha * (v1 / h) - k.att_beta * st[4];
  tv[8] += k.att_alpha * (v2 / h) - k.att_beta * st[5];
}

// Occupancy of voxel (kx, ky, kz) (global voxel coordinates, inside the map for dense
// maps): the block's radius or hash entry, then the brick bit.
template <int LAYOUT>
__device__ __forceinline__ bool voxel_occupied(const DevMap& m, int kx, int ky, int kz) {
  const uint4* src = nullptr;
  if (block_radius<LAYOUT>(m, m.radius, kx >> 3, ky >> 3, kz >> 3, &src) > 0) return false;
  Brick w;
  load_brick(src, w);
  return brick_bit(w, kx, ky, kz);
}

// One control step of point robot b (Sec. IV-A closed loop): the combined policy's
// acceleration f (res[b]) is integrated by semi-implicit Euler in FP64,
// xdot' = xdot + f dt, x' = x + xdot' dt; then, in this order: outside a dense grid ->
// LEFT_MAP; the voxel of x' occupied -> COLLIDED; |x' - goal| < goal_tol -> REACHED;
// steps == max_steps -> TIMEOUT.  Every seg_steps steps the displacement since the last
// segment end is a segment, and consecutive segments A, B add 1 - acos(cos(A, B)) / pi to
// the smoothness sum.  A robot that stops running gets 0 rays from then on.
template <int KIND, int LAYOUT>
__global__ void rollout_step_kernel(DevMap m, RolloutConsts rc, const rmp_result_t* __restrict__ res,
                                    double* states, const double* __restrict__ goals,
                                    uint32_t* n_rays, RolloutDev* rs, uint32_t n,
                                    uint32_t* running) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  RolloutDev& r = rs[b];
  if (r.status != RMP_ROLLOUT_RUNNING) {
    n_rays[b] = 0;
    return;
  }
  double* st = states + 6 * (size_t)b;
  const rmp_result_t& e = res[b];
  if (e.status != RMP_OK) {
    r.status = RMP_ROLLOUT_FAILED;
    n_rays[b] = 0;
    return;
  }
  double dl = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double vd = st[3 + a] + e.f[a] * rc.dt;
    const double xn = st[a] + vd * rc.dt;
    dl += (xn - st[a]) * (xn - st[a]);
    st[3 + a] = vd;
    st[a] = xn;
  }
  r.path_length += sqrt(dl);
  r.steps += 1;
  if (rc.seg_steps && r.steps % rc.seg_steps == 0) {
    double seg[3];
    for (int a = 0; a < 3; ++a) {
      seg[a] = st[a] - r.seg_start[a];
      r.seg_start[a] = st[a];
    }
    if (r.have_prev) {
      double dot = 0.0, na = 0.0, nb = 0.0;
      for (int a = 0; a < 3; ++a) {
        dot += r.prev_seg[a] * seg[a];
        na += r.prev_seg[a] * r.prev_seg[a];
        nb += seg[a] * seg[a];
      }
      if (na > 0.0 && nb > 0.0) {
        double cs = dot / (sqrt(na) * sqrt(nb));
        cs = cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs);
        r.smooth_sum += 1.0 - acos(cs) / 3.14159265358979323846;
        r.smooth_n += 1;
      }
    }
    for (int a = 0; a < 3; ++a) r.prev_seg[a] = seg[a];
    r.have_prev = 1;
  }
  int k[3];
  bool far = false;
  for (int a = 0; a < 3; ++a) {
    const double o = KIND == RMP_MAP_DENSE_U8 ? (a == 0 ? m.origin[0] : (a == 1 ? m.origin[1] : m.origin[2]))
                                              : 0.0;
    const double q = __dmul_rn(__ddiv_rn(__dsub_rn(st[a], o), m.vs), 65536.0);
    far = far || !(fabs(q) < 274877906944.0);
    k[a] = far ? 0 : (int)(__double2ll_rn(q) >> 16);
  }
  double dg = 0.0;
  for (int a = 0; a < 3; ++a) dg += (st[a] - goals[3 * (size_t)b + a]) * (st[a] - goals[3 * (size_t)b + a]);
  if (far || (KIND == RMP_MAP_DENSE_U8 && outside<KIND>(m, k))) r.status = RMP_ROLLOUT_LEFT_MAP;
  else if (voxel_occupied<LAYOUT>(m, k[0], k[1], k[2])) r.status = RMP_ROLLOUT_COLLIDED;
  else if (sqrt(dg) < rc.goal_tol) r.status = RMP_ROLLOUT_REACHED;
  else if (r.steps >= rc.max_steps) r.status = RMP_ROLLOUT_TIMEOUT;
  if (r.status != RMP_ROLLOUT_RUNNING) n_rays[b] = 0;
  else if (running) atomicAdd(running, 1u);
}

// The last chunk of a group sums the group's chunk partials into a group partial; the last
// group of a state sums the state's groups, adds the attractor (combined evaluations) and
// resolves.  Called by all 32 lanes of the warp whose chunk completed the group.  Kept
// out of line: it runs once per 32 chunks, and inlined it would sit between the march
// loops in the instruction stream.
__device__ __noinline__ void batch_group_finish(const EvalConsts& k, CtaPartial* cparts,
                                                CtaPartial* gparts, uint32_t* sticket,
                                                uint32_t chunk0, uint32_t gi, uint32_t gsz,
                                                uint32_t n_chunks, uint32_t group0, uint32_t b,
                                                uint32_t n_b, const double* states,
                                                const double* goals, rmp_result_t* out) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t stage = 0;
  // last chunk of its group: sum the group's chunk partials (lane i: chunk i)
  __threadfence();
  double gv[9] = {0., 0., 0., 0., 0., 0., 0., 0., 0.};
  unsigned gh = 0, ga = 0;
  if (lane < gsz) load_partial(cparts + chunk0 + gi * kBatchGroup + lane, gv, gh, ga);
  warp_sum_partial(gv, gh, ga);
  const uint32_t n_groups = (n_chunks + kBatchGroup - 1) / kBatchGroup;
  if (lane == 0) {
    CtaPartial p;
#pragma unroll
    for (int i = 0; i < 9; ++i) p.v[i] = gv[i];
    p.n_hits = gh;
    p.n_active = ga;
    gparts[group0 + gi] = p;
    __threadfence();
    stage = atomicAdd(&sticket[b], 1u) == n_groups - 1 ? 2u : 0u;
  }
  stage = __shfl_sync(0xffffffffu, stage, 0);
  if (stage == 2) {
    // last group of the state: lane i sums groups i, i + 32, ... in order, then the tree
    __threadfence();
    double tv[9] = {0., 0., 0., 0., 0., 0., 0., 0., 0.};
    unsigned th = 0, ta = 0;
    for (uint32_t j = lane; j < n_groups; j += 32) {
      double pv2[9];
      unsigned h2, a2;
      load_partial(gparts + group0 + j, pv2, h2, a2);
#pragma unroll
      for (int i = 0; i < 9; ++i) tv[i] += pv2[i];
      th += h2;
      ta += a2;
    }
    warp_sum_partial(tv, th, ta);
    if (goals && lane == 0)
      add_attractor(k, states + 6 * (size_t)b, goals + 3 * (size_t)b, n_b, tv);
#pragma unroll
    for (int i = 0; i < 9; ++i) tv[i] = __shfl_sync(0xffffffffu, tv[i], 0);
    rmp_result_t r;
    resolve_pinv(tv, tv + 6, r);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) r.A[i] = tv[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) r.Af[i] = tv[6 + i];
      r.n_rays = n_b;
      r.n_hits = th;
      r.n_active = ta;
      r.status = RMP_OK;
      r.reserved = 0;
      out[b] = r;
    }
  }
}

// Persistent batched evaluation: every warp takes chunks (its own index first, then from
// the work counter) until none is left; a chunk is 32 / S rays of one state (coherent ray order of that state), marched
// and evaluated as in the single-state kernel.  The chunk's 9 terms are summed over the
// warp (compensated FP32 or FP64 tree), stored, and the chunk's group and state tickets
// decide which warp sums a group (<= 32 chunk partials, one per lane) and which one sums
// the state's groups and resolves it -- every sum in a fixed order, so results do not
// depend on which warp ran which chunk.
// Register budget 64 (launch bounds 256 x 4): 32 warps per SM instead of 16; the few
// spills cost less than the latency the extra warps hide (measured: 3.42 against 2.77
// Grays/s on 256 states; 80 registers 3.20, 51 registers 3.21; again with the current
// march, 256 states: 64 registers 1.357 ms, 80: 1.516, 128: 1.734).  The in-warp split
// of long pieces is compiled out (its saved piece state made most of the spills: 208 ->
// 48 bytes; it never paid in the autotuner), and the per-state values used only after
// the march are read after it.
template <int KIND, int LAYOUT, int RED>
__global__ void __launch_bounds__(256, 4) raycast_batch_kernel(
    DevMap m, EvalConsts k, BatchHeader* hdr, const BatchState* __restrict__ bs,
    uint32_t* sticket, uint32_t* gticket, CtaPartial* cparts, CtaPartial* gparts,
    rmp_result_t* out, rmp_ray_hit_t* hits, float* per_ray, uint32_t max_rays,
    const double* __restrict__ states, const double* __restrict__ goals) {
  extern __shared__ uint4 smem_radius[];
  __shared__ __align__(8) uint64_t bm_bar;
  __shared__ int bm_timeout;
  const uint32_t bm_bytes = m.radius_words * 4u;
  const bool staged = LAYOUT == kLayoutGrid && bm_bytes <= kMaxSmemRadiusBytes;
  if (threadIdx.x == 0) {
    bm_timeout = 0;
    if (staged) bulk_load_begin(&bm_bar, smem_radius, m.radius, bm_bytes);
  }
  __syncthreads();
  if (staged && threadIdx.x == 0 && !bulk_load_wait(&bm_bar)) bm_timeout = 1;
  __syncthreads();
  // a copy that did not land in time leaves the CTA on the global copy of the field
  const uint32_t* bm = (staged && !bm_timeout) ? reinterpret_cast<const uint32_t*>(smem_radius)
                                               : m.radius;
  // this lane's brick column, after the radius field (batch_smem_bytes)
  uint32_t* sbr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem_radius) +
                                              (staged ? bm_bytes : 0u)) +
                  (threadIdx.x >> 5) * (kSmemBrickBytes / 4) + (threadIdx.x & 31);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t total = *(volatile const uint32_t*)&hdr->total_chunks;
  const uint32_t nst = *(volatile const uint32_t*)&hdr->n_states;
  // first chunk: the warp's index in the grid; later ones from the counter (offset by the
  // number of warps), requested as soon as a chunk starts so the atomic's latency is
  // hidden.  (Same-address atomics are serialised, several ns each: a grid-wide rush on
  // the counter at kernel start would delay every warp's first chunk.)
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  while (c < total) {
    uint32_t cn = 0xffffffffu;
    if (lane == 0 && total > n_warps) cn = n_warps + atomicAdd(&hdr->next_chunk, 1u);
    // the chunk's state: the last one whose first chunk is <= c
    uint32_t lo = 0, hi = nst;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&bs[mid].chunk0) <= c) lo = mid;
      else hi = mid;
    }
    const uint32_t b = lo;
    const BatchState* sp = bs + b;
    const long long P[3] = {__ldg(&sp->P[0]), __ldg(&sp->P[1]), __ldg(&sp->P[2])};
    const uint32_t n_b = __ldg(&sp->n_rays), chunk0 = __ldg(&sp->chunk0);
    const uint32_t q = c - chunk0;
    const uint32_t lgS = __ldg(&sp->lg_segs), S = 1u << lgS;
    const uint32_t g = q * 32 + lane;
    const uint32_t slot = g >> lgS, seg = g & (S - 1);
    const bool active = slot < n_b;
    const uint32_t pM = __ldg(&sp->perm_M), pQ = __ldg(&sp->perm_Q);
    const uint32_t ray_idx = ray_of_slot_p(active ? slot : 0, pM, pQ, n_b - pQ * pM);
    const Ray ray = make_ray(ray_idx + k.halton_offset);
    MarchState mo;
    const int mstat = march_ray<KIND, LAYOUT, true, true, 2>(m, bm, k, P, ray, seg, lgS, active, mo,
                                                          sbr);
    // read after the march, so that they are not held in registers across it
    const float v[3] = {__ldg(&sp->v[0]), __ldg(&sp->v[1]), __ldg(&sp->v[2])};
    const float vl[3] = {__ldg(&sp->vl[0]), __ldg(&sp->vl[1]), __ldg(&sp->vl[2])};
    const uint32_t n_chunks = __ldg(&sp->n_chunks), group0 = __ldg(&sp->group0);
    float vals[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned nh = 0, na = 0;
    if (active && seg == 0) {
      const size_t ro = (size_t)b * max_rays + ray_idx;
      ray_outputs(m, k, P, ray, mo, mstat, v, vl, hits ? hits + ro : nullptr,
                  per_ray ? per_ray + 9 * ro : nullptr, vals, nh, na);
    }
    // chunk partial
    double pv[9];
    if (RED == RMP_REDUCE_FP64) {
#pragma unroll
      for (int i = 0; i < 9; ++i) pv[i] = (double)vals[i];
      warp_sum_partial(pv, nh, na);
    } else {
      Acc32 acc;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        acc.s[i] = vals[i];
        acc.c[i] = 0.0f;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float s2 = __shfl_down_sync(0xffffffffu, acc.s[i], off);
          const float c2 = __shfl_down_sync(0xffffffffu, acc.c[i], off);
          acc_merge(acc, s2, c2, i);
        }
#pragma unroll
      for (int i = 0; i < 9; ++i) pv[i] = (double)acc.s[i] + (double)acc.c[i];
      nh = __reduce_add_sync(0xffffffffu, nh);
      na = __reduce_add_sync(0xffffffffu, na);
    }
    const uint32_t gi = q / kBatchGroup;
    const uint32_t gsz = min(kBatchGroup, n_chunks - gi * kBatchGroup);
    uint32_t stage = 0;
    if (lane == 0) {
      CtaPartial p;
#pragma unroll
      for (int i = 0; i < 9; ++i) p.v[i] = pv[i];
      p.n_hits = nh;
      p.n_active = na;
      cparts[chunk0 + q] = p;
      __threadfence();
      stage = atomicAdd(&gticket[group0 + gi], 1u) == gsz - 1 ? 1u : 0u;
    }
    stage = __shfl_sync(0xffffffffu, stage, 0);
    if (stage)
      batch_group_finish(k, cparts, gparts, sticket, chunk0, gi, gsz, n_chunks, group0, b, n_b,
                         states, goals, out);
    c = __shfl_sync(0xffffffffu, cn, 0);
  }
  if (staged && bm_timeout && threadIdx.x == 0) bulk_load_wait(&bm_bar);   // let a late copy land
}

// ------------------------------------------------------------------ L2 bandwidth probe
// Reads n16 uint4 words `passes` times, grid-stride, 16-byte loads cached in L2 only
// (ld.global.cg), four independent loads in flight per thread; XOR of everything read per
// CTA into checksum[blockIdx.x].
__global__ void __launch_bounds__(512) probe_l2_kernel(const uint4* __restrict__ buf, size_t n16,
                                                       uint32_t passes, uint64_t* checksum) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (uint32_t p = 0; p < passes; ++p) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride),
                  c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
             d.z ^ d.w;
    }
    for (; i < n16; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  acc = __reduce_xor_sync(0xffffffffu, acc);
  __shared__ uint32_t warp_acc[16];
  if ((threadIdx.x & 31) == 0) warp_acc[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) t ^= warp_acc[w];
    checksum[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------ ESDF policy (Sec. III-D)
// Signed distance of one primitive at x, in the fixed FP64 order of the ABI's definition
// (explicitly rounded operations: no contraction may change the distance or the argmin).
__device__ __forceinline__ double esdf_prim_sdf(const rmp_primitive_t& p, const double x[3]) {
  const double q0 = __dsub_rn(x[0], p.center[0]), q1 = __dsub_rn(x[1], p.center[1]),
               q2 = __dsub_rn(x[2], p.center[2]);
  if (p.kind == RMP_PRIM_SPHERE)
    return __dsub_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)),
                                          __dmul_rn(q2, q2))),
                     p.size[0]);
  const double a0 = __dsub_rn(fabs(q0), p.size[0]), a1 = __dsub_rn(fabs(q1), p.size[1]),
               a2 = __dsub_rn(fabs(q2), p.size[2]);
  const double o0 = a0 > 0.0 ? a0 : 0.0, o1 = a1 > 0.0 ? a1 : 0.0, o2 = a2 > 0.0 ? a2 : 0.0;
  const double out = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(o0, o0), __dmul_rn(o1, o1)),
                                          __dmul_rn(o2, o2)));
  double in = a0 > a1 ? a0 : a1;
  in = in > a2 ? in : a2;
  in = in < 0.0 ? in : 0.0;
  return __dadd_rn(out, in);
}

// Gradient of one primitive's distance at x (unit, pointing away from the primitive).
__device__ __forceinline__ void esdf_prim_grad(const rmp_primitive_t& p, const double x[3],
                                               double g[3]) {
  const double q[3] = {__dsub_rn(x[0], p.center[0]), __dsub_rn(x[1], p.center[1]),
                       __dsub_rn(x[2], p.center[2])};
  if (p.kind == RMP_PRIM_SPHERE) {
    const double L = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])),
                                          __dmul_rn(q[2], q[2])));
    for (int a = 0; a < 3; ++a) g[a] = L > 0.0 ? __ddiv_rn(q[a], L) : 0.0;
    return;
  }
  double ai[3], o[3];
  for (int a = 0; a < 3; ++a) {
    ai[a] = __dsub_rn(fabs(q[a]), p.size[a]);
    o[a] = ai[a] > 0.0 ? ai[a] : 0.0;
  }
  const double out = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(o[0], o[0]), __dmul_rn(o[1], o[1])),
                                          __dmul_rn(o[2], o[2])));
  if (out > 0.0) {
    for (int a = 0; a < 3; ++a) g[a] = __ddiv_rn(q[a] < 0.0 ? -o[a] : o[a], out);
    return;
  }
  const int k = (ai[0] >= ai[1] && ai[0] >= ai[2]) ? 0 : (ai[1] >= ai[2] ? 1 : 2);
  for (int a = 0; a < 3; ++a) g[a] = a == k ? (q[a] < 0.0 ? -1.0 : 1.0) : 0.0;
}

// One warp per state: the lanes scan the primitives (lane i: i, i + 32, ...), the warp keeps
// the smallest distance (lowest index on ties: the first minimum of a sequential scan);
// lane 0 evaluates the obstacle policy of Sec. III-C on (d, gradient) in FP64 and adds the
// attractor; the warp resolves Eq. (1).
__global__ void __launch_bounds__(256) esdf_eval_kernel(const rmp_primitive_t* __restrict__ prims,
                                                        uint32_t n_prims, EsdfConsts k,
                                                        const double* __restrict__ states,
                                                        const double* __restrict__ goals,
                                                        uint32_t n_states, rmp_result_t* out,
                                                        double* query) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < n_states;
       b += n_warps) {
    const double* st = states + 6 * (size_t)b;
    const double x[3] = {st[0], st[1], st[2]};
    const double v[3] = {st[3], st[4], st[5]};
    bool bad = false;
    for (int a = 0; a < 6; ++a) bad = bad || !isfinite(st[a]);
    double best = INFINITY;
    uint32_t bi = 0xffffffffu;
    if (!bad)
      for (uint32_t i = lane; i < n_prims; i += 32) {
        const double sd = esdf_prim_sdf(prims[i], x);
        if (sd < best) {                  // strict: a lane's earlier primitive wins ties
          best = sd;
          bi = i;
        }
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double b2 = __shfl_down_sync(0xffffffffu, best, off);
      const uint32_t i2 = __shfl_down_sync(0xffffffffu, bi, off);
      if (b2 < best || (b2 == best && i2 < bi)) {
        best = b2;
        bi = i2;
      }
    }
    double tv[9] = {0., 0., 0., 0., 0., 0., 0., 0., 0.};
    double d = INFINITY, g[3] = {0.0, 0.0, 0.0};
    unsigned hit = 0, act = 0;
    if (lane == 0 && !bad) {
      if (bi != 0xffffffffu) {
        d = best > 0.0 ? best : 0.0;
        esdf_prim_grad(prims[bi], x, g);
        hit = 1;
        // obstacle policy (Sec. III-C) on the single pair (d, r = g), FP64
        const double xr = __dadd_rn(__dadd_rn(__dmul_rn(v[0], g[0]), __dmul_rn(v[1], g[1])),
                                    __dmul_rn(v[2], g[2]));
        const bool active = xr < 0.0, in_r = d < k.r;
        act = (active && in_r) ? 1u : 0u;
        const double frep = k.eta_rep * exp(-d / k.nu_rep);
        const double m = active ? xr * xr : 0.0;
        const double kd = k.eta_damp / (d / k.nu_damp + k.eps);
        const double z = kd * m;                          // |f_damp|
        double w = 0.0;
        if (in_r) {
          const double y = (k.r - d) / k.r;               // 1 - d / r, exact difference
          w = k.w_mode == 0 ? y * y : y * y * (1.0 + 2.0 * (d / k.r));
        }
        const double h = z + k.c * log1p(exp(-2.0 * k.c * z));
        const double sc = h > 0.0 ? z / h : 0.0;
        const double alpha_m = w * sc * sc;               // A = alpha_m r r^T
        const double fr = frep + z;                       // f = fr r
        tv[0] = alpha_m * g[0] * g[0];
        tv[1] = alpha_m * g[0] * g[1];
        tv[2] = alpha_m * g[0] * g[2];
        tv[3] = alpha_m * g[1] * g[1];
        tv[4] = alpha_m * g[1] * g[2];
        tv[5] = alpha_m * g[2] * g[2];
        const double rf = fr * ((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
        for (int a = 0; a < 3; ++a) tv[6 + a] = alpha_m * rf * g[a];
      }
      if (goals) {                                         // attractor, metric I (Eq. 1)
        const double* gl = goals + 3 * (size_t)b;
        const double e0 = gl[0] - x[0], e1 = gl[1] - x[1], e2 = gl[2] - x[2];
        const double zz = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        const double hh = zz + k.c * log1p(exp(-2.0 * k.c * zz));
        tv[0] += 1.0;
        tv[3] += 1.0;
        tv[5] += 1.0;
        tv[6] += k.alpha * (e0 / hh) - k.beta * v[0];
        tv[7] += k.alpha * (e1 / hh) - k.beta * v[1];
        tv[8] += k.alpha * (e2 / hh) - k.beta * v[2];
      }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) tv[i] = __shfl_sync(0xffffffffu, tv[i], 0);
    rmp_result_t r;
    resolve_pinv(tv, tv + 6, r);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) r.A[i] = tv[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) r.Af[i] = tv[6 + i];
      r.n_rays = 1;
      r.n_hits = hit;
      r.n_active = act;
      r.status = bad ? RMP_ERR_INVALID_ARG : RMP_OK;
      r.reserved = 0;
      if (bad) {
        r.f[0] = r.f[1] = r.f[2] = 0.0;
        r.eig[0] = r.eig[1] = r.eig[2] = 0.0;
        r.rank = 0;
      }
      out[b] = r;
      if (query) {
        double* qd = query + 4 * (size_t)b;
        qd[0] = d;
        qd[1] = g[0];
        qd[2] = g[1];
        qd[3] = g[2];
      }
    }
  }
}

// ------------------------------------------------------------------ LiDAR scan kernel (Sec. III-G)
template <int RED>
__global__ void __launch_bounds__(256) scan_rmp_kernel(const float* __restrict__ pts,
                                                       EvalConsts k,
                                                       const double* __restrict__ state,
                                                       WsHeader* ws, CtaPartial* parts,
                                                       rmp_result_t* out, float* per_ray) {
  __shared__ CtaState cs;
  const int comp = state_component(threadIdx.x);
  if (comp >= 0 && comp < 3) cs.xf[comp] = __double2float_rn(state_at(state, k, comp));
  else if (comp >= 3) split_velocity(state_at(state, k, comp), cs, comp - 3);
  __syncthreads();
  typename BlockReduce<RED>::Acc acc;
  BlockReduce<RED>::init(acc);
  unsigned n_hit = 0, n_act = 0;
  const float v[3] = {cs.v[0], cs.v[1], cs.v[2]};
  const float vl[3] = {cs.vl[0], cs.vl[1], cs.vl[2]};
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < k.n_rays;
       j += gridDim.x * blockDim.x) {
    float q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = __fsub_rn(__ldg(pts + 3 * (size_t)j + a), cs.xf[a]);
    float f[3] = {0.f, 0.f, 0.f}, A[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, af[3];
    bool valid = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]);
    float d = 0.0f;
    if (valid) {
      d = __fsqrt_rn(__fmaf_rn(q[2], q[2], __fmaf_rn(q[1], q[1], __fmul_rn(q[0], q[0]))));
      valid = d > 0.0f && d >= k.min_up && d <= k.max_dn;
    }
    if (valid) {
      const float u[3] = {__fdiv_rn(q[0], d), __fdiv_rn(q[1], d), __fdiv_rn(q[2], d)};
      const bool act = active32(v, u);
      const bool inr = d < k.r_up;
      n_hit += 1;
      n_act += (act && inr) ? 1u : 0u;
      obstacle_policy(k, u, d, v, vl, act, inr, f, A, af);
      const float vals[9] = {A[0], A[1], A[2], A[3], A[4], A[5], af[0], af[1], af[2]};
      BlockReduce<RED>::add(acc, vals);
    }
    if (per_ray) {
      float* o = per_ray + 9 * (size_t)j;
      o[0] = f[0]; o[1] = f[1]; o[2] = f[2];
      o[3] = A[0]; o[4] = A[1]; o[5] = A[2]; o[6] = A[3]; o[7] = A[4]; o[8] = A[5];
    }
  }
  __shared__ CtaSums sums;
  BlockReduce<RED>::reduce(acc, n_hit, n_act, sums);
  grid_finish<RED>(sums, ws, parts, out, k.n_rays, RMP_OK);
}

// ------------------------------------------------------------------ map build kernels
// Dense grid -> bricks: thread per (brick, word); word w covers lz = w/2 and
// ly = 4 (w&1) .. +3, lx = 0..7.
__global__ void dense_bricks_kernel(const uint8_t* __restrict__ occ, int dx, int dy, int dz,
                                    int nbx, int nby, int nbz, uint32_t* __restrict__ bricks) {
  const size_t total = (size_t)nbx * nby * nbz * kBrickWords;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t brick = idx / kBrickWords;
    const int w = (int)(idx % kBrickWords);
    const int bx = (int)(brick % nbx), by = (int)((brick / nbx) % nby), bz = (int)(brick / ((size_t)nbx * nby));
    const int z = bz * 8 + (w >> 1);
    uint32_t word = 0;
    for (int r = 0; r < 4; ++r) {
      const int y = by * 8 + 4 * (w & 1) + r;
      for (int lx = 0; lx < 8; ++lx) {
        const int x = bx * 8 + lx;
        if (x < dx && y < dy && z < dz && occ[(size_t)x + (size_t)dx * ((size_t)y + (size_t)dy * z)] != 0)
          word |= 1u << (lx + 8 * r);
      }
    }
    bricks[idx] = word;
  }
}

// Free-radius field of a grid, in three steps: radius 0 for bricks with an occupied voxel
// and 15 otherwise; kMaxFreeRadius - 1 relaxation passes v(b) = min(v(b), 1 + min over the
// 26 neighbours v(n)) (neighbours outside the grid count as free), which yields the
// Chebyshev distance to the nearest occupied brick capped at 15; then packing to 4 bits.
__global__ void radius_init_kernel(const uint4* __restrict__ bricks, uint32_t n_bricks,
                                   uint8_t* __restrict__ v) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bricks;
       b += gridDim.x * blockDim.x) {
    const uint4* w = bricks + 4 * (size_t)b;
    uint32_t any = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 x = w[q];
      any |= x.x | x.y | x.z | x.w;
    }
    v[b] = any ? 0 : (uint8_t)kMaxFreeRadius;
  }
}

__global__ void radius_relax_kernel(const uint8_t* __restrict__ vin, uint8_t* __restrict__ vout,
                                    int gx, int gy, int gz) {
  const uint32_t n = (uint32_t)gx * gy * gz;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    const int x = (int)(b % (uint32_t)gx), y = (int)((b / (uint32_t)gx) % (uint32_t)gy),
              z = (int)(b / ((uint32_t)gx * gy));
    int best = vin[b];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x + dx, yy = y + dy, zz = z + dz;
          if ((unsigned)xx >= (unsigned)gx || (unsigned)yy >= (unsigned)gy || (unsigned)zz >= (unsigned)gz)
            continue;
          const int c = vin[(uint32_t)xx + (uint32_t)gx * ((uint32_t)yy + (uint32_t)gy * (uint32_t)zz)] + 1;
          best = c < best ? c : best;
        }
    vout[b] = (uint8_t)best;
  }
}

__global__ void radius_pack_kernel(const uint8_t* __restrict__ v, uint32_t n, uint32_t words,
                                   uint32_t* __restrict__ radius) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
    uint32_t word = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t b = w * 8 + i;
      const uint32_t r = b < n ? v[b] : (uint32_t)kMaxFreeRadius;
      word |= (r & 15u) << (4 * i);
    }
    radius[w] = word;
  }
}

// Free distance of each 2^3 cell of the occupied bricks: the Chebyshev distance in voxels
// from the cell to the nearest occupied voxel, capped at kCellDistCap (a free cell at
// distance dv holds no voxel closer than dv to an obstacle, so every voxel of it centres a
// free box of half-width dv - 1).  One CTA per brick: the 3^3 bricks around it are loaded
// into shared memory as a 24^3 bit volume (rows of 24 x-bits), dilated by one voxel in the
// Chebyshev metric kCellDistCap - 1 times (the 3^3 maximum, one pass per dilation); a cell's
// distance is the first dilation that reaches one of its 8 voxels.  Only voxels within
// kCellDistCap - 1 of the centre brick matter, and they lie inside the volume.  Free bricks
// get 0 (never read).
static_assert(kCellDistCap == 4, "the halo of one brick covers dilations up to 3 voxels");
__global__ void __launch_bounds__(256) cell_dist_kernel(const uint32_t* __restrict__ bricks,
                                                        DevMap m, uint64_t n_bricks,
                                                        uint32_t* __restrict__ cells) {
  __shared__ uint32_t vol[2][24][24];   // [z][y], bit x
  __shared__ uint32_t words[8];
  __shared__ int occupied;
  const int t = threadIdx.x;
  const int gx = m.gdim[0], gy = m.gdim[1], gz = m.gdim[2];
  for (uint64_t b = blockIdx.x; b < n_bricks; b += gridDim.x) {
    __syncthreads();                    // the previous brick's shared data is no longer read
    if (t == 0) occupied = 0;
    if (t < 8) words[t] = 0;
    __syncthreads();
    if (t < 16 && __ldg(bricks + 16 * b + t) != 0u) occupied = 1;
    __syncthreads();
    if (!occupied) {
      if (t < 8) cells[8 * b + t] = 0u;
      continue;
    }
    const int bx = (int)(b % (uint64_t)gx);
    const int by = (int)((b / (uint64_t)gx) % (uint64_t)gy);
    const int bz = (int)(b / ((uint64_t)gx * (uint64_t)gy));
    for (int r = t; r < 576; r += blockDim.x) {
      const int zz = r / 24, yy = r - 24 * (r / 24);
      const int nz = bz + zz / 8 - 1, ny = by + yy / 8 - 1;
      const int lz = zz & 7, ly = yy & 7;
      uint32_t row = 0u;
      if ((unsigned)nz < (unsigned)gz && (unsigned)ny < (unsigned)gy) {
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int nx = bx + dx - 1;
          if ((unsigned)nx >= (unsigned)gx) continue;
          const size_t nb = (size_t)nx + (size_t)gx * ((size_t)ny + (size_t)gy * (size_t)nz);
          const uint32_t w = __ldg(bricks + 16 * nb + (ly >> 2) + 2 * lz);
          row |= ((w >> (8 * (ly & 3))) & 0xffu) << (8 * dx);
        }
      }
      vol[0][zz][yy] = row;
    }
    __syncthreads();
    // thread c < 64: cell c of the centre brick (voxels 8 + 2 (c & 3) .. +1 in x, etc.)
    const int cx = 8 + 2 * (t & 3), cy = 8 + 2 * ((t >> 2) & 3), cz = 8 + 2 * ((t >> 4) & 3);
    const uint32_t cmask = 3u << cx;
    int d = kCellDistCap;
    auto touches = [&](int buf) {
      return ((vol[buf][cz][cy] | vol[buf][cz][cy + 1] | vol[buf][cz + 1][cy] |
               vol[buf][cz + 1][cy + 1]) & cmask) != 0u;
    };
    if (t < 64 && touches(0)) d = 0;
    for (int k = 1; k < kCellDistCap; ++k) {
      const int src = (k - 1) & 1, dst = k & 1;
      for (int r = t; r < 576; r += blockDim.x) {
        const int zz = r / 24, yy = r - 24 * (r / 24);
        uint32_t acc = 0u;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const int z2 = zz + dz, y2 = yy + dy;
            if ((unsigned)z2 < 24u && (unsigned)y2 < 24u) acc |= vol[src][z2][y2];
          }
        }
        vol[dst][zz][yy] = (acc | (acc << 1) | (acc >> 1)) & 0xffffffu;
      }
      __syncthreads();
      // the next dilation writes vol[src], whose reads ended at the barrier above, and only
      // reads vol[dst]: no second barrier is needed
      if (t < 64 && d == kCellDistCap && touches(dst)) d = k;
    }
    if (t < 64) atomicOr(&words[t >> 3], (uint32_t)d << (4 * (t & 7)));
    __syncthreads();
    if (t < 8) cells[8 * b + t] = words[t];
  }
}

// Bounding box (min xyz, max xyz) of the blocks whose brick holds an occupied voxel.
__global__ void key_bbox_kernel(const int32_t* __restrict__ keys, const uint4* __restrict__ bricks,
                                uint32_t n_blocks, int* bbox) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += gridDim.x * blockDim.x) {
    const uint4* w = bricks + 4 * (size_t)b;
    uint32_t any = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 x = w[q];
      any |= x.x | x.y | x.z | x.w;
    }
    if (!any) continue;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(bbox + a, keys[3 * (size_t)b + a]);
      atomicMax(bbox + 3 + a, keys[3 * (size_t)b + a]);
    }
  }
}

// Scatter the non-empty bricks of a hashed map into the grid layout.
__global__ void grid_scatter_kernel(const int32_t* __restrict__ keys, const uint4* __restrict__ bricks,
                                    uint32_t n_blocks, DevMap m, uint4* __restrict__ grid) {
  const int gx = m.gmin[0], gy = m.gmin[1], gz = m.gmin[2], dx = m.gdim[0], dy = m.gdim[1];
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += gridDim.x * blockDim.x) {
    const uint4* w = bricks + 4 * (size_t)b;
    const uint4 w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
    const uint32_t any = w0.x | w0.y | w0.z | w0.w | w1.x | w1.y | w1.z | w1.w | w2.x | w2.y |
                         w2.z | w2.w | w3.x | w3.y | w3.z | w3.w;
    if (!any) continue;
    const int x = keys[3 * (size_t)b] - gx, y = keys[3 * (size_t)b + 1] - gy,
              z = keys[3 * (size_t)b + 2] - gz;
    const uint32_t idx = (uint32_t)x + (uint32_t)dx * ((uint32_t)y + (uint32_t)dy * (uint32_t)z);
    uint4* dst = grid + 4 * (size_t)idx;
    dst[0] = w0;
    dst[1] = w1;
    dst[2] = w2;
    dst[3] = w3;
  }
}

// TSDF blocks -> bricks: bit b of block n is tsdf[n*512 + b] <= 0 (the TSDF voxel order
// lx + 8 ly + 64 lz is the brick's bit order).
__global__ void tsdf_bricks_kernel(const float* __restrict__ tsdf, uint32_t n_blocks,
                                   uint32_t* __restrict__ bricks) {
  const size_t total = (size_t)n_blocks * kBrickWords;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const float* t = tsdf + idx * 32;
    uint32_t word = 0;
#pragma unroll 8
    for (int b = 0; b < 32; ++b) word |= (t[b] <= 0.0f ? 1u : 0u) << b;
    bricks[idx] = word;
  }
}

// Insert block keys into the open-addressing table (linear probing, bounded).
// err bits: 1 key out of range, 2 duplicate key, 4 table full.
__global__ void hash_build_kernel(const int32_t* __restrict__ keys, uint32_t n_blocks,
                                  const uint4* __restrict__ bricks, HashEntry* table,
                                  uint32_t cap_mask, int hash_shift, unsigned int* err) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
       b += gridDim.x * blockDim.x) {
    const int bx = keys[3 * (size_t)b], by = keys[3 * (size_t)b + 1], bz = keys[3 * (size_t)b + 2];
    if (bx < -kKeyBias || bx >= kKeyBias || by < -kKeyBias || by >= kKeyBias ||
        bz < -kKeyBias || bz >= kKeyBias) {
      atomicOr(err, 1u);
      continue;
    }
    const unsigned long long key = (unsigned long long)(uint32_t)(bx + kKeyBias) |
                                   ((unsigned long long)(uint32_t)(by + kKeyBias) << 21) |
                                   ((unsigned long long)(uint32_t)(bz + kKeyBias) << 42);
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> hash_shift);
    bool done = false;
    for (uint32_t probe = 0; probe <= cap_mask; ++probe) {
      const unsigned long long prev = atomicCAS(&table[h].key, kEmptyKey, key);
      if (prev == kEmptyKey) {
        const uint4* w = bricks + 4 * (size_t)b;
        uint32_t any = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 x = w[q];
          any |= x.x | x.y | x.z | x.w;
        }
        table[h].slot = any ? b : 0xFFFFFFFFu;   // all-free bricks read as missing
        done = true;
        break;
      }
      if (prev == key) {
        atomicOr(err, 2u);
        done = true;
        break;
      }
      h = (h + 1) & cap_mask;
    }
    if (!done) atomicOr(err, 4u);
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
// The staged radius field (a multiple of 16 bytes) where it fits in shared memory.
static size_t radius_smem_bytes(const DevMap& m) {
  const uint32_t bytes = m.radius_words * 4u;
  if (m.layout == kLayoutGrid && bytes <= kMaxSmemRadiusBytes) return bytes;
  return 0;
}

// Single-state kernel: the radius field, then 16 x 32 brick words for each of up to 8 warps.
size_t raycast_smem_bytes(const DevMap& m) { return radius_smem_bytes(m) + 8 * kSmemBrickBytes; }

// Batch kernel: the radius field, then 16 x 32 brick words per warp of the block.
size_t batch_smem_bytes(const DevMap& m, int block) {
  return radius_smem_bytes(m) + (size_t)(block / 32) * kSmemBrickBytes;
}

// The kernels keep up to 48 KB of the map's radius field in shared memory: ask for the
// largest shared-memory carveout once per device so that register use, not the L1/shared
// split, bounds the CTAs resident per SM (a whole evaluation should fit in one wave).
template <auto Fn>
static void prefer_shared() {
  static uint64_t done_mask = 0;   // one bit per device id < 64, per kernel
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return;
  if (__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & (1ull << dev)) return;
  cudaFuncSetAttribute(Fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  // the batch kernel's dynamic shared memory may exceed the default 48 KB: the radius field
  // (up to kMaxSmemRadiusBytes) plus the staged bricks of up to 8 warps
  cudaFuncSetAttribute(Fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kMaxSmemRadiusBytes + 8 * kSmemBrickBytes));
  __atomic_fetch_or(&done_mask, 1ull << dev, __ATOMIC_ACQ_REL);
}

template <int KIND, int LAYOUT, bool CELLS>
static void launch_raycast_c(const DevMap& m, const EvalConsts& k, const double* state_dev,
                             WsHeader* hdr, CtaPartial* parts, rmp_result_t* out_dev,
                             rmp_ray_hit_t* hits, float* per_ray, int block, int grid,
                             size_t smem, cudaStream_t stream) {
  if (k.reduce_mode == RMP_REDUCE_FP64) {
    prefer_shared<raycast_rmp_kernel<KIND, LAYOUT, RMP_REDUCE_FP64, CELLS>>();
    raycast_rmp_kernel<KIND, LAYOUT, RMP_REDUCE_FP64, CELLS><<<grid, block, smem, stream>>>(
        m, k, state_dev, hdr, parts, out_dev, hits, per_ray);
  } else {
    prefer_shared<raycast_rmp_kernel<KIND, LAYOUT, RMP_REDUCE_KAHAN32, CELLS>>();
    raycast_rmp_kernel<KIND, LAYOUT, RMP_REDUCE_KAHAN32, CELLS><<<grid, block, smem, stream>>>(
        m, k, state_dev, hdr, parts, out_dev, hits, per_ray);
  }
}

template <int KIND, int LAYOUT>
static void launch_raycast_t(const DevMap& m, const EvalConsts& k, const double* state_dev,
                             WsHeader* hdr, CtaPartial* parts, rmp_result_t* out_dev,
                             rmp_ray_hit_t* hits, float* per_ray, int block, int grid,
                             size_t smem, cudaStream_t stream) {
  if (LAYOUT == kLayoutGrid && m.cells)
    launch_raycast_c<KIND, LAYOUT, LAYOUT == kLayoutGrid>(m, k, state_dev, hdr, parts, out_dev,
                                                          hits, per_ray, block, grid, smem, stream);
  else
    launch_raycast_c<KIND, LAYOUT, false>(m, k, state_dev, hdr, parts, out_dev, hits, per_ray,
                                          block, grid, smem, stream);
}

int raycast_occupancy(const DevMap& m, int reduce_mode, int block) {
  int n = 0;
  const size_t smem = raycast_smem_bytes(m);
  cudaError_t e;
  if (m.kind == RMP_MAP_DENSE_U8)
    e = reduce_mode ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_DENSE_U8, kLayoutGrid, RMP_REDUCE_FP64, false>, block, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_DENSE_U8, kLayoutGrid, RMP_REDUCE_KAHAN32, false>, block, smem);
  else if (m.layout == kLayoutGrid)
    e = reduce_mode ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_HASHED_TSDF, kLayoutGrid, RMP_REDUCE_FP64, false>, block, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_HASHED_TSDF, kLayoutGrid, RMP_REDUCE_KAHAN32, false>, block, smem);
  else
    e = reduce_mode ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_HASHED_TSDF, kLayoutHash, RMP_REDUCE_FP64, false>, block, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_rmp_kernel<RMP_MAP_HASHED_TSDF, kLayoutHash, RMP_REDUCE_KAHAN32, false>, block, smem);
  return e == cudaSuccess ? n : -1;
}

cudaError_t launch_raycast(const DevMap& m, const EvalConsts& k, const double* state_dev,
                           void* ws, rmp_result_t* out_dev, rmp_ray_hit_t* hits,
                           float* per_ray, int block, int grid, cudaStream_t stream) {
  // grid_finish needs whole warps 0 and 1 (the resolve's named barrier) and at least 64
  // threads (each summing thread takes at most two of the up to 128 group partials)
  if (block != 64 && block != 128 && block != 256) return cudaErrorInvalidValue;
  WsHeader* hdr = (WsHeader*)ws;
  CtaPartial* parts = (CtaPartial*)((char*)ws + kWsHeaderBytes);
  const size_t smem = raycast_smem_bytes(m);
  if (m.kind == RMP_MAP_DENSE_U8)
    launch_raycast_t<RMP_MAP_DENSE_U8, kLayoutGrid>(m, k, state_dev, hdr, parts, out_dev, hits,
                                                    per_ray, block, grid, smem, stream);
  else if (m.layout == kLayoutGrid)
    launch_raycast_t<RMP_MAP_HASHED_TSDF, kLayoutGrid>(m, k, state_dev, hdr, parts, out_dev, hits,
                                                       per_ray, block, grid, smem, stream);
  else
    launch_raycast_t<RMP_MAP_HASHED_TSDF, kLayoutHash>(m, k, state_dev, hdr, parts, out_dev, hits,
                                                       per_ray, block, grid, smem, stream);
  return cudaGetLastError();
}

template <int KIND, int LAYOUT, int RED>
static int batch_occupancy_t(int block, size_t smem) {
  int n = 0;
  prefer_shared<raycast_batch_kernel<KIND, LAYOUT, RED>>();
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, raycast_batch_kernel<KIND, LAYOUT, RED>,
                                                       block, smem) == cudaSuccess ? n : -1;
}

int batch_occupancy(const DevMap& m, int reduce_mode, int block) {
  const size_t smem = batch_smem_bytes(m, block);
  if (m.kind == RMP_MAP_DENSE_U8)
    return reduce_mode ? batch_occupancy_t<RMP_MAP_DENSE_U8, kLayoutGrid, RMP_REDUCE_FP64>(block, smem)
                       : batch_occupancy_t<RMP_MAP_DENSE_U8, kLayoutGrid, RMP_REDUCE_KAHAN32>(block, smem);
  if (m.layout == kLayoutGrid)
    return reduce_mode ? batch_occupancy_t<RMP_MAP_HASHED_TSDF, kLayoutGrid, RMP_REDUCE_FP64>(block, smem)
                       : batch_occupancy_t<RMP_MAP_HASHED_TSDF, kLayoutGrid, RMP_REDUCE_KAHAN32>(block, smem);
  return reduce_mode ? batch_occupancy_t<RMP_MAP_HASHED_TSDF, kLayoutHash, RMP_REDUCE_FP64>(block, smem)
                     : batch_occupancy_t<RMP_MAP_HASHED_TSDF, kLayoutHash, RMP_REDUCE_KAHAN32>(block, smem);
}

template <int KIND, int LAYOUT, int RED>
static void launch_batch_t(const DevMap& m, const EvalConsts& k, BatchHeader* hdr,
                           const BatchState* bs, uint32_t* sticket, uint32_t* gticket,
                           CtaPartial* cparts, CtaPartial* gparts, rmp_result_t* out,
                           rmp_ray_hit_t* hits, float* per_ray, uint32_t max_rays, int block,
                           int grid, size_t smem, cudaStream_t stream, const double* states,
                           const double* goals) {
  prefer_shared<raycast_batch_kernel<KIND, LAYOUT, RED>>();
  raycast_batch_kernel<KIND, LAYOUT, RED><<<grid, block, smem, stream>>>(
      m, k, hdr, bs, sticket, gticket, cparts, gparts, out, hits, per_ray, max_rays, states,
      goals);
}

template <int KIND, int LAYOUT>
static void launch_batch_r(const DevMap& m, const EvalConsts& k, BatchHeader* hdr,
                           const BatchState* bs, uint32_t* sticket, uint32_t* gticket,
                           CtaPartial* cparts, CtaPartial* gparts, rmp_result_t* out,
                           rmp_ray_hit_t* hits, float* per_ray, uint32_t max_rays, int block,
                           int grid, size_t smem, cudaStream_t stream, const double* states,
                           const double* goals) {
  if (k.reduce_mode == RMP_REDUCE_FP64)
    launch_batch_t<KIND, LAYOUT, RMP_REDUCE_FP64>(m, k, hdr, bs, sticket, gticket, cparts, gparts,
                                                  out, hits, per_ray, max_rays, block, grid, smem,
                                                  stream, states, goals);
  else
    launch_batch_t<KIND, LAYOUT, RMP_REDUCE_KAHAN32>(m, k, hdr, bs, sticket, gticket, cparts,
                                                     gparts, out, hits, per_ray, max_rays, block,
                                                     grid, smem, stream, states, goals);
}

cudaError_t launch_batch(const DevMap& m, const EvalConsts& k, const double* states_dev,
                         const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                         void* ws, rmp_result_t* out_dev, rmp_ray_hit_t* hits, float* per_ray,
                         int block, int grid, cudaStream_t stream, const double* goals_dev) {
  const BatchLayout L = batch_layout(n_states, max_rays);
  char* w = (char*)ws;
  BatchHeader* hdr = (BatchHeader*)w;
  BatchState* bs = (BatchState*)(w + L.states);
  uint32_t* sticket = (uint32_t*)(w + L.sticket);
  uint32_t* gticket = (uint32_t*)(w + L.gticket);
  CtaPartial* cparts = (CtaPartial*)(w + L.cparts);
  CtaPartial* gparts = (CtaPartial*)(w + L.gparts);
  batch_prep_kernel<<<1, 1024, 0, stream>>>(states_dev, n_rays_dev, n_states, max_rays, m, k, hdr,
                                            bs, sticket, gticket, out_dev);
  const size_t smem = batch_smem_bytes(m, block);
  if (m.kind == RMP_MAP_DENSE_U8)
    launch_batch_r<RMP_MAP_DENSE_U8, kLayoutGrid>(m, k, hdr, bs, sticket, gticket, cparts, gparts,
                                                  out_dev, hits, per_ray, max_rays, block, grid,
                                                  smem, stream, states_dev, goals_dev);
  else if (m.layout == kLayoutGrid)
    launch_batch_r<RMP_MAP_HASHED_TSDF, kLayoutGrid>(m, k, hdr, bs, sticket, gticket, cparts,
                                                     gparts, out_dev, hits, per_ray, max_rays,
                                                     block, grid, smem, stream, states_dev,
                                                     goals_dev);
  else
    launch_batch_r<RMP_MAP_HASHED_TSDF, kLayoutHash>(m, k, hdr, bs, sticket, gticket, cparts,
                                                     gparts, out_dev, hits, per_ray, max_rays,
                                                     block, grid, smem, stream, states_dev,
                                                     goals_dev);
  return cudaGetLastError();
}

cudaError_t launch_rollout_step(const DevMap& m, const RolloutConsts& rc, const rmp_result_t* res,
                                double* states, const double* goals, uint32_t* n_rays,
                                RolloutDev* rs, uint32_t n, uint32_t* running,
                                cudaStream_t stream) {
  const int block = 128;
  const int grid = (int)((n + block - 1) / block);
  if (m.kind == RMP_MAP_DENSE_U8)
    rollout_step_kernel<RMP_MAP_DENSE_U8, kLayoutGrid><<<grid, block, 0, stream>>>(
        m, rc, res, states, goals, n_rays, rs, n, running);
  else if (m.layout == kLayoutGrid)
    rollout_step_kernel<RMP_MAP_HASHED_TSDF, kLayoutGrid><<<grid, block, 0, stream>>>(
        m, rc, res, states, goals, n_rays, rs, n, running);
  else
    rollout_step_kernel<RMP_MAP_HASHED_TSDF, kLayoutHash><<<grid, block, 0, stream>>>(
        m, rc, res, states, goals, n_rays, rs, n, running);
  return cudaGetLastError();
}

cudaError_t launch_probe_l2(const uint4* buf, size_t n16, uint32_t passes, int grid,
                            uint64_t* checksum, cudaStream_t stream) {
  probe_l2_kernel<<<grid, 512, 0, stream>>>(buf, n16, passes, checksum);
  return cudaGetLastError();
}

cudaError_t launch_esdf_eval(const rmp_primitive_t* prims, uint32_t n_prims, const EsdfConsts& k,
                             const double* states, const double* goals, uint32_t n_states,
                             rmp_result_t* out, double* query, cudaStream_t stream) {
  if (n_states == 0) return cudaSuccess;
  const uint32_t warps = 8;                         // states per 256-thread CTA
  uint32_t grid = (n_states + warps - 1) / warps;
  if (grid > 65535) grid = 65535;                   // warp-stride beyond
  esdf_eval_kernel<<<grid, 32 * warps, 0, stream>>>(prims, n_prims, k, states, goals, n_states,
                                                     out, query);
  return cudaGetLastError();
}

cudaError_t launch_scan(const float* pts, const EvalConsts& k, const double* state_dev,
                        void* ws, rmp_result_t* out_dev, float* per_ray, int block, int grid,
                        cudaStream_t stream) {
  if (block != 64 && block != 128 && block != 256) return cudaErrorInvalidValue;  // as above
  WsHeader* hdr = (WsHeader*)ws;
  CtaPartial* parts = (CtaPartial*)((char*)ws + kWsHeaderBytes);
  if (k.reduce_mode == RMP_REDUCE_FP64)
    scan_rmp_kernel<RMP_REDUCE_FP64><<<grid, block, 0, stream>>>(pts, k, state_dev, hdr, parts,
                                                                 out_dev, per_ray);
  else
    scan_rmp_kernel<RMP_REDUCE_KAHAN32><<<grid, block, 0, stream>>>(pts, k, state_dev, hdr, parts,
                                                                    out_dev, per_ray);
  return cudaGetLastError();
}

cudaError_t launch_dense_bricks(const uint8_t* occ, const int dims[3], const int nb[3],
                                uint32_t* bricks, cudaStream_t stream) {
  const size_t total = (size_t)nb[0] * nb[1] * nb[2] * kBrickWords;
  const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  dense_bricks_kernel<<<grid, 256, 0, stream>>>(occ, dims[0], dims[1], dims[2], nb[0], nb[1],
                                                nb[2], bricks);
  return cudaGetLastError();
}

static int grid_for(size_t n) { return (int)((n + 255) / 256 < 65535 ? ((n + 255) / 256 > 0 ? (n + 255) / 256 : 1) : 65535); }

cudaError_t launch_grid_radius(const uint32_t* bricks, const DevMap& m, uint8_t* scratch_a,
                               uint8_t* scratch_b, uint32_t* radius, cudaStream_t stream) {
  const size_t n = (size_t)m.gdim[0] * m.gdim[1] * m.gdim[2];
  radius_init_kernel<<<grid_for(n), 256, 0, stream>>>((const uint4*)bricks, (uint32_t)n, scratch_a);
  uint8_t* a = scratch_a;
  uint8_t* b = scratch_b;
  for (int it = 0; it < kMaxFreeRadius - 1; ++it) {
    radius_relax_kernel<<<grid_for(n), 256, 0, stream>>>(a, b, m.gdim[0], m.gdim[1], m.gdim[2]);
    uint8_t* t = a;
    a = b;
    b = t;
  }
  radius_pack_kernel<<<grid_for(m.radius_words), 256, 0, stream>>>(a, (uint32_t)n, m.radius_words,
                                                                   radius);
  return cudaGetLastError();
}

cudaError_t launch_cell_dist(const uint32_t* bricks, const DevMap& m, uint32_t* cells,
                             cudaStream_t stream) {
  const uint64_t n = (uint64_t)m.gdim[0] * m.gdim[1] * m.gdim[2];
  const uint64_t g = n < 65536u ? n : 65536u;          // grid-stride beyond
  cell_dist_kernel<<<(unsigned)(g > 0 ? g : 1), 256, 0, stream>>>(bricks, m, n, cells);
  return cudaGetLastError();
}

cudaError_t launch_key_bbox(const int32_t* keys, const uint32_t* bricks, uint32_t n_blocks,
                            int* bbox, cudaStream_t stream) {
  key_bbox_kernel<<<grid_for(n_blocks), 256, 0, stream>>>(keys, (const uint4*)bricks, n_blocks, bbox);
  return cudaGetLastError();
}

cudaError_t launch_grid_scatter(const int32_t* keys, const uint32_t* bricks, uint32_t n_blocks,
                                const DevMap& m, uint32_t* grid_bricks, cudaStream_t stream) {
  grid_scatter_kernel<<<grid_for(n_blocks), 256, 0, stream>>>(keys, (const uint4*)bricks, n_blocks,
                                                              m, (uint4*)grid_bricks);
  return cudaGetLastError();
}

cudaError_t launch_tsdf_bricks(const float* tsdf, uint32_t n_blocks, uint32_t* bricks,
                               cudaStream_t stream) {
  const size_t total = (size_t)n_blocks * kBrickWords;
  const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  tsdf_bricks_kernel<<<grid, 256, 0, stream>>>(tsdf, n_blocks, bricks);
  return cudaGetLastError();
}

cudaError_t launch_hash_build(const int32_t* keys, uint32_t n_blocks, const uint32_t* bricks,
                              HashEntry* table, uint32_t cap_mask, int hash_shift,
                              unsigned int* err, cudaStream_t stream) {
  const int grid = (int)((n_blocks + 255) / 256 < 65535 ? (n_blocks + 255) / 256 : 65535);
  hash_build_kernel<<<grid > 0 ? grid : 1, 256, 0, stream>>>(keys, n_blocks, (const uint4*)bricks,
                                                             table, cap_mask, hash_shift, err);
  return cudaGetLastError();
}

}  // namespace rmp
