/* rmp_oracle.c -- CPU oracle for raycast-RMP evaluation (arXiv 2301.08068).
 *
 * TEST INFRASTRUCTURE, not part of the library: only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg load this file's shared object.  It is a plain,
 * slow, single-threaded statement of the method, kept independent of the CUDA code.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math: several steps are
 * specified to the last bit, and contraction of a*b+c into fma would change them).
 *
 * What each part follows:
 *   Halton directions ........ Sec. III-E, Eq. (halton) and the direction vector after it
 *   raycast function R ....... Sec. III-E (d_i = R(x, r_i)) and Sec. III-F; the exact
 *                              fixed-point DDA below is this project's reading (the
 *                              paper's sphere-traced nvblox march has no hit/tie rule)
 *   obstacle policy .......... Sec. III-C: f_rep, g_obs, f_damp, A_obs = w_r s s^T,
 *                              soft normalisation s (Eq. softmax), weight w_r
 *   ray policy ............... Sec. III-E, Eq. (raytracing_policy)
 *   combination / resolve .... Sec. III-A, Eq. (1): f = (sum A)^+ sum A f
 *   LiDAR policy ............. Sec. III-G (beam direction and range replace Halton + R)
 * Parity status: every function here is pinned by the not-gpu tests (closed forms,
 * brute force, library routines, exact rationals); none is "parity unpinned".
 */
#include "rmp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FX_POS 65536        /* 2^16 fixed-point units per voxel along each axis */
#define FX_DIR 16777216.0f  /* 2^24: direction quantisation scale */
#define POW3_20 3486784401u /* 3^20 */

/* ------------------------------------------------------------------ Halton (Eq. halton)
 * H(i, b) is the radical inverse of i in base b: the base-b digits of i mirrored
 * about the radix point. */
float orc_halton2(uint32_t i) {
  double h = 0.0, f = 0.5;            /* every partial sum k/2^m (m <= 32) is exact */
  while (i) {
    if (i & 1u) h += f;
    i >>= 1;
    f *= 0.5;
  }
  return (float)h;                    /* round to nearest float */
}

/* H(i,3) * 3^20 for i < 3^20: the 20 base-3 digits of i in reverse order. */
uint32_t orc_halton3_numerator(uint32_t i) {
  uint64_t num = 0;
  for (int k = 0; k < 20; ++k) {
    num = num * 3u + (i % 3u);
    i /= 3u;
  }
  return (uint32_t)num;
}

/* |num/3^20 - g| scaled by 2^80 * 3^20, exactly (g a float in [0,1]). */
static unsigned __int128 h3_dist(uint32_t num, float g) {
  unsigned __int128 lhs = (unsigned __int128)num << 80;
  double gs = ldexp((double)g, 80);               /* exact: g has 24 significant bits */
  unsigned __int128 rhs = (unsigned __int128)gs * POW3_20;
  return lhs > rhs ? lhs - rhs : rhs - lhs;
}

/* H(i,3) rounded to the nearest float.  The FP64 quotient is a first guess; the
 * nearest of it and its two float neighbours is then picked by exact integer
 * comparison (no ties are possible because 3^20 is odd and num < 3^20). */
float orc_halton3(uint32_t i) {
  uint32_t num = orc_halton3_numerator(i);
  if (num == 0) return 0.0f;
  float g = (float)((double)num / (double)POW3_20);
  float cand[3] = {nextafterf(g, 0.0f), g, nextafterf(g, 2.0f)};
  float best = cand[1];
  unsigned __int128 bd = h3_dist(num, best);
  for (int k = 0; k < 3; k += 2) {
    unsigned __int128 dk = h3_dist(num, cand[k]);
    if (dk < bd) { bd = dk; best = cand[k]; }
  }
  return best;
}

/* ------------------------------------------------------------------ deterministic sincos
 * cos and sin of the angle 2*pi*v (v in [0,1)) in FP32, by one fixed recipe that the
 * CUDA side also follows, so both produce the same bits:
 *   octant q = floor(8v), fraction t = 8v - q (both exact);
 *   reduced argument a = x * RN(pi/4) with x = t for even q and x = 1 - t for odd q;
 *   sin a and cos a from their Taylor series (coefficients RN(1/n!), through a^11 and
 *   a^12), evaluated by Horner's rule with fused multiply-adds;
 *   the octant's symmetry then maps (cos a, sin a) to the full angle. */
static const float PI_4 = 0.78539816339744830962f;

void orc_sincos_turns(float v, float* c_out, float* s_out) {
  float w = v * 8.0f;
  int q = (int)w;
  float t = w - (float)q;
  float x = (q & 1) ? (1.0f - t) : t;
  float a = x * PI_4;
  float a2 = a * a;
  float f3 = 1.0f / 6.0f, f5 = 1.0f / 120.0f, f7 = 1.0f / 5040.0f, f9 = 1.0f / 362880.0f,
        f11 = 1.0f / 39916800.0f;
  float f2 = 1.0f / 2.0f, f4 = 1.0f / 24.0f, f6 = 1.0f / 720.0f, f8 = 1.0f / 40320.0f,
        f10 = 1.0f / 3628800.0f, f12 = 1.0f / 479001600.0f;
  float ps = -f11;
  ps = fmaf(ps, a2, f9);
  ps = fmaf(ps, a2, -f7);
  ps = fmaf(ps, a2, f5);
  ps = fmaf(ps, a2, -f3);
  float a3 = a2 * a;
  float sa = fmaf(a3, ps, a);
  float pc = f12;
  pc = fmaf(pc, a2, -f10);
  pc = fmaf(pc, a2, f8);
  pc = fmaf(pc, a2, -f6);
  pc = fmaf(pc, a2, f4);
  pc = fmaf(pc, a2, -f2);
  float ca = fmaf(a2, pc, 1.0f);
  float c, s;
  switch (q & 7) {
    case 0: c = ca;  s = sa;  break;   /* a            */
    case 1: c = sa;  s = ca;  break;   /* pi/2 - a     */
    case 2: c = -sa; s = ca;  break;   /* pi/2 + a     */
    case 3: c = -ca; s = sa;  break;   /* pi - a       */
    case 4: c = -ca; s = -sa; break;   /* pi + a       */
    case 5: c = -sa; s = -ca; break;   /* 3pi/2 - a    */
    case 6: c = sa;  s = -ca; break;   /* 3pi/2 + a    */
    default: c = ca; s = -sa; break;   /* 2pi - a      */
  }
  *c_out = c;
  *s_out = s;
}

/* Ray direction of Halton index i (Eq. halton with the direction vector after it):
 * polar angle acos(1 - 2 H(i,2)), azimuth 2 pi H(i,3).  cos(polar) = 1 - 2u and
 * sin(polar) = 2 sqrt(u (1 - u)). */
void orc_ray_dir(uint32_t i, float dir[3]) {
  float u = orc_halton2(i);
  float v = orc_halton3(i);
  float z = 1.0f - 2.0f * u;
  float s = 2.0f * sqrtf(u * (1.0f - u));
  float c, sn;
  orc_sincos_turns(v, &c, &sn);
  dir[0] = s * c;
  dir[1] = s * sn;
  dir[2] = z;
}

void orc_ray_dirs(uint32_t n, uint32_t offset, float* dirs) {
  for (uint32_t j = 0; j < n; ++j) orc_ray_dir(j + offset, dirs + 3 * (size_t)j);
}

void orc_quantize_dir(const float dir[3], int32_t D[3]) {
  for (int a = 0; a < 3; ++a) D[a] = (int32_t)rintf(dir[a] * FX_DIR);
}

int64_t orc_quantize_pos(double x, double origin, double vs) {
  return llrint(((x - origin) / vs) * 65536.0);
}

int64_t orc_range_fx(double max_range, double vs) {
  return llrint((max_range / vs) * 65536.0);
}

/* ------------------------------------------------------------------ map lookups */
static const orc_map_t* g_sort_map;

static int key_cmp3(const int32_t* a, const int32_t* b) {
  for (int k = 2; k >= 0; --k) {
    if (a[k] < b[k]) return -1;
    if (a[k] > b[k]) return 1;
  }
  return 0;
}

static int sort_cmp(const void* pa, const void* pb) {
  uint32_t a = *(const uint32_t*)pa, b = *(const uint32_t*)pb;
  return key_cmp3(g_sort_map->keys + 3 * (size_t)a, g_sort_map->keys + 3 * (size_t)b);
}

int orc_map_prepare(orc_map_t* m) {
  m->sorted = NULL;
  if (m->kind != 1) return 0;
  if (m->n_blocks == 0) return 0;
  m->sorted = (uint32_t*)malloc(sizeof(uint32_t) * m->n_blocks);
  if (!m->sorted) return -1;
  for (uint32_t b = 0; b < m->n_blocks; ++b) m->sorted[b] = b;
  g_sort_map = m;
  qsort(m->sorted, m->n_blocks, sizeof(uint32_t), sort_cmp);
  for (uint32_t b = 1; b < m->n_blocks; ++b)   /* duplicate block keys are an error */
    if (key_cmp3(m->keys + 3 * (size_t)m->sorted[b - 1], m->keys + 3 * (size_t)m->sorted[b]) == 0)
      return -2;
  return 0;
}

void orc_map_free(orc_map_t* m) {
  free(m->sorted);
  m->sorted = NULL;
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

/* Block index holding block key kb, or -1 (binary search over the sorted keys). */
static long find_block(const orc_map_t* m, const int32_t kb[3]) {
  long lo = 0, hi = (long)m->n_blocks - 1;
  while (lo <= hi) {
    long mid = (lo + hi) / 2;
    uint32_t b = m->sorted[mid];
    int c = key_cmp3(m->keys + 3 * (size_t)b, kb);
    if (c == 0) return (long)b;
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int inside_dense(const orc_map_t* m, const int64_t k[3]) {
  for (int a = 0; a < 3; ++a)
    if (k[a] < 0 || k[a] >= m->dims[a]) return 0;
  return 1;
}

/* Occupancy of voxel k: dense grid value != 0; hashed map: the voxel's block exists and
 * its TSDF value at the voxel centre is <= 0 (unallocated space is free). */
static int occupied(const orc_map_t* m, const int64_t k[3]) {
  if (m->kind == 0) {
    size_t idx = (size_t)k[0] + (size_t)m->dims[0] * ((size_t)k[1] + (size_t)m->dims[1] * (size_t)k[2]);
    return m->occ[idx] != 0;
  }
  if (m->n_blocks == 0) return 0;
  int32_t kb[3];
  int l[3];
  for (int a = 0; a < 3; ++a) {
    kb[a] = (int32_t)floor_div(k[a], 8);
    l[a] = (int)(k[a] - 8 * (int64_t)kb[a]);
  }
  long b = find_block(m, kb);
  if (b < 0) return 0;
  return m->tsdf[(size_t)b * 512 + (size_t)(l[0] + 8 * l[1] + 64 * l[2])] <= 0.0f;
}

/* ------------------------------------------------------------------ raycast R (exact DDA)
 * Fixed point: position P (units of voxel/2^16, voxel k on an axis spans
 * [k 2^16, (k+1) 2^16)), direction D (units of 2^-24).  The ray crosses the next
 * boundary B_a of axis a at parameter t_a = |B_a - P_a| / |D_a|.  Each iteration
 * steps the one axis with the smallest t_a (exact rational comparison; ties go to
 * the lowest axis, x before y before z).  A voxel is entered only if its entry
 * parameter is within range: N 2^24 <= R_fx |D| with N = |B - P|.  The reported
 * distance of a voxel entered through N/|D| is RN(RN(RN(N/|D|) * 256) * RN(vs)) in
 * FP32 metres (0 for the start voxel). */
static int frac_less(uint64_t n1, uint64_t d1, uint64_t n2, uint64_t d2) {
  return (unsigned __int128)n1 * d2 < (unsigned __int128)n2 * d1;
}

static float entry_distance(uint64_t N, uint64_t absD, double vs) {
  float t = (float)N / (float)absD;
  float t256 = t * 256.0f;
  return t256 * (float)vs;
}

/* Block (8^3-aligned) of voxel k, for counting the distinct blocks a ray tests. */
static void block_of(const int64_t k[3], int64_t b[3]) {
  for (int a = 0; a < 3; ++a) b[a] = floor_div(k[a], 8);
}

int orc_dda(const orc_map_t* m, const int64_t P[3], const int32_t D[3], int64_t R_fx,
            orc_hit_t* out) {
  int64_t k[3], B[3], blk[3], nb[3];
  int sgn[3];
  uint32_t steps = 0, blocks = 0;
  float d = 0.0f;
  for (int a = 0; a < 3; ++a) {
    k[a] = floor_div(P[a], FX_POS);
    sgn[a] = D[a] > 0 ? 1 : (D[a] < 0 ? -1 : 0);
    B[a] = D[a] > 0 ? (k[a] + 1) * FX_POS : k[a] * FX_POS;
  }
  int status;
  block_of(k, blk);
  if (m->kind == 0 && !inside_dense(m, k)) {
    status = ORC_RAY_MISS_EXIT;
  } else if ((blocks = 1, occupied(m, k))) {
    status = ORC_RAY_HIT;
  } else {
    for (;;) {
      int best = -1;
      uint64_t bn = 0, bd = 1;
      for (int a = 0; a < 3; ++a) {
        if (D[a] == 0) continue;                   /* never crosses a boundary */
        uint64_t n = (uint64_t)llabs(B[a] - P[a]);
        uint64_t dd = (uint64_t)llabs((long long)D[a]);
        if (best < 0 || frac_less(n, dd, bn, bd)) { best = a; bn = n; bd = dd; }
      }
      if (((unsigned __int128)bn << 24) > (unsigned __int128)R_fx * bd) {
        status = ORC_RAY_MISS_RANGE;
        break;
      }
      k[best] += sgn[best];
      B[best] += (int64_t)sgn[best] * FX_POS;
      steps += 1;
      d = entry_distance(bn, bd, m->voxel_size);
      if (m->kind == 0 && !inside_dense(m, k)) { status = ORC_RAY_MISS_EXIT; break; }
      block_of(k, nb);
      if (nb[0] != blk[0] || nb[1] != blk[1] || nb[2] != blk[2]) {
        blocks += 1;
        for (int a = 0; a < 3; ++a) blk[a] = nb[a];
      }
      if (occupied(m, k)) { status = ORC_RAY_HIT; break; }
    }
  }
  memset(out, 0, sizeof(*out));
  for (int a = 0; a < 3; ++a) out->voxel[a] = (int32_t)k[a];
  out->steps = steps;
  out->d = d;
  out->status = (uint8_t)status;
  out->blocks = (uint16_t)blocks;
  return 0;
}

/* ------------------------------------------------------------------ obstacle policy (Sec. III-C)
 * r: unit vector pointing away from the obstacle; d: distance to it.
 * f = f_rep + f_damp with f_rep = eta_rep exp(-d/nu_rep) r and
 * f_damp = eta_damp / (d/nu_damp + eps) * g_obs, g_obs = max(0, -xdot.r)^2 r.
 * A = w_r(d) s(f_damp) s(f_damp)^T with s(v) = v / (|v| + c log(1 + exp(-2 c |v|))).
 * w_r(d) = d^2/r^2 - 2d/r + 1 as printed (w_mode 0), or the cubic 1 - 3x^2 + 2x^3,
 * x = d/r, that the text describes (w_mode 1); 0 outside the radius.
 * active: the caller's FP32 decision that -xdot.r > 0 (else g_obs = 0);
 * in_radius: the caller's decision that d < r (else w = 0). */
void orc_ray_policy(const orc_params_t* p, const double r[3], double d, const double xdot[3],
                    int active, int in_radius, double f[3], double A[6]) {
  double frep = p->eta_rep * exp(-d / p->nu_rep);
  double xr = xdot[0] * r[0] + xdot[1] * r[1] + xdot[2] * r[2];
  double m = active ? xr * xr : 0.0;              /* max(0, -xdot.r)^2 */
  double kd = p->eta_damp / (d / p->nu_damp + p->eps);
  double fdamp[3];
  for (int a = 0; a < 3; ++a) {
    fdamp[a] = kd * m * r[a];
    f[a] = frep * r[a] + fdamp[a];
  }
  /* w_r(d): the printed d^2/r^2 - 2d/r + 1, or the cubic 1 - 3x^2 + 2x^3 (x = d/r), each
   * evaluated in its factored form y^2 and y^2 (1 + 2x) with y = 1 - x = (r - d) / r: the
   * same polynomials, whose FP64 values keep their relative accuracy near d = r (r - d is
   * exact there), where the expanded sums cancel (1e-5 relative error at 1 - d/r = 5e-6). */
  double w = 0.0;
  if (in_radius) {
    double x = d / p->r;
    double y = (p->r - d) / p->r;
    w = p->w_mode == 0 ? y * y : y * y * (1.0 + 2.0 * x);
  }
  double z = sqrt(fdamp[0] * fdamp[0] + fdamp[1] * fdamp[1] + fdamp[2] * fdamp[2]);
  double h = z + p->c * log1p(exp(-2.0 * p->c * z));
  double s[3] = {fdamp[0] / h, fdamp[1] / h, fdamp[2] / h};
  A[0] = w * s[0] * s[0];
  A[1] = w * s[0] * s[1];
  A[2] = w * s[0] * s[2];
  A[3] = w * s[1] * s[1];
  A[4] = w * s[1] * s[2];
  A[5] = w * s[2] * s[2];
}

/* FP32 decision shared in specification with the CUDA side: u points towards the
 * obstacle (u = -r), and the ray is active (g_obs != 0) iff xdot . u > 0, evaluated as
 * fma(vz, uz, fma(vy, uy, vx * ux)) with v = RN32(xdot). */
int orc_active32(const double xdot[3], const float u[3]) {
  float vx = (float)xdot[0], vy = (float)xdot[1], vz = (float)xdot[2];
  float dot = fmaf(vz, u[2], fmaf(vy, u[1], vx * u[0]));
  return dot > 0.0f;
}

/* ------------------------------------------------------------------ pseudo-inverse (Eq. 1)
 * Symmetric 3x3 pseudo-inverse through an eigen-decomposition by the cyclic Jacobi
 * method (rotations that zero one off-diagonal entry at a time; Golub and Van Loan,
 * Matrix Computations, Sec. 8.5).  Eigenvalues <= 1e-12 * lambda_max (and all of them
 * when lambda_max <= 1e-300) count as zero. */
void orc_pinv3(const double S[6], double Pinv[6], double eig[3], uint32_t* rank) {
  double a[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    if (off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* a <- J^T a J with J the rotation in the (p,q) plane */
        for (int k = 0; k < 3; ++k) {
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
    }
    double diag = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
    double off2 = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    if (off2 <= 1e-300 || off2 <= diag * 1e-18) break;
  }
  int idx[3] = {0, 1, 2};
  double lam[3] = {a[0][0], a[1][1], a[2][2]};
  for (int i = 0; i < 3; ++i)            /* sort ascending */
    for (int j = i + 1; j < 3; ++j)
      if (lam[idx[j]] < lam[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  double lmax = lam[idx[2]];
  for (int i = 0; i < 6; ++i) Pinv[i] = 0.0;
  uint32_t rk = 0;
  for (int i = 0; i < 3; ++i) {
    int e = idx[i];
    eig[i] = lam[e];
    if (!(lmax > 1e-300) || lam[e] <= 1e-12 * lmax) continue;
    rk += 1;
    double inv = 1.0 / lam[e];
    double u0 = v[0][e], u1 = v[1][e], u2 = v[2][e];
    Pinv[0] += inv * u0 * u0;
    Pinv[1] += inv * u0 * u1;
    Pinv[2] += inv * u0 * u2;
    Pinv[3] += inv * u1 * u1;
    Pinv[4] += inv * u1 * u2;
    Pinv[5] += inv * u2 * u2;
  }
  *rank = rk;
}

/* ------------------------------------------------------------------ summation and resolve */
typedef struct { double s[9], c[9]; } acc9_t;

/* Kahan-Babuska (Neumaier) compensated summation, in ray order. */
static void acc_add(acc9_t* acc, const double v[9]) {
  for (int k = 0; k < 9; ++k) {
    double t = acc->s[k] + v[k];
    if (fabs(acc->s[k]) >= fabs(v[k])) acc->c[k] += (acc->s[k] - t) + v[k];
    else acc->c[k] += (v[k] - t) + acc->s[k];
    acc->s[k] = t;
  }
}

static void resolve(const acc9_t* acc, orc_result_t* out) {
  for (int k = 0; k < 6; ++k) out->sumA[k] = acc->s[k] + acc->c[k];
  for (int k = 0; k < 3; ++k) out->sumAf[k] = acc->s[6 + k] + acc->c[6 + k];
  double P[6];
  orc_pinv3(out->sumA, P, out->eig, &out->rank);
  const double* b = out->sumAf;
  out->f[0] = P[0] * b[0] + P[1] * b[1] + P[2] * b[2];
  out->f[1] = P[1] * b[0] + P[3] * b[1] + P[4] * b[2];
  out->f[2] = P[2] * b[0] + P[4] * b[1] + P[5] * b[2];
}

/* A f for symmetric A (6 unique entries). */
static void sym_mul(const double A[6], const double f[3], double out[3]) {
  out[0] = A[0] * f[0] + A[1] * f[1] + A[2] * f[2];
  out[1] = A[1] * f[0] + A[3] * f[1] + A[4] * f[2];
  out[2] = A[2] * f[0] + A[4] * f[1] + A[5] * f[2];
}

/* ------------------------------------------------------------------ ray policy (Eq. raytracing_policy)
 * Ray j (0 <= j < n_rays) uses Halton index j + halton_offset.  Each ray is marched
 * from the quantised robot position; a HIT contributes A_obs(r = -dir, d) and
 * A_obs f_obs; a miss (range or map exit) contributes nothing.  per_ray (nullable)
 * receives f (3) then A (6) per ray, zeros for misses. */
int orc_raycast_eval(const orc_map_t* m, const double x[3], const double xdot[3],
                     uint32_t n_rays, const orc_params_t* p, orc_result_t* out,
                     orc_hit_t* hits, double* per_ray) {
  double vs = m->voxel_size;
  int64_t P[3];
  for (int a = 0; a < 3; ++a) P[a] = orc_quantize_pos(x[a], m->kind == 0 ? m->origin[a] : 0.0, vs);
  int64_t R_fx = orc_range_fx(p->max_range, vs);
  acc9_t acc;
  memset(&acc, 0, sizeof(acc));
  memset(out, 0, sizeof(*out));
  out->n_rays = n_rays;
  for (uint32_t j = 0; j < n_rays; ++j) {
    float dir[3];
    int32_t D[3];
    orc_ray_dir(j + p->halton_offset, dir);
    orc_quantize_dir(dir, D);
    orc_hit_t h;
    orc_dda(m, P, D, R_fx, &h);
    if (hits) hits[j] = h;
    double v[9] = {0};
    double f[3] = {0, 0, 0}, A[6] = {0, 0, 0, 0, 0, 0};
    if (h.status == ORC_RAY_HIT) {
      out->n_hits += 1;
      double r[3] = {-(double)dir[0], -(double)dir[1], -(double)dir[2]};
      int act = orc_active32(xdot, dir);
      int inr = (double)h.d < p->r;
      out->n_active += (uint32_t)(act && inr);
      orc_ray_policy(p, r, (double)h.d, xdot, act, inr, f, A);
      double Af[3];
      sym_mul(A, f, Af);
      for (int k = 0; k < 6; ++k) v[k] = A[k];
      for (int k = 0; k < 3; ++k) v[6 + k] = Af[k];
      acc_add(&acc, v);
    }
    if (per_ray) {
      for (int k = 0; k < 3; ++k) per_ray[9 * (size_t)j + k] = f[k];
      for (int k = 0; k < 6; ++k) per_ray[9 * (size_t)j + 3 + k] = A[k];
    }
  }
  resolve(&acc, out);
  return 0;
}

/* ------------------------------------------------------------------ LiDAR policy (Sec. III-G)
 * Each point p (FP32) is a beam's end point; with q = p - RN32(x) (FP32), the beam's
 * range is |q| and the direction away from the obstacle is r = -q/|q|.  Points that are
 * not finite, or whose FP32 range d32 = sqrt(fma(qz,qz, fma(qy,qy, qx*qx))) is zero,
 * below min_range or above max_range, are skipped.  The activity decision uses the
 * FP32 unit vector q/d32; the radius decision d32 < r; the policy values use FP64
 * range and direction computed from q. */
int orc_scan_eval(const float* pts, uint32_t n, const double x[3], const double xdot[3],
                  const orc_params_t* p, orc_result_t* out, double* per_ray) {
  acc9_t acc;
  memset(&acc, 0, sizeof(acc));
  memset(out, 0, sizeof(*out));
  out->n_rays = n;
  float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
  for (uint32_t j = 0; j < n; ++j) {
    float q[3];
    for (int a = 0; a < 3; ++a) q[a] = pts[3 * (size_t)j + a] - xf[a];
    double f[3] = {0, 0, 0}, A[6] = {0, 0, 0, 0, 0, 0};
    int valid = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]);
    float d32 = 0.0f;
    if (valid) {
      d32 = sqrtf(fmaf(q[2], q[2], fmaf(q[1], q[1], q[0] * q[0])));
      valid = d32 > 0.0f && (double)d32 >= p->min_range && (double)d32 <= p->max_range;
    }
    if (valid) {
      out->n_hits += 1;
      float u32[3] = {q[0] / d32, q[1] / d32, q[2] / d32};
      int act = orc_active32(xdot, u32);
      int inr = (double)d32 < p->r;
      out->n_active += (uint32_t)(act && inr);
      double qd[3] = {q[0], q[1], q[2]};
      double d = sqrt(qd[0] * qd[0] + qd[1] * qd[1] + qd[2] * qd[2]);
      double r[3] = {-qd[0] / d, -qd[1] / d, -qd[2] / d};
      orc_ray_policy(p, r, d, xdot, act, inr, f, A);
      double Af[3], v[9];
      sym_mul(A, f, Af);
      for (int k = 0; k < 6; ++k) v[k] = A[k];
      for (int k = 0; k < 3; ++k) v[6 + k] = Af[k];
      acc_add(&acc, v);
    }
    if (per_ray) {
      for (int k = 0; k < 3; ++k) per_ray[9 * (size_t)j + k] = f[k];
      for (int k = 0; k < 6; ++k) per_ray[9 * (size_t)j + 3 + k] = A[k];
    }
  }
  resolve(&acc, out);
  return 0;
}

/* ------------------------------------------------------------------ attractor (Sec. III-B)
 * f_a = alpha s(goal - x) - beta xdot, s(v) = v / (|v| + c log(1 + exp(-2c|v|))). */
void orc_attractor(const double x[3], const double xdot[3], const double goal[3], double alpha,
                   double beta, double c, double fa[3]) {
  double v[3] = {goal[0] - x[0], goal[1] - x[1], goal[2] - x[2]};
  double z = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double h = z + c * log1p(exp(-2.0 * c * z));
  for (int a = 0; a < 3; ++a) fa[a] = alpha * (v[a] / h) - beta * xdot[a];
}

/* Eq. (1) over the raycasting policy and the attractor (metric I); with metric_mean the
 * ray policies' sums are divided by the ray count first (their mean). */
int orc_combined_eval(const orc_map_t* m, const double x[3], const double xdot[3],
                      uint32_t n_rays, const orc_params_t* p, const double goal[3],
                      double alpha, double beta, int metric_mean, orc_result_t* out) {
  orc_raycast_eval(m, x, xdot, n_rays, p, out, NULL, NULL);
  if (metric_mean && n_rays > 0) {
    for (int k = 0; k < 6; ++k) out->sumA[k] /= (double)n_rays;
    for (int k = 0; k < 3; ++k) out->sumAf[k] /= (double)n_rays;
  }
  double fa[3];
  orc_attractor(x, xdot, goal, alpha, beta, p->c, fa);
  out->sumA[0] += 1.0;
  out->sumA[3] += 1.0;
  out->sumA[5] += 1.0;
  for (int a = 0; a < 3; ++a) out->sumAf[a] += fa[a];
  double P[6];
  orc_pinv3(out->sumA, P, out->eig, &out->rank);
  const double* b = out->sumAf;
  out->f[0] = P[0] * b[0] + P[1] * b[1] + P[2] * b[2];
  out->f[1] = P[1] * b[0] + P[3] * b[1] + P[4] * b[2];
  out->f[2] = P[2] * b[0] + P[4] * b[1] + P[5] * b[2];
  return 0;
}

/* ------------------------------------------------------------------ closed loop (Sec. IV-A)
 * A point robot integrates the combined policy's acceleration. */
/* Semi-implicit Euler with acceleration f, path and smoothness statistics, then the
 * stopping checks (see orc_rollout_step). */
static void rollout_advance(const orc_map_t* m, const orc_rollout_params_t* rp,
                            const double goal[3], const double f_in[3], orc_rollout_t* st) {
  const double f[3] = {f_in[0], f_in[1], f_in[2]};
  double xn[3], dl = 0.0;
  for (int a = 0; a < 3; ++a) {
    st->xdot[a] = st->xdot[a] + f[a] * rp->dt;
    xn[a] = st->x[a] + st->xdot[a] * rp->dt;
    dl += (xn[a] - st->x[a]) * (xn[a] - st->x[a]);
    st->x[a] = xn[a];
  }
  st->path_length += sqrt(dl);
  st->steps += 1;
  if (rp->seg_steps && st->steps % rp->seg_steps == 0) {
    double seg[3];
    for (int a = 0; a < 3; ++a) {
      seg[a] = st->x[a] - st->seg_start[a];
      st->seg_start[a] = st->x[a];
    }
    if (st->have_prev) {
      double dot = 0, na = 0, nb = 0;
      for (int a = 0; a < 3; ++a) {
        dot += st->prev_seg[a] * seg[a];
        na += st->prev_seg[a] * st->prev_seg[a];
        nb += seg[a] * seg[a];
      }
      if (na > 0.0 && nb > 0.0) {
        double cs = dot / (sqrt(na) * sqrt(nb));
        cs = cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs);
        st->smooth_sum += 1.0 - acos(cs) / 3.14159265358979323846;
        st->smooth_n += 1;
      }
    }
    for (int a = 0; a < 3; ++a) st->prev_seg[a] = seg[a];
    st->have_prev = 1;
  }
  int64_t k[3];
  for (int a = 0; a < 3; ++a)
    k[a] = orc_quantize_pos(st->x[a], m->kind == 0 ? m->origin[a] : 0.0, m->voxel_size) >> 16;
  double dg = 0.0;
  for (int a = 0; a < 3; ++a) dg += (st->x[a] - goal[a]) * (st->x[a] - goal[a]);
  if (m->kind == 0 && !inside_dense(m, k)) st->status = ORC_ROLL_LEFT_MAP;
  else if (occupied(m, k)) st->status = ORC_ROLL_COLLIDED;
  else if (sqrt(dg) < rp->goal_tol) st->status = ORC_ROLL_REACHED;
  else if (st->steps >= rp->max_steps) st->status = ORC_ROLL_TIMEOUT;
}

void orc_rollout_step(const orc_map_t* m, const orc_params_t* p, const orc_rollout_params_t* rp,
                      const double goal[3], orc_rollout_t* st) {
  if (st->status != ORC_ROLL_RUNNING) return;
  orc_result_t r;
  orc_combined_eval(m, st->x, st->xdot, rp->n_rays, p, goal, rp->alpha, rp->beta,
                    (int)rp->metric_mean, &r);
  rollout_advance(m, rp, goal, r.f, st);
}

/* ------------------------------------------------------------------ ESDF policy (Sec. III-D) */
static double sign_of(double v) { return v < 0.0 ? -1.0 : 1.0; }

static double prim_sdf(const orc_prim_t* pr, const double x[3]) {
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = x[a] - pr->center[a];
  if (pr->kind == ORC_PRIM_SPHERE)
    return sqrt((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) - pr->size[0];
  double ai[3], o[3];
  for (int a = 0; a < 3; ++a) {
    ai[a] = fabs(q[a]) - pr->size[a];
    o[a] = ai[a] > 0.0 ? ai[a] : 0.0;
  }
  const double out = sqrt((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]);
  double in = ai[0] > ai[1] ? ai[0] : ai[1];
  in = in > ai[2] ? in : ai[2];
  in = in < 0.0 ? in : 0.0;
  return out + in;
}

static void prim_grad(const orc_prim_t* pr, const double x[3], double g[3]) {
  double q[3];
  for (int a = 0; a < 3; ++a) q[a] = x[a] - pr->center[a];
  if (pr->kind == ORC_PRIM_SPHERE) {
    const double L = sqrt((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]);
    for (int a = 0; a < 3; ++a) g[a] = L > 0.0 ? q[a] / L : 0.0;
    return;
  }
  double ai[3], o[3];
  for (int a = 0; a < 3; ++a) {
    ai[a] = fabs(q[a]) - pr->size[a];
    o[a] = ai[a] > 0.0 ? ai[a] : 0.0;
  }
  const double out = sqrt((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]);
  if (out > 0.0) {
    for (int a = 0; a < 3; ++a) g[a] = sign_of(q[a]) * o[a] / out;
    return;
  }
  const int k = (ai[0] >= ai[1] && ai[0] >= ai[2]) ? 0 : (ai[1] >= ai[2] ? 1 : 2);
  for (int a = 0; a < 3; ++a) g[a] = a == k ? sign_of(q[a]) : 0.0;
}

int orc_esdf_query(const orc_prim_t* prims, uint32_t n, const double x[3], double* d,
                   double grad[3]) {
  int best = -1;
  double bv = INFINITY;
  for (uint32_t i = 0; i < n; ++i) {
    const double v = prim_sdf(&prims[i], x);
    if (v < bv) {
      bv = v;
      best = (int)i;
    }
  }
  grad[0] = grad[1] = grad[2] = 0.0;
  if (best < 0) {
    *d = INFINITY;
    return -1;
  }
  *d = bv > 0.0 ? bv : 0.0;
  prim_grad(&prims[best], x, grad);
  return best;
}

void orc_esdf_eval(const orc_prim_t* prims, uint32_t n, const double x[3], const double xdot[3],
                   const orc_params_t* p, const double* goal, double alpha, double beta,
                   orc_result_t* out, double* query) {
  memset(out, 0, sizeof(*out));
  double d, r[3];
  const int idx = orc_esdf_query(prims, n, x, &d, r);
  if (query) {
    query[0] = d;
    for (int a = 0; a < 3; ++a) query[1 + a] = r[a];
  }
  double S[6] = {0, 0, 0, 0, 0, 0}, b[3] = {0, 0, 0};
  out->n_rays = 1;
  if (idx >= 0) {
    const double xr = (xdot[0] * r[0] + xdot[1] * r[1]) + xdot[2] * r[2];
    const int active = xr < 0.0, in_radius = d < p->r;
    double f[3], A[6];
    orc_ray_policy(p, r, d, xdot, active, in_radius, f, A);
    for (int k = 0; k < 6; ++k) S[k] = A[k];
    sym_mul(A, f, b);
    out->n_hits = 1;
    out->n_active = (uint32_t)(active && in_radius);
  }
  if (goal) {
    double fa[3];
    orc_attractor(x, xdot, goal, alpha, beta, p->c, fa);
    S[0] += 1.0;
    S[3] += 1.0;
    S[5] += 1.0;
    for (int a = 0; a < 3; ++a) b[a] += fa[a];
  }
  for (int k = 0; k < 6; ++k) out->sumA[k] = S[k];
  for (int k = 0; k < 3; ++k) out->sumAf[k] = b[k];
  double P[6];
  orc_pinv3(S, P, out->eig, &out->rank);
  out->f[0] = P[0] * b[0] + P[1] * b[1] + P[2] * b[2];
  out->f[1] = P[1] * b[0] + P[3] * b[1] + P[4] * b[2];
  out->f[2] = P[2] * b[0] + P[4] * b[1] + P[5] * b[2];
}

void orc_esdf_rollout_step(const orc_map_t* m, const orc_prim_t* prims, uint32_t n,
                           const orc_params_t* p, const orc_rollout_params_t* rp,
                           const double goal[3], orc_rollout_t* st) {
  if (st->status != ORC_ROLL_RUNNING) return;
  orc_result_t r;
  orc_esdf_eval(prims, n, st->x, st->xdot, p, goal, rp->alpha, rp->beta, &r, NULL);
  rollout_advance(m, rp, goal, r.f, st);
}

/* ------------------------------------------------------------------ batch helpers (tests) */
void orc_halton_batch(uint32_t n, uint32_t offset, float* u, float* v, uint32_t* num3) {
  for (uint32_t j = 0; j < n; ++j) {
    u[j] = orc_halton2(j + offset);
    v[j] = orc_halton3(j + offset);
    num3[j] = orc_halton3_numerator(j + offset);
  }
}

void orc_sincos_batch(uint32_t n, const float* v, float* c, float* s) {
  for (uint32_t j = 0; j < n; ++j) orc_sincos_turns(v[j], c + j, s + j);
}

void orc_quantize_dirs(uint32_t n, const float* dirs, int32_t* D) {
  for (uint32_t j = 0; j < n; ++j) orc_quantize_dir(dirs + 3 * (size_t)j, D + 3 * (size_t)j);
}

int orc_dda_batch(const orc_map_t* m, uint32_t n, const int64_t* P, const int32_t* D,
                  int64_t R_fx, orc_hit_t* out) {
  for (uint32_t j = 0; j < n; ++j)
    orc_dda(m, P + 3 * (size_t)j, D + 3 * (size_t)j, R_fx, out + j);
  return 0;
}
