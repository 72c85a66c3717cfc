/* rmp_oracle.h -- CPU oracle for raycast-RMP evaluation (arXiv 2301.08068).
 *
 * TEST INFRASTRUCTURE, not part of the library.  A plain, slow, single-threaded C
 * statement of what the GPU path computes, used only by the test suite, the smoke
 * check and the benchmark's CPU-baseline leg to check and time the CUDA library.  It
 * shares no code with the library: neither includes nor links the other.
 *
 * All policy arithmetic is FP64.  The pieces the method defines bit-for-bit (the
 * Halton ray directions, the fixed-point DDA and its hit distance, and the FP32
 * decisions that gate a ray's contribution) follow one written specification that
 * the CUDA side implements separately.
 */
#ifndef RMP_ORACLE_H
#define RMP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_RAY_HIT = 1, ORC_RAY_MISS_RANGE = 2, ORC_RAY_MISS_EXIT = 3 };

typedef struct {
  double eta_rep, nu_rep, eta_damp, nu_damp, r, c, eps, max_range, min_range;
  uint32_t halton_offset, w_mode;
} orc_params_t;

typedef struct {
  int32_t voxel[3];
  uint32_t steps;
  float d;
  uint8_t status;
  uint8_t pad;
  uint16_t blocks;  /* distinct 8^3 blocks whose occupancy was tested */
} orc_hit_t;

typedef struct {
  double sumA[6];  /* xx xy xz yy yz zz */
  double sumAf[3];
  double f[3];     /* (sum A)^+ (sum A f) */
  double eig[3];   /* eigenvalues of sum A, ascending */
  uint32_t n_rays, n_hits, n_active, rank;
} orc_result_t;

typedef struct {
  int kind;                 /* 0 dense uint8, 1 hashed TSDF blocks of 8^3 */
  double voxel_size;
  double origin[3];         /* dense only */
  int32_t dims[3];          /* dense only */
  const uint8_t* occ;       /* dense: x fastest */
  uint32_t n_blocks;        /* hashed */
  const int32_t* keys;      /* hashed: n x 3 block coordinates */
  const float* tsdf;        /* hashed: n x 512, voxel lx + 8 ly + 64 lz */
  uint32_t* sorted;         /* oracle-private: block indices sorted by key */
} orc_map_t;

int orc_map_prepare(orc_map_t* m);
void orc_map_free(orc_map_t* m);

float orc_halton2(uint32_t i);
uint32_t orc_halton3_numerator(uint32_t i);
float orc_halton3(uint32_t i);
void orc_sincos_turns(float v, float* c, float* s);
void orc_ray_dir(uint32_t i, float dir[3]);
void orc_ray_dirs(uint32_t n, uint32_t offset, float* dirs);
void orc_quantize_dir(const float dir[3], int32_t D[3]);
int64_t orc_quantize_pos(double x, double origin, double vs);
int64_t orc_range_fx(double max_range, double vs);

int orc_dda(const orc_map_t* m, const int64_t P[3], const int32_t D[3], int64_t R_fx,
            orc_hit_t* out);

void orc_ray_policy(const orc_params_t* p, const double r[3], double d, const double xdot[3],
                    int active, int in_radius, double f[3], double A[6]);
int orc_active32(const double xdot[3], const float u[3]);

void orc_pinv3(const double S[6], double Pinv[6], double eig[3], uint32_t* rank);

int orc_raycast_eval(const orc_map_t* m, const double x[3], const double xdot[3],
                     uint32_t n_rays, const orc_params_t* p, orc_result_t* out,
                     orc_hit_t* hits, double* per_ray);

int orc_scan_eval(const float* pts, uint32_t n, const double x[3], const double xdot[3],
                  const orc_params_t* p, orc_result_t* out, double* per_ray);

/* Attractor policy (Sec. III-B, Eq. attractorPolicy): f_a = alpha s(goal - x) - beta xdot,
 * A_a = I, with the soft normalisation s of Eq. softmax (parameter c). */
void orc_attractor(const double x[3], const double xdot[3], const double goal[3], double alpha,
                   double beta, double c, double fa[3]);

/* Raycasting policy combined with the attractor by Eq. (1):
 * f_c = (M + I)^+ (M f_ray + f_a) with M f_ray = sum A f and M = sum A (Eq.
 * raytracing_policy as printed) or, with metric_mean, M = sum A / n_rays and
 * M f_ray = sum A f / n_rays (the mean the text describes).  out->sumA / sumAf hold the
 * combined sums (M + I, M f_ray + f_a), out->eig and out->rank describe M + I. */
int orc_combined_eval(const orc_map_t* m, const double x[3], const double xdot[3],
                      uint32_t n_rays, const orc_params_t* p, const double goal[3],
                      double alpha, double beta, int metric_mean, orc_result_t* out);

enum { ORC_ROLL_RUNNING = 0, ORC_ROLL_REACHED = 1, ORC_ROLL_COLLIDED = 2, ORC_ROLL_TIMEOUT = 3,
       ORC_ROLL_LEFT_MAP = 4 };

typedef struct {
  double alpha, beta, dt, goal_tol;
  uint32_t max_steps, seg_steps, n_rays, metric_mean;
} orc_rollout_params_t;

typedef struct {
  double x[3], xdot[3];
  double path_length;    /* sum of the step lengths |x' - x| */
  double smooth_sum;     /* sum of 1 - acos(cos angle)/pi over consecutive segments */
  double seg_start[3], prev_seg[3];
  uint32_t status, steps, smooth_n, have_prev;
} orc_rollout_t;

/* One closed-loop control step of a point robot: f = f_c(x, xdot); then
 * xdot' = xdot + f dt, x' = x + xdot' dt (semi-implicit Euler).  Then, in this order:
 * left the dense grid -> LEFT_MAP; the voxel holding x' is occupied -> COLLIDED;
 * |x' - goal| < goal_tol -> REACHED; steps == max_steps -> TIMEOUT.  Every seg_steps
 * steps the displacement since the last segment end is a segment; consecutive segments
 * A, B add 1 - acos(A.B / (|A||B|)) / pi to smooth_sum.  No-op unless RUNNING.  A new
 * state is all zero except x, xdot and seg_start = x. */
void orc_rollout_step(const orc_map_t* m, const orc_params_t* p, const orc_rollout_params_t* rp,
                      const double goal[3], orc_rollout_t* st);

/* batch helpers used by the tests */
void orc_halton_batch(uint32_t n, uint32_t offset, float* u, float* v, uint32_t* num3);
void orc_sincos_batch(uint32_t n, const float* v, float* c, float* s);
void orc_quantize_dirs(uint32_t n, const float* dirs, int32_t* D);
int orc_dda_batch(const orc_map_t* m, uint32_t n, const int64_t* P, const int32_t* D,
                  int64_t R_fx, orc_hit_t* out);

#ifdef __cplusplus
}
#endif
#endif
