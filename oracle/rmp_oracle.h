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

/* ------------------------------------------------------------------ ESDF policy (Sec. III-D)
 * The single-query baseline: the distance to the closest obstacle d_obs(x) and its gradient
 * stand in for a ray's d and r in the obstacle policy of Sec. III-C.  The ESDF is the exact
 * Euclidean signed distance of a union of primitives (spheres, boxes): the minimum over
 * primitives, the first minimum on ties; d = max(sdf, 0) (inside an obstacle the distance
 * to the closest obstacle is 0); the gradient is that of the minimising primitive's
 * distance (a unit vector pointing away from it).  Evaluation order (FP64, one rounding
 * per operation, no fused operations) is part of the definition, since the GPU side
 * reproduces d and the gradient bit for bit:
 *   sphere (centre c, radius rho): q = x - c, L = sqrt((q0 q0 + q1 q1) + q2 q2),
 *     sdf = L - rho, gradient q_a / L (0 if L = 0);
 *   box (centre c, half-extents h): q = x - c, a_i = |q_i| - h_i, o_i = max(a_i, 0),
 *     out = sqrt((o0 o0 + o1 o1) + o2 o2), in = min(max(max(a0, a1), a2), 0),
 *     sdf = out + in; gradient: out > 0: sign(q_i) o_i / out; else sign(q_k) e_k for
 *     k = argmax a_i (lowest index on ties); sign(0) = +1. */
enum { ORC_PRIM_SPHERE = 0, ORC_PRIM_BOX = 1 };

typedef struct {
  uint32_t kind, reserved;
  double center[3];
  double size[3];           /* sphere: size[0] = radius; box: half-extents */
} orc_prim_t;

/* d (+inf with no primitives) and the gradient at x; returns the minimising primitive's
 * index, -1 with none. */
int orc_esdf_query(const orc_prim_t* prims, uint32_t n, const double x[3], double* d,
                   double grad[3]);

/* The ESDF policy at (x, xdot): the obstacle policy with d = d_obs(x), r = its gradient,
 * active iff xdot . r < 0 and in radius iff d < r_w (both FP64); with a goal (non-null) the
 * attractor is combined by Eq. (1): f = (A_obs + I)^+ (A_obs f_obs + f_a), else
 * f = A_obs^+ A_obs f_obs.  out->sumA / sumAf hold the metric and the metric-weighted force
 * that are resolved; n_rays = 1, n_hits = 1 if there is a primitive, n_active = 1 if the
 * policy is active and in radius.  query (nullable): d and the gradient (4 doubles). */
void orc_esdf_eval(const orc_prim_t* prims, uint32_t n, const double x[3], const double xdot[3],
                   const orc_params_t* p, const double* goal, double alpha, double beta,
                   orc_result_t* out, double* query);

/* One closed-loop step as orc_rollout_step, with the ESDF policy combined with the
 * attractor in place of the raycasting policy (the voxel map m still decides collisions). */
void orc_esdf_rollout_step(const orc_map_t* m, const orc_prim_t* prims, uint32_t n,
                           const orc_params_t* p, const orc_rollout_params_t* rp,
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
