/* rmp.h -- C ABI of librmp.so: raycast Riemannian Motion Policy evaluation on one GPU.
 *
 * Method: Pantic, Meijer et al., "Obstacle avoidance using raycasting and Riemannian
 * Motion Policies at kHz rates for MAVs" (arXiv 2301.08068).  From one robot state
 * (x, xdot), N rays with Halton directions (Sec. III-E, Eq. halton) are marched through a
 * voxel map (Sec. III-F), each ray yields an obstacle policy (f_i, A_i) (Sec. III-C), the
 * policies are summed and resolved by Eq. (1): f = (sum A_i)^+ sum A_i f_i (Sec. III-A,
 * Eq. raytracing_policy).  The LiDAR variant (Sec. III-G) takes a scan's points as the
 * rays' end points.
 *
 * Conventions for every call:
 *  - Every call returns an int status (RMP_OK = 0, else an RMP_ERR_* code); no C++
 *    exception crosses this boundary.  Out-parameters are written only on RMP_OK.
 *  - Pointers named *_dev are device pointers on the context's device; all others are
 *    host pointers.  The caller keeps ownership of every buffer it passes in; the
 *    context owns what it allocates (maps, internal scratch, pinned staging).
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy default stream).
 *    Synchronous calls return after their stream has finished their work; _async calls
 *    only enqueue work and never synchronise.
 *  - A context may be used from several host threads; synchronous calls on one context
 *    serialise on an internal lock.
 *  - Arithmetic: FP32 march, direction and per-ray policy; the cross-ray reduction is a
 *    compensated FP32 sum (default) or FP64; the 3x3 pseudo-inverse resolve is FP64.
 */
#ifndef RMP_H
#define RMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RMP_ABI_VERSION 1

/* ------------------------------------------------------------------ status codes */
#define RMP_OK 0
#define RMP_ERR_INVALID_ARG 1   /* a pointer, size, parameter or map is invalid        */
#define RMP_ERR_NO_MEMORY 2     /* device or pinned host allocation failed             */
#define RMP_ERR_CUDA 3          /* a CUDA runtime call or kernel launch failed         */
#define RMP_ERR_TIMEOUT 4       /* a bounded wait expired (serving, device waits)      */
#define RMP_ERR_BUSY 5          /* no free slot / over the memory budget (serving)     */
#define RMP_ERR_UNKNOWN_MAP 6   /* map id not registered in this context               */
#define RMP_ERR_NOT_READY 7     /* polled work has not completed yet (serving)         */

/* Per-ray march outcome (rmp_ray_hit_t.status). */
#define RMP_RAY_HIT 1           /* entered an occupied voxel                           */
#define RMP_RAY_MISS_RANGE 2    /* next voxel's entry distance exceeds max_range       */
#define RMP_RAY_MISS_EXIT 3     /* left the dense grid (dense maps only)               */

typedef struct rmp_ctx rmp_ctx;
typedef void* rmp_stream_t;

/* ------------------------------------------------------------------ parameters
 * Obstacle-policy tuning of Sec. III-C / Table I plus this library's settings.
 *  eta_rep, nu_rep     repulsive gain and length scale:  f_rep = eta_rep exp(-d/nu_rep) r
 *  eta_damp, nu_damp   damping gain and length scale:
 *                      f_damp = eta_damp / (d/nu_damp + eps) * max(0, -xdot.r)^2 r
 *  r                   policy radius of w_r (metres)
 *  c                   soft-normalisation parameter of s(v) (Eq. softmax)
 *  eps                 the paper's 0 < eps << 1 (no value given; preset 1e-3)
 *  max_range           rays: march limit in metres (<= 16384 voxels); scans: points
 *                      farther than this are ignored
 *  min_range           scans only: points nearer than this are ignored (vehicle body)
 *  halton_offset       ray j uses Halton index j + halton_offset (preset 1; 0 adds the
 *                      degenerate pole ray H(0) = 0 of the paper's i = 0)
 *  w_mode              0: w_r(d) = d^2/r^2 - 2d/r + 1 as printed; 1: the cubic spline
 *                      1 - 3(d/r)^2 + 2(d/r)^3 the text describes; both 0 for d >= r
 *  reduce_mode         RMP_REDUCE_KAHAN32 (compensated FP32) or RMP_REDUCE_FP64
 *  flags               must be 0 */
typedef struct {
  double eta_rep, nu_rep, eta_damp, nu_damp, r, c, eps;
  double max_range, min_range;
  uint32_t halton_offset, w_mode, reduce_mode, flags;
} rmp_params_t;

#define RMP_PRESET_STATIC_MAP 0 /* Table I "Static Map" column, max_range 10 m        */
#define RMP_PRESET_LIDAR 1      /* Table I "LiDAR" column, max_range 30 m, min 0.2 m   */
#define RMP_REDUCE_KAHAN32 0
#define RMP_REDUCE_FP64 1

/* ------------------------------------------------------------------ results
 * Result of one evaluation (Eq. 1 / Eq. raytracing_policy).  A and Af hold sum_i A_i
 * (6 unique entries xx xy xz yy yz zz) and sum_i A_i f_i; f = A^+ Af; eig are A's
 * eigenvalues in ascending order; rank counts eigenvalues above 1e-12 * the largest.
 * n_rays: rays (or points) evaluated; n_hits: rays that hit (points that were valid);
 * n_active: hits with a nonzero metric (moving towards the obstacle, d < r).
 * status: RMP_OK, or RMP_ERR_INVALID_ARG when the device-side state was unusable
 * (non-finite or out of the map's coordinate range) -- then all sums are zero. */
typedef struct {
  double f[3];
  double A[6];
  double Af[3];
  double eig[3];
  uint32_t n_rays, n_hits, n_active, rank;
  int32_t status;
  uint32_t reserved;
} rmp_result_t; /* 144 bytes */

/* Per-ray march record: the last voxel the ray entered (global voxel index), the
 * number of voxel steps to it (= its L1 distance from the start voxel), its entry
 * distance d in metres along the ray (0 for the start voxel), the outcome, and the
 * number of distinct 8^3-aligned blocks whose occupancy the march looked up. */
typedef struct {
  int32_t voxel[3];
  uint32_t steps;
  float d;
  uint8_t status;
  uint8_t pad;
  uint16_t blocks;
} rmp_ray_hit_t; /* 24 bytes */

/* ------------------------------------------------------------------ maps
 * RMP_MAP_DENSE_U8: dims[0] x dims[1] x dims[2] uint8 voxels, x fastest; nonzero =
 *   occupied.  Voxel (i,j,k) covers origin + [i,i+1) x [j,j+1) x [k,k+1) voxel sizes.
 *   Rays that leave the grid end with RMP_RAY_MISS_EXIT.
 * RMP_MAP_HASHED_TSDF: n_blocks blocks of 8^3 float TSDF values, voxblox-style and
 *   world-anchored (voxel k covers [k, k+1) voxel sizes; origin is ignored).
 *   block_keys: n_blocks x 3 int32 block coordinates (|key| < 2^20, no duplicates);
 *   tsdf: n_blocks x 512 floats, voxel lx + 8 ly + 64 lz of each block.  A voxel is
 *   occupied iff its block exists and its TSDF value is <= 0; missing blocks are free.
 * data_on_device: 0 = occ/block_keys/tsdf are host pointers, 1 = device pointers.
 * The library copies what it needs; the caller's buffers may be freed after upload. */
#define RMP_MAP_DENSE_U8 0
#define RMP_MAP_HASHED_TSDF 1

typedef struct {
  int32_t kind;
  int32_t data_on_device;
  double voxel_size;
  double origin[3];
  int32_t dims[3];
  uint32_t n_blocks;
  const uint8_t* occ;
  const int32_t* block_keys;
  const float* tsdf;
} rmp_map_desc_t;

typedef struct {
  int32_t kind;
  uint32_t n_bricks;        /* 8^3 occupancy bricks held on the device */
  uint32_t hash_capacity;   /* hash layout: table entries (power of two); else 0 */
  uint32_t layout;          /* 0: grid (bricks over the bounding box of occupied blocks plus a
                               1-bit block bitmap); 1: hash table of blocks */
  uint64_t device_bytes;    /* device memory held by the map */
} rmp_map_info_t;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  *out receives the handle. */
int rmp_ctx_create(rmp_ctx** out, int device);

/* Destroy a context and free every map and buffer it owns.  No work of this context
 * may still be running. */
int rmp_ctx_destroy(rmp_ctx* ctx);

/* Static description of a status code (never NULL). */
const char* rmp_status_string(int status);

/* Fill *out with a parameter preset (Table I). */
int rmp_params_preset(int preset, rmp_params_t* out);

/* Upload a map (Sec. III-F: the map lives in GPU memory, shared by all evaluations).
 * Work is enqueued on `stream` and completed before return.  *map_id receives a
 * context-local id.  INVALID_ARG on bad dims, keys out of range or duplicate keys. */
int rmp_map_upload(rmp_ctx* ctx, const rmp_map_desc_t* desc, rmp_stream_t stream,
                   uint32_t* map_id);

/* Free a map.  No evaluation using it may still be running. */
int rmp_map_release(rmp_ctx* ctx, uint32_t map_id);

/* Kind, layout, bricks held, hash capacity and device bytes of a map (*out: host).
 * RMP_ERR_UNKNOWN_MAP for an id not registered in this context. */
int rmp_map_info(rmp_ctx* ctx, uint32_t map_id, rmp_map_info_t* out);

/* Free-space data of a grid-layout map, for diagnostics and tests (evaluation does not need
 * it).  grid_min / grid_dim (3 int32 each, host) receive the block coordinates of the grid's
 * first brick (x, y, z; dense maps: 0) and its bricks per axis.  cells (nullable, host,
 * cells_words uint32 words, caller-owned) receives 8 words per brick in brick order
 * (x + dim_x (y + dim_y z)): the Chebyshev distance in voxels from each 2^3 cell
 * c = cx + 4 cy + 16 cz of the brick to the nearest occupied voxel, capped at 4, in bits
 * 4 (c & 7) of word c >> 3; 0 for bricks without an occupied voxel.  Synchronous.
 * RMP_ERR_INVALID_ARG for a hash-layout map, a map without cell distances (cells given),
 * or cells_words below 8 x bricks. */
int rmp_map_cell_distances(rmp_ctx* ctx, uint32_t map_id, int32_t grid_min[3],
                           int32_t grid_dim[3], uint32_t* cells, uint64_t cells_words);

/* ------------------------------------------------------------------ evaluation
 * Raycast RMP evaluation of one state (Sec. III-E, Eq. raytracing_policy, resolved by
 * Eq. 1), synchronous: runs one fused kernel on `stream` (Halton direction, exact DDA
 * march, per-ray policy, reduction, FP64 resolve) with x and xdot (3 doubles each, host)
 * carried in the launch itself, waits for it and returns the result in *out (host; the
 * kernel writes it into pinned host memory of the context).
 * n_rays in [1, 2^24 - halton_offset].  hits_dev (nullable) receives n_rays records;
 * per_ray_dev (nullable) receives n_rays x 9 floats: f_i (3) then A_i (6), zero for
 * rays that did not hit. */
int rmp_raycast_eval(rmp_ctx* ctx, uint32_t map_id, const double x[3], const double xdot[3],
                     uint32_t n_rays, const rmp_params_t* params, rmp_stream_t stream,
                     rmp_result_t* out, rmp_ray_hit_t* hits_dev, float* per_ray_dev);

/* Bytes of device scratch one in-flight _async evaluation needs (independent of the
 * ray count). */
size_t rmp_workspace_bytes(void);

/* Initialise a workspace before its first use (enqueued on `stream`): a zero header and
 * every per-CTA partial slot empty (all bytes 0xFF).  Each evaluation leaves its
 * workspace ready for the next one, so this is needed once -- and again after an
 * evaluation on it returned status RMP_ERR_TIMEOUT (a bounded device wait expired; the
 * workspace then stays marked and every evaluation on it reports RMP_ERR_TIMEOUT until
 * it is initialised again).  The synchronous calls re-initialise their own workspace. */
int rmp_workspace_init(void* workspace_dev, size_t bytes, rmp_stream_t stream);

/* Asynchronous form of rmp_raycast_eval for device-resident inputs and outputs:
 * state_dev holds x[3] then xdot[3] (doubles), the result is written to *out_dev.
 * Only enqueues one kernel; no host synchronisation, no allocation, so it may be
 * captured in a CUDA graph.  workspace_dev (>= rmp_workspace_bytes(), set up once by
 * rmp_workspace_init) must not be shared by evaluations that may run concurrently. */
int rmp_raycast_eval_async(rmp_ctx* ctx, uint32_t map_id, const double* state_dev,
                           uint32_t n_rays, const rmp_params_t* params, void* workspace_dev,
                           size_t workspace_bytes, rmp_stream_t stream, rmp_result_t* out_dev,
                           rmp_ray_hit_t* hits_dev, float* per_ray_dev);

/* LiDAR scan policy (Sec. III-G), synchronous.  points_dev: n x 3 floats (device,
 * caller-owned), each a beam's end point in the same frame as x; NaN/inf rows and
 * points whose range |p - x| is 0, below min_range or above max_range are skipped.
 * Each valid point gives d = |p - x|, r = -(p - x)/d and the obstacle policy. */
int rmp_scan_eval(rmp_ctx* ctx, const float* points_dev, uint32_t n, const double x[3],
                  const double xdot[3], const rmp_params_t* params, rmp_stream_t stream,
                  rmp_result_t* out, float* per_ray_dev);

/* Asynchronous form of rmp_scan_eval; state_dev as for rmp_raycast_eval_async. */
int rmp_scan_eval_async(rmp_ctx* ctx, const float* points_dev, uint32_t n,
                        const double* state_dev, const rmp_params_t* params,
                        void* workspace_dev, size_t workspace_bytes, rmp_stream_t stream,
                        rmp_result_t* out_dev, float* per_ray_dev);

/* ------------------------------------------------------------------ batched evaluation
 * Many independent evaluations in one launch: state b (x then xdot, 6 doubles at
 * states_dev + 6 b) casts n_rays_dev[b] rays (Halton indices halton_offset ..
 * halton_offset + n_b - 1, as rmp_raycast_eval) with the shared map and params; result b
 * goes to out_dev[b], exactly what rmp_raycast_eval computes for that state up to the
 * order of the floating-point reduction.  The paper evaluates one state per call; the
 * batch is this library's throughput form of the same computation (candidate states of
 * a planner, or many robots).  Work is cut into chunks of 32 threads that a persistent
 * grid takes from a counter, so states of any ray counts share the device evenly.
 *
 * Capacity: n_states in [1, 65536]; every n_rays_dev[b] <= max_rays, max_rays +
 * halton_offset <= 2^24.  A state with n_b > max_rays or an invalid position gets
 * status RMP_ERR_INVALID_ARG in its result (the others are unaffected); n_b = 0 gives a
 * zero result with status RMP_OK.  hits_dev / per_ray_dev (nullable): the records of
 * state b start at index b * max_rays (same layout as rmp_raycast_eval per state); for a
 * state with an error status they are not written. */

/* Bytes of device workspace a batch of n_states states of at most max_rays rays needs
 * (any tuning); 0 for out-of-range arguments.  No initialisation is needed: every launch
 * resets what it uses. */
size_t rmp_batch_workspace_bytes(uint32_t n_states, uint32_t max_rays);

/* Enqueues two kernels on `stream` (per-state set-up, then the persistent evaluation);
 * no host synchronisation and no allocation, so the call may be captured in a CUDA graph
 * and the graph replayed with new contents of states_dev / n_rays_dev.  The workspace
 * must not be shared by batches that may run concurrently. */
int rmp_raycast_eval_batch_async(rmp_ctx* ctx, uint32_t map_id, const double* states_dev,
                                 const uint32_t* n_rays_dev, uint32_t n_states,
                                 uint32_t max_rays, const rmp_params_t* params,
                                 void* workspace_dev, size_t workspace_bytes,
                                 rmp_stream_t stream, rmp_result_t* out_dev,
                                 rmp_ray_hit_t* hits_dev, float* per_ray_dev);

/* Synchronous batch with host arrays (states: 6 n_states doubles, n_rays: n_states
 * counts, out: n_states results); allocates and frees its device buffers. */
int rmp_raycast_eval_batch(rmp_ctx* ctx, uint32_t map_id, const double* states,
                           const uint32_t* n_rays, uint32_t n_states,
                           const rmp_params_t* params, rmp_stream_t stream, rmp_result_t* out);

/* Autotuner of the batch launch: times every combination of threads per CTA {64, 128,
 * 256} and segments per ray 2^{0,1,2} (rays per thread 1, 1/2, 1/4) on this batch (one
 * untimed launch, then the median of `reps` timed launches, CUDA events on `stream`;
 * synchronises), and leaves the fastest in the context's knobs.  times_ms (nullable,
 * n_times entries) receives the 9 medians in the order block-major, then segments.  The
 * workspace must be sized for the batch (rmp_batch_workspace_bytes). */
int rmp_batch_autotune(rmp_ctx* ctx, uint32_t map_id, const double* states_dev,
                       const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                       const rmp_params_t* params, void* workspace_dev, size_t workspace_bytes,
                       rmp_stream_t stream, rmp_result_t* out_dev, int reps, float* times_ms,
                       int n_times);

/* Batched evaluation without caller-provided memory (no counterpart in the paper: a
 * deployment form of rmp_raycast_eval_batch_async).  The workspace is a 4 MiB array owned
 * by the library on each device, so the call allocates nothing and needs no workspace
 * argument -- for callers that must not allocate device memory after start-up, such as a
 * control loop with a fixed memory footprint (cudaMalloc may synchronise the device and
 * has no bounded latency).  Per-ray outputs are not offered.
 * Limit: batches whose workspace (rmp_batch_workspace_bytes(n_states, max_rays)) exceeds
 * 4 MiB are rejected with RMP_ERR_NO_MEMORY (one state of up to 406016 rays, or up to six
 * states of 65536).  Nothing in the array has to start at zero: each call's set-up kernel clears
 * what it uses.  The first call on a device looks up the array's address with that device
 * current (which can load module data), so make one call before any stream capture.
 * The address is kept for the life of the process: do not use this entry point after a
 * cudaDeviceReset of its device (the kept address would then be stale).
 * All calls on a device share the one array: calls that may overlap in time (different
 * streams without ordering, other threads) race on it and give wrong results; order them
 * on one stream or synchronise between them. */
int rmp_raycast_eval_batch_static(rmp_ctx* ctx, uint32_t map_id, const double* states_dev,
                                  const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                                  const rmp_params_t* params, rmp_stream_t stream,
                                  rmp_result_t* out_dev);

/* ------------------------------------------------------------------ attractor and closed loop
 * The raycasting policy combined with a goal attractor (Sec. III-B Eq. attractorPolicy:
 * f_a = alpha s(goal - x) - beta xdot with the soft normalisation s of Eq. softmax and
 * parameter params->c, metric I) by Eq. (1): f_c = (M + I)^+ (M f_ray + f_a), where
 * M f_ray = sum A f and M = sum A (Eq. raytracing_policy as printed; metric_mean = 0), or
 * both divided by the state's ray count (metric_mean = 1: the ray policies' mean, as the
 * text describes the combined acceleration; it keeps the attractor's weight independent of
 * the ray count).  A result's A and Af then hold the combined sums (M + I, M f_ray + f_a),
 * f = f_c and eig / rank describe M + I.  alpha, beta: Table I alpha_g, beta_g. */
int rmp_combined_eval_batch_async(rmp_ctx* ctx, uint32_t map_id, const double* states_dev,
                                  const uint32_t* n_rays_dev, uint32_t n_states,
                                  uint32_t max_rays, const rmp_params_t* params,
                                  const double* goals_dev, double alpha, double beta,
                                  uint32_t metric_mean, void* workspace_dev,
                                  size_t workspace_bytes, rmp_stream_t stream,
                                  rmp_result_t* out_dev);

/* Closed-loop rollout of point robots (the map-based experiment of Sec. IV-A): every control
 * step evaluates f_c for all running robots in one batched launch and integrates it by
 * semi-implicit Euler in FP64 (xdot' = xdot + f_c dt, x' = x + xdot' dt).  A robot stops
 * when, in this order, it leaves a dense grid (LEFT_MAP), the voxel holding it is occupied
 * (COLLIDED), it is within goal_tol of its goal (REACHED), or it has taken max_steps steps
 * (TIMEOUT); an evaluation error stops it with FAILED.  Smoothness is the mean over
 * consecutive segments (displacements over seg_steps steps) of the angular similarity
 * 1 - acos(A.B / (|A||B|)) / pi (1 = straight; the paper's path smoothness). */
#define RMP_ROLLOUT_RUNNING 0
#define RMP_ROLLOUT_REACHED 1
#define RMP_ROLLOUT_COLLIDED 2
#define RMP_ROLLOUT_TIMEOUT 3
#define RMP_ROLLOUT_LEFT_MAP 4
#define RMP_ROLLOUT_FAILED 5

typedef struct {
  double alpha, beta;      /* attractor gain and damping */
  double dt;               /* control period, s */
  double goal_tol;         /* m */
  uint32_t max_steps;
  uint32_t seg_steps;      /* smoothness segment length, steps (0: no smoothness) */
  uint32_t n_rays;         /* rays per evaluation */
  uint32_t metric_mean;    /* 0: M = sum A, 1: M = mean of the A_i (see above) */
} rmp_rollout_params_t;

typedef struct {
  double x[3], xdot[3];    /* final state */
  double path_length;      /* sum of step lengths, m */
  double smoothness;       /* mean angular similarity of consecutive segments (1 if none) */
  uint32_t status;         /* RMP_ROLLOUT_* */
  uint32_t steps;
  uint32_t smooth_segments;
  uint32_t reserved;
} rmp_rollout_result_t;

/* robots: host, 9 doubles per robot (start x, start xdot, goal).  Synchronous: allocates its
 * device buffers, runs until every robot has stopped, copies the results to out (host). */
int rmp_rollout(rmp_ctx* ctx, uint32_t map_id, const double* robots, uint32_t n_robots,
                const rmp_params_t* params, const rmp_rollout_params_t* rollout,
                rmp_stream_t stream, rmp_rollout_result_t* out);

/* ------------------------------------------------------------------ streamed LiDAR scans
 * A pipeline of `slots` (2..8) scan slots for a sensor stream (e.g. an OS-0 scan of
 * 128 x 2048 = 262144 points at 20 Hz): submitting a scan copies its points from the
 * caller's host memory (pinned, for the copy to be asynchronous; it must stay unchanged
 * until the scan's result is waited for) on a copy stream and evaluates it
 * (rmp_scan_eval semantics) on a compute stream, so the copy of one scan overlaps the
 * evaluation of the previous one.  submit waits only when the slot it reuses still holds
 * a scan in flight; wait blocks until that scan's result is in *out (host).  A ticket can
 * be waited for until its slot is reused (`slots` submits later: RMP_ERR_BUSY). */
typedef struct rmp_scan_pipeline rmp_scan_pipeline;
/* max_points (>= 1) per scan, slots in 2..8: allocates per-slot device buffers, pinned
 * staging and two streams on the context's device; *out receives the pipeline, which must
 * not outlive the context.  RMP_ERR_INVALID_ARG, RMP_ERR_NO_MEMORY. */
int rmp_scan_pipeline_create(rmp_ctx* ctx, uint32_t max_points, uint32_t slots,
                             rmp_scan_pipeline** out);
/* Waits for the scans in flight, then frees everything the pipeline holds. */
int rmp_scan_pipeline_destroy(rmp_scan_pipeline* pipeline);
/* points_host: n x 3 floats (x, y, z in the frame of x), n in [1, max_points]; x, xdot: host,
 * 3 doubles each.  *ticket identifies the scan.  RMP_ERR_INVALID_ARG for bad arguments or
 * parameters (as rmp_scan_eval), RMP_ERR_CUDA if a copy or launch fails. */
int rmp_scan_pipeline_submit(rmp_scan_pipeline* pipeline, const float* points_host, uint32_t n,
                             const double x[3], const double xdot[3], const rmp_params_t* params,
                             uint64_t* ticket);
/* Blocks until the ticket's scan is evaluated and writes its result to *out (host).
 * RMP_ERR_INVALID_ARG for a ticket never issued, RMP_ERR_BUSY once its slot was reused. */
int rmp_scan_pipeline_wait(rmp_scan_pipeline* pipeline, uint64_t ticket, rmp_result_t* out);

/* ------------------------------------------------------------------ request server
 * Continuous batching of single-state requests (a serving layer over the batched
 * evaluation; the paper evaluates one state per control step and has no counterpart).
 * Requests are submitted from any thread and complete asynchronously; a worker thread
 * keeps up to `slots` batches in flight on separate CUDA streams, admitting the oldest
 * pending request together with later pending ones of the same map and params (up to
 * max_batch_states) whenever a slot and enough of the device-memory budget are free.
 * Batches in flight overlap on the device.  Each request's result is what
 * rmp_raycast_eval returns for it, up to the order of the floating-point reduction.
 * A request whose batch alone exceeds the budget completes with RMP_ERR_NO_MEMORY; a
 * parameter or map error, or a CUDA error, completes the batch's requests with that
 * status.  Each result is delivered once (poll or wait). */
typedef struct rmp_server rmp_server;

typedef struct {
  uint32_t slots;              /* batches in flight at most (streams), 1..16 */
  uint32_t max_batch_states;   /* requests per batch, 1..65536 */
  uint32_t max_rays;           /* largest accepted request */
  uint32_t reserved;
  uint64_t mem_budget_bytes;   /* device memory for all batches in flight (allocated once) */
} rmp_server_config_t;

typedef struct {
  uint64_t submitted, completed, rejected;   /* rejected: completed with an error status */
  uint64_t batches, batched_states;          /* batches launched, requests in them */
  uint64_t pending;                          /* waiting for admission now */
  uint64_t max_inflight;                     /* most batches in flight at once */
  uint64_t mem_high_water;                   /* most budget bytes in use at once */
} rmp_server_stats_t;

/* Defaults: 4 slots, 256 states per batch, 262144 rays, 1 GiB. */
int rmp_server_config_default(rmp_server_config_t* cfg);
/* Start a server on the context's device (allocates the budget, streams, pinned staging
 * and the worker thread).  The context must outlive the server. */
int rmp_server_create(rmp_ctx* ctx, const rmp_server_config_t* cfg, rmp_server** out);
/* Finish every submitted request, then stop and free everything. */
int rmp_server_destroy(rmp_server* server);
/* Queue one evaluation (x, xdot: host, 3 doubles each; n_rays in [1, max_rays]);
 * *ticket identifies it.  Never blocks on the device. */
int rmp_server_submit(rmp_server* server, uint32_t map_id, const double x[3],
                      const double xdot[3], uint32_t n_rays, const rmp_params_t* params,
                      uint64_t* ticket);
/* RMP_OK and the result (and its submit-to-completion latency in seconds, nullable) if
 * done, which collects it; RMP_ERR_NOT_READY if not yet; RMP_ERR_INVALID_ARG for a ticket
 * never issued or already collected. */
int rmp_server_poll(rmp_server* server, uint64_t ticket, rmp_result_t* out, double* latency_s);
/* Like poll, but waits up to timeout_ms; RMP_ERR_TIMEOUT if the result is not there then;
 * RMP_ERR_INVALID_ARG for a ticket never issued or collected (also while waiting). */
int rmp_server_wait(rmp_server* server, uint64_t ticket, uint32_t timeout_ms, rmp_result_t* out,
                    double* latency_s);
/* Counters since the server started (*out: host). */
int rmp_server_stats(rmp_server* server, rmp_server_stats_t* out);

/* ------------------------------------------------------------------ ESDF policy (Sec. III-D)
 * The paper's single-query baseline: an ESDF gives the distance d_obs(x) to the closest
 * obstacle and its gradient, which stand in for one ray's d and r in the obstacle policy
 * of Sec. III-C; combined with the goal attractor by Eq. (1) it is a simple local planner,
 * the comparison for the raycasting policy.  The ESDF here is the exact Euclidean signed
 * distance of a union of primitives (spheres, boxes -- the seeded scenes the maps are built
 * from), kept on the device: d = max(0, min over primitives of their signed distance), the
 * first minimum on ties; the gradient is that of the minimising primitive's distance (a
 * unit vector pointing away from it; inside a box, the normal of its nearest face, the
 * lowest axis on ties).  Everything is FP64; d and the gradient are reproduced bit for bit
 * by a fixed operation order: sphere (centre c, radius rho): q = x - c,
 * L = sqrt((q0 q0 + q1 q1) + q2 q2), sdf = L - rho, gradient q / L (0 at the centre); box
 * (centre c, half-extents h): a_i = |x_i - c_i| - h_i, o_i = max(a_i, 0),
 * out = sqrt((o0 o0 + o1 o1) + o2 o2), sdf = out + min(max(max(a0, a1), a2), 0),
 * gradient sign(x_i - c_i) o_i / out when out > 0 (sign(0) = +1). */
typedef struct {
  uint32_t kind;            /* RMP_PRIM_SPHERE or RMP_PRIM_BOX */
  uint32_t reserved;        /* 0 */
  double center[3];
  double size[3];           /* sphere: size[0] = radius (others ignored); box: half-extents */
} rmp_primitive_t;
#define RMP_PRIM_SPHERE 0
#define RMP_PRIM_BOX 1

/* Copy n primitives (host; n in [0, 2^20], finite, sizes > 0) to the device as an ESDF;
 * *esdf_id names it (ids are shared with maps, never equal to a map's).  Synchronous. */
int rmp_esdf_upload(rmp_ctx* ctx, const rmp_primitive_t* prims, uint32_t n, uint32_t* esdf_id);
int rmp_esdf_release(rmp_ctx* ctx, uint32_t esdf_id);

/* The ESDF policy for n_states states (states_dev: x then xdot, 6 doubles each).  Per state:
 * d, r from the ESDF; active iff xdot . r < 0 and in radius iff d < params->r (both FP64);
 * f_obs, A_obs as for one ray (Sec. III-C, FP64); with goals_dev (3 doubles per state,
 * nullable) the attractor f_a = alpha s(goal - x) - beta xdot (metric I) is combined by
 * Eq. (1): out.f = (A_obs + I)^+ (A_obs f_obs + f_a), out.A / out.Af the combined sums;
 * without goals out.f = A_obs^+ A_obs f_obs.  out.n_rays = 1, n_hits = 1 if the ESDF has a
 * primitive, n_active = 1 if the policy is active and in radius; a state with a non-finite
 * component gets RMP_ERR_INVALID_ARG in its status.  query_dev (nullable): d and the
 * gradient per state (4 doubles; d = +inf with no primitive).  One warp per state, one
 * kernel on `stream`, no allocation; the result is written to out_dev[n_states]. */
int rmp_esdf_eval_async(rmp_ctx* ctx, uint32_t esdf_id, const double* states_dev,
                        const double* goals_dev, uint32_t n_states, const rmp_params_t* params,
                        double alpha, double beta, rmp_stream_t stream, rmp_result_t* out_dev,
                        double* query_dev);

/* Closed loop with the ESDF policy in place of the raycasting policy: as rmp_rollout (same
 * robots layout, integrator, stopping rules and statistics; collisions from the voxel map
 * map_id), each control step evaluating the ESDF policy combined with the attractor
 * (rp->alpha, rp->beta; rp->n_rays and rp->metric_mean are not used). */
int rmp_rollout_esdf(rmp_ctx* ctx, uint32_t map_id, uint32_t esdf_id, const double* robots,
                     uint32_t n_robots, const rmp_params_t* params,
                     const rmp_rollout_params_t* rp, rmp_stream_t stream,
                     rmp_rollout_result_t* out);

/* ------------------------------------------------------------------ diagnostics
 * L2 read bandwidth probe (measurement support, no counterpart in the paper): reads the
 * `bytes` at buf_dev (a multiple of 16, 16-byte aligned; sized to stay resident in L2,
 * e.g. 32 MiB) `passes` times with 16-byte loads that bypass L1, on every SM, and XORs
 * them into checksum_dev[0..(grid - 1)] (uint64, grid = SMs x 4 entries; keeps the loads
 * live).  Enqueues one kernel on `stream`; the caller times it (bytes x passes / time). */
int rmp_probe_l2_read(rmp_ctx* ctx, const void* buf_dev, size_t bytes, uint32_t passes,
                      rmp_stream_t stream, uint64_t* checksum_dev);

/* ------------------------------------------------------------------ launch tuning
 * Knobs of the evaluation kernels (per context; picked by the batch autotuner, settable by
 * hand).  They change the launch shape only: results are identical up to the order of
 * the floating-point reduction, hit records are identical.
 *  RMP_TUNE_BLOCK        threads per CTA: 64, 128 or 256, or 0 (default) automatic: for
 *                        one state, 256 when the launch fits in one wave of 256-thread CTAs,
 *                        else 128; scans 256; batches 128
 *  RMP_TUNE_LG_SEGMENTS  log2 of the segments each ray is split into and marched by that
 *                        many threads (0..5; batches use at most 2, a larger value counts
 *                        as 2 there), or -1 (default) to choose: one state, the most (up
 *                        to 32) that keep the launch within one wave of 256-thread CTAs;
 *                        batches, per state the most (up to 4) whose threads the
 *                        persistent launch holds at once
 *  RMP_TUNE_RAY_ORDER    0 (default): rays of one direction cell share warps (coherent
 *                        march); 1: Halton index order
 *  RMP_TUNE_SPLIT_BUDGET single-state evaluations: block visits after which the pieces
 *                        still running in a warp are cut into sub-pieces marched by the
 *                        warp's idle lanes (1..65536), 0 never, -1 (default) the library's
 *                        choice (currently never); batches never split
 *  RMP_TUNE_CELL_SKIP    free boxes of voxels inside occupied blocks crossed in one step
 *                        (grid layout maps): 1 always, 0 never, -1 (default) in batched
 *                        evaluations and in single-state ones marched as 4 or more segments
 *                        per ray (measured faster there, slower for one segment per ray) */
#define RMP_TUNE_BLOCK 1
#define RMP_TUNE_LG_SEGMENTS 2
#define RMP_TUNE_RAY_ORDER 3
#define RMP_TUNE_SPLIT_BUDGET 4
#define RMP_TUNE_CELL_SKIP 5
/* Set / read one knob of the context.  RMP_ERR_INVALID_ARG for an unknown knob or a value
 * outside its range; *value receives 0 or -1 where the library chooses. */
int rmp_tune_set(rmp_ctx* ctx, int knob, int value);
int rmp_tune_get(rmp_ctx* ctx, int knob, int* value);

/* Launch shape rmp_raycast_eval[_async] would use for this map, ray count and parameters:
 * threads per CTA, CTAs, log2 segments per ray, resident CTAs per SM (occupancy), SMs,
 * dynamic shared memory per CTA (the staged free-radius field and brick words) and the
 * number of direction cells of the ray order.  Host-side only; launches nothing. */
typedef struct {
  int32_t block, grid, lg_segments, ctas_per_sm, sm_count, smem_bytes, ray_cells, reserved;
} rmp_launch_info_t;
int rmp_eval_launch_info(rmp_ctx* ctx, uint32_t map_id, uint32_t n_rays,
                         const rmp_params_t* params, rmp_launch_info_t* out);

#ifdef __cplusplus
}
#endif
#endif /* RMP_H */
