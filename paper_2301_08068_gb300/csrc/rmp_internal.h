// rmp_internal.h -- types shared by the library's host code and kernels (not part of the
// public ABI).  Layouts in HBM:
//   * occupancy brick: one 8^3 voxel block = 512 bits = 64 bytes = 16 uint32 words; bit
//     b = lx + 8 ly + 64 lz lives in word b >> 5, bit b & 31 (a TSDF voxel is occupied iff
//     its value is <= 0; a dense voxel iff it is nonzero).
//   * grid layout (dense maps, and hashed maps whose block bounding box is moderate): the
//     bricks of every block in the bounding box, x fastest (all-zero where free), plus a
//     4-bit free radius per block: 0 if the block holds an occupied voxel, else
//     min(15, Chebyshev distance in blocks to the nearest such block), so the blocks
//     within radius - 1 of it are all free.  The march stages the radii in shared memory
//     and crosses a whole free box of blocks in one exact step.
//   * hash layout (fallback for very large extents): power-of-two array of 16-byte entries
//     {key, slot}; key packs the block coordinates (21 bits each, offset by 2^20); empty
//     entries hold ~0; linear probing from a Fibonacci (multiply-shift) hash, load factor
//     <= 1/4; blocks without occupied voxels keep their key with slot -1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rmp.h"

namespace rmp {

constexpr int kBrickWords = 16;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kKeyBias = 1 << 20;
constexpr int kMaxGrid = 4096;          // CTAs of one evaluation (grid-stride beyond)
constexpr int kWsHeaderBytes = 1024;
constexpr int kMaxRangeVoxels = 16384;  // keeps every DDA crossing numerator below 2^31
// Block visits before a warp's unfinished pieces are split over its idle lanes; by default
// never (measured: with coherent ray order the split does not shorten the slowest warps)
constexpr uint32_t kDefaultSplitBudget = 0xffffffffu;

struct HashEntry {
  unsigned long long key;
  uint32_t slot;
  uint32_t pad;
};

constexpr int kLayoutGrid = 0;
constexpr int kLayoutHash = 1;
constexpr uint32_t kMaxSmemRadiusBytes = 48 * 1024;   // staged in shared memory up to this
constexpr int kMaxFreeRadius = 15;
constexpr int kSmemBrickBytes = 16 * 32 * 4;           // batch kernel: one warp's staged bricks
constexpr int kCellDistCap = 4;                       // cell free distances are capped here
constexpr uint64_t kMaxCellBytes = 256ull << 20;      // cell distances kept up to this size
constexpr uint64_t kMaxGridBricks = 1ull << 26;       // grid layout up to 4 GiB of bricks

struct DevMap {
  int kind;                 // RMP_MAP_DENSE_U8 (rays exit at the grid) / RMP_MAP_HASHED_TSDF
  int layout;               // kLayoutGrid / kLayoutHash
  int hash_shift;           // 64 - log2(capacity)
  uint32_t cap_mask;
  float vs_f;               // RN32(voxel size)
  uint32_t radius_words;    // grid: uint32 words of the radius field (8 per word, multiple of 4)
  double vs;
  double origin[3];         // dense only (hashed maps are world-anchored)
  int dims[3];              // dense voxels per axis
  int gmin[3];              // grid: block coordinates of the grid's first brick
  int gdim[3];              // grid: bricks per axis
  const uint4* bricks;      // grid: brick (x + gdim0 (y + gdim1 z)); hash: by slot
  const uint32_t* radius;   // grid: 4-bit free radius of brick idx at bits 4 (idx & 7)
  const uint32_t* cells;    // grid (optional): 8 words per brick, the 4-bit free distance of
                            // each 2^3 cell c = cx + 4 cy + 16 cz at word c >> 3, bits 4 (c & 7)
  const HashEntry* table;   // hash layout only
};

// Constants of one evaluation derived on the host from rmp_params_t.
struct EvalConsts {
  float eta_rep, inv_nu_rep, eta_damp, inv_nu_damp, eps, c, r_up, inv_r;
  float r_hi, r_lo;         // r = r_hi + r_lo (FP32 pair)
  float min_up, max_dn;     // scans: d >= min_range <=> d >= min_up; d <= max <=> d <= max_dn
  long long R_fx;           // llrint(max_range / vs * 2^16)
  uint32_t n_rays, halton_offset;
  uint32_t perm_M, perm_Q, perm_R;   // coherent ray order (see ray_of_slot)
  uint32_t lg_segs;                  // each ray is marched as 2^lg_segs segments
  uint32_t split_budget;             // block visits before unfinished pieces are split (~0: never)
  int w_mode, reduce_mode;
  double c64;                        // soft-normalisation c (FP64, attractor)
  double att_alpha, att_beta;        // attractor gain and damping (combined evaluations)
  int att_mean;                      // combined: ray sums divided by the ray count first
  uint32_t seg_threads;              // batches: threads of the persistent launch (segments)
  double x0[6];                      // x, xdot carried in the launch itself, read when the
                                     // kernel's state pointer is null (synchronous calls)
};

// Closed-loop rollout of point robots (per robot, device-resident).
struct RolloutDev {
  double seg_start[3], prev_seg[3];
  double path_length, smooth_sum;
  uint32_t status, steps, smooth_n, have_prev;
};

struct RolloutConsts {
  double dt, goal_tol;
  uint32_t max_steps, seg_steps, n_rays, pad;
};

// Workspace of one single-state evaluation: a header, then one partial slot per CTA.  A
// slot is empty when every byte is 0xFF; CTA i > 0 fills slot i, CTA 0 waits for the
// slots, reads them and empties them again (see grid_finish).
struct WsHeader {
  unsigned int poisoned;    // nonzero after a timed-out finish: re-initialise the workspace
  unsigned int pad[kWsHeaderBytes / 4 - 1];
};

struct CtaPartial {         // 80 bytes per CTA
  double v[9];              // sum A (6), sum A f (3)
  unsigned int n_hits, n_active;
};

inline size_t workspace_bytes() {
  return kWsHeaderBytes + sizeof(CtaPartial) * (size_t)kMaxGrid;
}

// Header zero, partial slots empty: the state every evaluation leaves a workspace in.
inline cudaError_t workspace_reset(void* ws, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ws, 0, kWsHeaderBytes, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync((char*)ws + kWsHeaderBytes, 0xFF, workspace_bytes() - kWsHeaderBytes, s);
  return e;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ batched evaluation
// Work of a batch is cut into chunks of 32 threads (32 / S rays of one state, S segments
// per ray, S chosen per state) that the warps of a persistent grid take from a counter.  Each chunk stores a
// partial; kBatchGroup consecutive chunks of a state form a group (the last chunk of a
// group to finish sums them), and the last group of a state sums the groups and resolves.
constexpr uint32_t kBatchGroup = 32;
constexpr uint32_t kMaxBatchStates = 1u << 16;
constexpr uint32_t kMaxBatchSegs = 4;        // workspace is sized for up to 4 segments per ray

struct BatchState {         // 80 bytes, written by the prep kernel
  long long P[3];           // quantised position (2^-16 voxels)
  float v[3], vl[3];        // velocity as an FP32 pair
  uint32_t n_rays, chunk0, n_chunks, group0;
  uint32_t perm_M, perm_Q;  // direction cells (the remainder n_rays - perm_Q perm_M is derived)
  uint32_t lg_segs;         // log2 segments per ray of this state
  int status;               // RMP_OK or RMP_ERR_INVALID_ARG
};

struct BatchHeader {        // 128 bytes
  uint32_t next_chunk;      // work counter of the persistent grid
  uint32_t total_chunks;
  uint32_t n_states;
  uint32_t pad[29];
};

struct BatchLayout {
  size_t states, sticket, gticket, cparts, gparts, total;
  uint64_t chunks_per_state, groups_per_state;
};

inline BatchLayout batch_layout(uint32_t n_states, uint32_t max_rays) {
  BatchLayout L;
  L.chunks_per_state = ((uint64_t)max_rays * kMaxBatchSegs + 31) / 32;
  L.groups_per_state = (L.chunks_per_state + kBatchGroup - 1) / kBatchGroup;
  const uint64_t n = n_states;
  L.states = align256(sizeof(BatchHeader));
  L.sticket = align256(L.states + sizeof(BatchState) * n);
  L.gticket = align256(L.sticket + 4 * n);
  L.cparts = align256(L.gticket + 4 * n * L.groups_per_state);
  L.gparts = align256(L.cparts + sizeof(CtaPartial) * n * L.chunks_per_state);
  L.total = align256(L.gparts + sizeof(CtaPartial) * n * L.groups_per_state);
  return L;
}

inline unsigned long long pack_key(int bx, int by, int bz) {
  return (unsigned long long)(uint32_t)(bx + kKeyBias) |
         ((unsigned long long)(uint32_t)(by + kKeyBias) << 21) |
         ((unsigned long long)(uint32_t)(bz + kKeyBias) << 42);
}

// ESDF policy constants (FP64) of one evaluation.
struct EsdfConsts {
  double eta_rep, nu_rep, eta_damp, nu_damp, r, c, eps;
  double alpha, beta;       // attractor (with goals)
  int w_mode;
  int pad;
};

// Launchers (rmp_kernels.cu).  All enqueue on `stream` and return cudaGetLastError().
size_t raycast_smem_bytes(const DevMap& m);
size_t batch_smem_bytes(const DevMap& m, int block);   // + the staged bricks, per warp
int raycast_occupancy(const DevMap& m, int reduce_mode, int block);   // CTAs per SM
cudaError_t launch_raycast(const DevMap& m, const EvalConsts& k, const double* state_dev,
                           void* ws, rmp_result_t* out_dev, rmp_ray_hit_t* hits,
                           float* per_ray, int block, int grid, cudaStream_t stream);

int ctx_device(const rmp_ctx* ctx);                                  // CUDA device of a context
int batch_occupancy(const DevMap& m, int reduce_mode, int block);     // CTAs per SM
// Prep kernel + persistent batch kernel; n_rays_dev / states_dev on the device.  With
// goals_dev (3 doubles per state) each state's rays are combined with its attractor.
cudaError_t launch_batch(const DevMap& m, const EvalConsts& k, const double* states_dev,
                         const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                         void* ws, rmp_result_t* out_dev, rmp_ray_hit_t* hits, float* per_ray,
                         int block, int grid, cudaStream_t stream,
                         const double* goals_dev = nullptr);
// One control step of every robot (see rollout_step_kernel); counts running robots into
// *running (which the caller zeroes) when running is not null.
// L2 read-bandwidth probe (see rmp_probe_l2_read): grid CTAs of 512 threads.
cudaError_t launch_probe_l2(const uint4* buf, size_t n16, uint32_t passes, int grid,
                            uint64_t* checksum, cudaStream_t stream);
// The ESDF policy for n states, one warp each (see rmp_esdf_eval_async).
cudaError_t launch_esdf_eval(const rmp_primitive_t* prims, uint32_t n_prims, const EsdfConsts& k,
                             const double* states, const double* goals, uint32_t n_states,
                             rmp_result_t* out, double* query, cudaStream_t stream);
cudaError_t launch_rollout_step(const DevMap& m, const RolloutConsts& rc, const rmp_result_t* res,
                                double* states, const double* goals, uint32_t* n_rays,
                                RolloutDev* rs, uint32_t n, uint32_t* running,
                                cudaStream_t stream);
cudaError_t launch_scan(const float* pts, const EvalConsts& k, const double* state_dev,
                        void* ws, rmp_result_t* out_dev, float* per_ray, int block, int grid,
                        cudaStream_t stream);
cudaError_t launch_dense_bricks(const uint8_t* occ, const int dims[3], const int nb[3],
                                uint32_t* bricks, cudaStream_t stream);
// Free-radius field of a grid from its bricks (scratch: two byte arrays, one per brick).
cudaError_t launch_grid_radius(const uint32_t* bricks, const DevMap& m, uint8_t* scratch_a,
                               uint8_t* scratch_b, uint32_t* radius, cudaStream_t stream);
// Free distance of every 2^3 cell of the occupied bricks of a grid (see DevMap::cells).
cudaError_t launch_cell_dist(const uint32_t* bricks, const DevMap& m, uint32_t* cells,
                             cudaStream_t stream);
cudaError_t launch_key_bbox(const int32_t* keys, const uint32_t* bricks, uint32_t n_blocks,
                            int* bbox, cudaStream_t stream);
cudaError_t launch_grid_scatter(const int32_t* keys, const uint32_t* bricks, uint32_t n_blocks,
                                const DevMap& m, uint32_t* grid_bricks, cudaStream_t stream);
cudaError_t launch_tsdf_bricks(const float* tsdf, uint32_t n_blocks, uint32_t* bricks,
                               cudaStream_t stream);
cudaError_t launch_hash_build(const int32_t* keys, uint32_t n_blocks, const uint32_t* bricks,
                              HashEntry* table, uint32_t cap_mask, int hash_shift,
                              unsigned int* err, cudaStream_t stream);

}  // namespace rmp
