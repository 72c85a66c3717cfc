// rmp_api.cu -- host implementation of the C ABI declared in include/rmp.h: contexts,
// map upload (Sec. III-F: the map is kept in GPU memory and shared by all evaluations),
// parameter validation and the evaluation entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "rmp_internal.h"
#include "rmp_policy.h"

using namespace rmp;

namespace {

struct MapRec {
  DevMap dm;
  void* bricks = nullptr;
  void* table = nullptr;
  void* radius = nullptr;
  void* cells = nullptr;
  uint32_t n_bricks = 0;
  uint32_t cap = 0;
  uint64_t bytes = 0;
  uint64_t wave256[2] = {0, 0};   // threads of one wave of 256-thread CTAs, per reduction
};

}  // namespace

// An ESDF of primitives on the device (rmp_esdf_upload).
struct EsdfRec {
  rmp_primitive_t* prims = nullptr;
  uint32_t n = 0;
};

struct rmp_ctx {
  int device = 0;
  int sm_count = 0;
  std::mutex mu;
  std::map<uint32_t, MapRec> maps;
  std::map<uint32_t, EsdfRec> esdfs;
  uint32_t next_id = 1;
  int tune_block = 0;        // threads per CTA of the evaluation kernels (0: automatic)
  int tune_lg_segs = -1;     // log2 segments per ray (-1: chosen from the ray count)
  int tune_ray_order = 0;    // 0: coherent direction cells, 1: Halton index order
  int tune_split = -1;       // split budget (-1: default, 0: never split)
  int tune_cells = -1;       // voxel-box skipping (-1: batches, 4-segment states; 0: off; 1: on)
  // scratch of the synchronous calls (serialised by mu): the state travels in the launch's
  // constants; the kernel writes the result straight into mapped pinned host memory
  void* ws = nullptr;
  rmp_result_t* result_host = nullptr;  // pinned, mapped
  rmp_result_t* result_map = nullptr;   // its device address
};

namespace {

// Makes `dev` current for a scope and restores the caller's device; no driver call when
// it already is current (the common case, on the synchronous path of every evaluation).
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    ok_ = cudaGetDevice(&prev_) == cudaSuccess;
    switched_ = ok_ && prev_ != dev;
    if (switched_) ok_ = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok_ && switched_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false;
  bool switched_ = false;
};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RMP_OK;
  if (e == cudaErrorMemoryAllocation) return RMP_ERR_NO_MEMORY;
  cudaGetLastError();  // clear a sticky launch error so later calls can proceed
  return RMP_ERR_CUDA;
}

#define RMP_CUDA(expr)                       \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Smallest float >= v (v finite, in float range).
float round_up_f32(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

// Largest float <= v.
float round_down_f32(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}

// Snapshot of the context's launch knobs; call with c->mu held (rmp_tune_set writes them).
Tuning tuning_of(const rmp_ctx* c) {
  Tuning t;
  t.lg_segs = c->tune_lg_segs;
  t.ray_order = c->tune_ray_order;
  t.split = c->tune_split;
  t.block = c->tune_block;
  t.cells = c->tune_cells;
  return t;
}

// Derive the per-evaluation constants; validates every parameter.
int make_consts(const rmp_params_t* p, double vs, uint32_t n, bool scan, EvalConsts* k,
                const Tuning& tune = Tuning()) {
  if (!p) return RMP_ERR_INVALID_ARG;
  if (!(std::isfinite(p->eta_rep) && p->eta_rep >= 0.0) || !finite_pos(p->nu_rep) ||
      !(std::isfinite(p->eta_damp) && p->eta_damp >= 0.0) || !finite_pos(p->nu_damp) ||
      !finite_pos(p->r) || !finite_pos(p->c) || !finite_pos(p->eps) ||
      !finite_pos(p->max_range) || !(std::isfinite(p->min_range) && p->min_range >= 0.0) ||
      p->r > 1e30 || p->max_range > 1e30 || p->w_mode > 1 || p->reduce_mode > 1 ||
      p->flags != 0)
    return RMP_ERR_INVALID_ARG;
  if (n == 0) return RMP_ERR_INVALID_ARG;
  std::memset(k, 0, sizeof(*k));
  k->eta_rep = (float)p->eta_rep;
  k->inv_nu_rep = (float)(1.0 / p->nu_rep);
  k->eta_damp = (float)p->eta_damp;
  k->inv_nu_damp = (float)(1.0 / p->nu_damp);
  k->eps = (float)p->eps;
  k->c = (float)p->c;
  k->r_up = round_up_f32(p->r);
  k->inv_r = (float)(1.0 / p->r);
  k->r_hi = (float)p->r;
  k->r_lo = (float)(p->r - (double)k->r_hi);
  k->min_up = round_up_f32(p->min_range);
  k->max_dn = round_down_f32(p->max_range);
  k->n_rays = n;
  k->halton_offset = p->halton_offset;
  k->w_mode = (int)p->w_mode;
  k->reduce_mode = (int)p->reduce_mode;
  k->c64 = p->c;
  if (!scan) {
    if ((uint64_t)n + p->halton_offset > (1ull << 24)) return RMP_ERR_INVALID_ARG;
    const double vox = p->max_range / vs;
    if (!(vox <= (double)kMaxRangeVoxels)) return RMP_ERR_INVALID_ARG;
    k->R_fx = std::llrint(vox * 65536.0);
    if (tune.ray_order == 0) {
      pick_ray_cells(n, k);
    } else {
      k->perm_M = 1;
      k->perm_Q = n;
      k->perm_R = 0;
    }
    // small evaluations are latency-bound: marching each ray as 4 (2) segments shortens
    // every thread's serial chain; large ones are issue-bound, where segments only add work
    k->lg_segs = n <= 4096u ? 2u : (n <= 16384u ? 1u : 0u);
    if (tune.lg_segs >= 0) k->lg_segs = (uint32_t)tune.lg_segs;
    k->split_budget = tune.split < 0 ? kDefaultSplitBudget
                      : (tune.split == 0 ? 0xffffffffu : (uint32_t)tune.split);
  } else {
    k->perm_M = 1;
    k->perm_Q = n;
    k->perm_R = 0;
  }
  return RMP_OK;
}

// Enqueue one single-state evaluation with the launch shape of the ray count and the
// context's knobs.  k comes from make_consts; state_dev null: the state is in k.x0.
cudaError_t launch_single(const MapRec& mr, const Tuning& t, EvalConsts k,
                          const double* state_dev, void* ws, rmp_result_t* out,
                          rmp_ray_hit_t* hits, float* per_ray, cudaStream_t s) {
  DevMap dm = mr.dm;
  const uint64_t wave = mr.wave256[k.reduce_mode];
  auto_segments(t, k.n_rays, wave, &k);
  single_state_cells(t.cells, k, &dm);
  int block, grid;
  launch_shape(t, (uint64_t)k.n_rays << k.lg_segs, wave, &block, &grid);
  return launch_raycast(dm, k, state_dev, ws, out, hits, per_ray, block, grid, s);
}

void free_map(MapRec& r) {
  if (r.bricks) cudaFree(r.bricks);
  if (r.table) cudaFree(r.table);
  if (r.radius) cudaFree(r.radius);
  if (r.cells) cudaFree(r.cells);
  r.bricks = r.table = r.radius = r.cells = nullptr;
}

// uint32 words of a 4-bit-per-brick radius field, in whole uint4s (TMA copy granularity)
uint32_t radius_words_for(uint64_t n_bricks) {
  const uint64_t w = (n_bricks + 7) / 8;
  return (uint32_t)((w + 3) / 4 * 4);
}

// Free-radius field of a grid layout map whose bricks are in r.bricks.
int build_radius(MapRec& r, cudaStream_t s) {
  const uint64_t n = (uint64_t)r.dm.gdim[0] * r.dm.gdim[1] * r.dm.gdim[2];
  r.dm.radius_words = radius_words_for(n);
  uint8_t* a = nullptr;
  uint8_t* b = nullptr;
  cudaError_t e = cudaMalloc(&r.radius, (size_t)r.dm.radius_words * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&a, n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b, n);
  if (e == cudaSuccess)
    e = launch_grid_radius((const uint32_t*)r.bricks, r.dm, a, b, (uint32_t*)r.radius, s);
  // 2^3-cell free distances for voxel-box skipping inside occupied blocks (optional)
  if (e == cudaSuccess && n * 32 <= kMaxCellBytes) {
    e = cudaMalloc(&r.cells, n * 32);
    if (e == cudaSuccess) e = launch_cell_dist((const uint32_t*)r.bricks, r.dm, (uint32_t*)r.cells, s);
    if (e == cudaSuccess) r.dm.cells = (const uint32_t*)r.cells;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  return e == cudaSuccess ? RMP_OK : cuda_status(e);
}

// After a finish that timed out the context's workspace is poisoned (see grid_finish):
// reset it before the next synchronous call.  Caller holds c->mu.
cudaError_t refresh_ws(rmp_ctx* c, cudaStream_t s) {
  cudaError_t e = workspace_reset(c->ws, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

extern "C" {

const char* rmp_status_string(int status) {
  switch (status) {
    case RMP_OK: return "ok";
    case RMP_ERR_INVALID_ARG: return "invalid argument";
    case RMP_ERR_NO_MEMORY: return "out of memory";
    case RMP_ERR_CUDA: return "CUDA error";
    case RMP_ERR_TIMEOUT: return "timed out";
    case RMP_ERR_BUSY: return "busy";
    case RMP_ERR_UNKNOWN_MAP: return "unknown map id";
    case RMP_ERR_NOT_READY: return "not ready";
    default: return "unknown status";
  }
}

int rmp_params_preset(int preset, rmp_params_t* out) {
  if (!out) return RMP_ERR_INVALID_ARG;
  rmp_params_t p;
  std::memset(&p, 0, sizeof(p));
  if (preset == RMP_PRESET_STATIC_MAP) {         // Table I, "Static Map"
    p.eta_rep = 88.0; p.nu_rep = 1.4; p.eta_damp = 140.0; p.nu_damp = 1.2;
    p.r = 2.4; p.c = 0.2; p.max_range = 10.0; p.min_range = 0.0;
  } else if (preset == RMP_PRESET_LIDAR) {       // Table I, "LiDAR"
    p.eta_rep = 1.2; p.nu_rep = 1.5; p.eta_damp = 3.0; p.nu_damp = 1.0;
    p.r = 1.3; p.c = 1.0; p.max_range = 30.0; p.min_range = 0.2;
  } else {
    return RMP_ERR_INVALID_ARG;
  }
  p.eps = 1e-3;
  p.halton_offset = 1;
  p.w_mode = 0;
  p.reduce_mode = RMP_REDUCE_KAHAN32;
  *out = p;
  return RMP_OK;
}

int rmp_ctx_create(rmp_ctx** out, int device) {
  if (!out) return RMP_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) { cudaGetLastError(); return RMP_ERR_CUDA; }
  if (device < 0 || device >= n) return RMP_ERR_INVALID_ARG;
  DeviceGuard g(device);
  if (!g.ok()) return RMP_ERR_CUDA;
  rmp_ctx* c = new (std::nothrow) rmp_ctx();
  if (!c) return RMP_ERR_NO_MEMORY;
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMalloc(&c->ws, workspace_bytes());
  if (e == cudaSuccess) e = workspace_reset(c->ws, 0);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&c->result_host, sizeof(rmp_result_t), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->result_map, c->result_host, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rmp_ctx_destroy(c);
    return cuda_status(e);
  }
  *out = c;
  return RMP_OK;
}

int rmp_ctx_destroy(rmp_ctx* c) {
  if (!c) return RMP_ERR_INVALID_ARG;
  {
    DeviceGuard g(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& kv : c->maps) free_map(kv.second);
    c->maps.clear();
    for (auto& kv : c->esdfs)
      if (kv.second.prims) cudaFree(kv.second.prims);
    c->esdfs.clear();
    if (c->ws) cudaFree(c->ws);
    if (c->result_host) cudaFreeHost(c->result_host);
  }
  delete c;
  return RMP_OK;
}

int rmp_map_upload(rmp_ctx* c, const rmp_map_desc_t* d, rmp_stream_t stream, uint32_t* map_id) {
  if (!c || !d || !map_id) return RMP_ERR_INVALID_ARG;
  if (!finite_pos(d->voxel_size) || d->voxel_size > 1e6) return RMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  MapRec r;
  std::memset(&r.dm, 0, sizeof(r.dm));
  r.dm.kind = d->kind;
  r.dm.vs = d->voxel_size;
  r.dm.vs_f = (float)d->voxel_size;
  void* tmp_a = nullptr;
  void* tmp_b = nullptr;
  void* compact = nullptr;
  void* table = nullptr;
  unsigned int* err_dev = nullptr;
  int* bbox_dev = nullptr;
  auto cleanup = [&]() {
    if (tmp_a) cudaFree(tmp_a);
    if (tmp_b) cudaFree(tmp_b);
    if (compact) cudaFree(compact);
    if (table) cudaFree(table);
    if (err_dev) cudaFree(err_dev);
    if (bbox_dev) cudaFree(bbox_dev);
    tmp_a = tmp_b = compact = table = nullptr;
    err_dev = nullptr;
    bbox_dev = nullptr;
  };
  auto fail = [&](int st) {
    cleanup();
    free_map(r);
    return st;
  };
  if (d->kind == RMP_MAP_DENSE_U8) {
    for (int a = 0; a < 3; ++a) {
      if (d->dims[a] <= 0 || d->dims[a] > (1 << 20) || !std::isfinite(d->origin[a]))
        return RMP_ERR_INVALID_ARG;
      r.dm.dims[a] = d->dims[a];
      r.dm.gdim[a] = (d->dims[a] + 7) / 8;
      r.dm.gmin[a] = 0;
      r.dm.origin[a] = d->origin[a];
    }
    if (!d->occ) return RMP_ERR_INVALID_ARG;
    const uint64_t nvox = (uint64_t)d->dims[0] * d->dims[1] * d->dims[2];
    const uint64_t nbr = (uint64_t)r.dm.gdim[0] * r.dm.gdim[1] * r.dm.gdim[2];
    if (nbr > kMaxGridBricks) return RMP_ERR_INVALID_ARG;
    const uint8_t* occ = d->occ;
    if (!d->data_on_device) {
      cudaError_t e = cudaMalloc(&tmp_a, nvox);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp_a, d->occ, nvox, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return fail(cuda_status(e));
      occ = (const uint8_t*)tmp_a;
    }
    r.dm.layout = kLayoutGrid;
    r.n_bricks = (uint32_t)nbr;
    cudaError_t e = cudaMalloc(&r.bricks, nbr * 64);
    if (e == cudaSuccess) e = launch_dense_bricks(occ, r.dm.dims, r.dm.gdim, (uint32_t*)r.bricks, s);
    if (e != cudaSuccess) return fail(cuda_status(e));
    const int rs = build_radius(r, s);
    if (rs != RMP_OK) return fail(rs);
    r.bytes = nbr * 64 + (uint64_t)r.dm.radius_words * 4 + (r.cells ? nbr * 32 : 0);
  } else if (d->kind == RMP_MAP_HASHED_TSDF) {
    const uint32_t n = d->n_blocks;
    if (n > (1u << 26)) return RMP_ERR_INVALID_ARG;
    if (n > 0 && (!d->block_keys || !d->tsdf)) return RMP_ERR_INVALID_ARG;
    uint32_t cap = 16;
    while (cap < 4ull * n) cap <<= 1;
    int log2cap = 0;
    while ((1u << log2cap) < cap) ++log2cap;
    r.dm.cap_mask = cap - 1;
    r.dm.hash_shift = 64 - log2cap;
    // 1) bricks of every block, and the hash table (validates keys and duplicates)
    cudaError_t e = cudaMalloc(&table, (size_t)cap * sizeof(HashEntry));
    if (e == cudaSuccess) e = cudaMemsetAsync(table, 0xFF, (size_t)cap * sizeof(HashEntry), s);
    if (e == cudaSuccess && n > 0) e = cudaMalloc(&compact, (size_t)n * 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&err_dev, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err_dev, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMalloc((void**)&bbox_dev, 6 * sizeof(int));
    const int bbox_init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
    int bbox[6];
    std::memcpy(bbox, bbox_init, sizeof(bbox));
    if (e == cudaSuccess) e = cudaMemcpyAsync(bbox_dev, bbox, sizeof(bbox), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cuda_status(e));
    const int32_t* keys = d->block_keys;
    if (n > 0) {
      const float* tsdf = d->tsdf;
      if (!d->data_on_device) {
        e = cudaMalloc(&tmp_a, (size_t)n * 3 * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&tmp_b, (size_t)n * 512 * sizeof(float));
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(tmp_a, d->block_keys, (size_t)n * 3 * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(tmp_b, d->tsdf, (size_t)n * 512 * sizeof(float),
                              cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(cuda_status(e));
        keys = (const int32_t*)tmp_a;
        tsdf = (const float*)tmp_b;
      }
      e = launch_tsdf_bricks(tsdf, n, (uint32_t*)compact, s);
      if (e == cudaSuccess)
        e = launch_hash_build(keys, n, (const uint32_t*)compact, (HashEntry*)table, r.dm.cap_mask,
                              r.dm.hash_shift, err_dev, s);
      if (e == cudaSuccess) e = launch_key_bbox(keys, (const uint32_t*)compact, n, bbox_dev, s);
      if (e != cudaSuccess) return fail(cuda_status(e));
    }
    unsigned int err_host = 0;
    e = cudaMemcpyAsync(&err_host, err_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bbox, bbox_dev, sizeof(bbox), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_status(e));
    if (err_host != 0) return fail(RMP_ERR_INVALID_ARG);
    // 2) layout: a grid over the bounding box of the occupied blocks unless it is much
    //    larger than the blocks themselves; otherwise keep the hash table
    const bool none = bbox[0] > bbox[3];
    uint64_t gprod = 1;
    int gdim[3] = {1, 1, 1}, gmin[3] = {0, 0, 0};
    if (!none) {
      for (int a = 0; a < 3; ++a) {
        gmin[a] = bbox[a];
        gdim[a] = bbox[3 + a] - bbox[a] + 1;
        gprod *= (uint64_t)gdim[a];
      }
    }
    const uint64_t grid_bytes = gprod * 64;
    const bool use_grid = gprod <= kMaxGridBricks &&
                          (grid_bytes <= (256ull << 20) || grid_bytes <= 16ull * 64 * n);
    if (use_grid) {
      r.dm.layout = kLayoutGrid;
      for (int a = 0; a < 3; ++a) {
        r.dm.gmin[a] = gmin[a];
        r.dm.gdim[a] = gdim[a];
      }
      r.n_bricks = (uint32_t)gprod;
      e = cudaMalloc(&r.bricks, grid_bytes);
      if (e == cudaSuccess) e = cudaMemsetAsync(r.bricks, 0, grid_bytes, s);
      if (e == cudaSuccess && n > 0 && !none)
        e = launch_grid_scatter(keys, (const uint32_t*)compact, n, r.dm, (uint32_t*)r.bricks, s);
      if (e != cudaSuccess) return fail(cuda_status(e));
      const int rs = build_radius(r, s);
      if (rs != RMP_OK) return fail(rs);
      r.bytes = grid_bytes + (uint64_t)r.dm.radius_words * 4 + (r.cells ? gprod * 32 : 0);
    } else {
      r.dm.layout = kLayoutHash;
      r.bricks = compact;
      r.table = table;
      compact = table = nullptr;
      r.cap = cap;
      r.n_bricks = n;
      r.bytes = (uint64_t)cap * sizeof(HashEntry) + (uint64_t)n * 64;
    }
  } else {
    return RMP_ERR_INVALID_ARG;
  }
  cleanup();
  r.dm.bricks = (const uint4*)r.bricks;
  r.dm.table = (const HashEntry*)r.table;
  r.dm.radius = (const uint32_t*)r.radius;
  for (int red = 0; red < 2; ++red) {
    const int occ = raycast_occupancy(r.dm, red, 256);
    r.wave256[red] = occ > 0 ? (uint64_t)c->sm_count * (uint64_t)occ * 256u : 0;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  const uint32_t id = c->next_id++;
  c->maps[id] = r;
  *map_id = id;
  return RMP_OK;
}

int rmp_map_release(rmp_ctx* c, uint32_t map_id) {
  if (!c) return RMP_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->maps.find(map_id);
  if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
  free_map(it->second);
  c->maps.erase(it);
  return RMP_OK;
}

int rmp_map_info(rmp_ctx* c, uint32_t map_id, rmp_map_info_t* out) {
  if (!c || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->maps.find(map_id);
  if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
  std::memset(out, 0, sizeof(*out));
  out->kind = it->second.dm.kind;
  out->layout = (uint32_t)it->second.dm.layout;
  out->n_bricks = it->second.n_bricks;
  out->hash_capacity = it->second.cap;
  out->device_bytes = it->second.bytes;
  return RMP_OK;
}

int rmp_map_cell_distances(rmp_ctx* c, uint32_t map_id, int32_t grid_min[3],
                           int32_t grid_dim[3], uint32_t* cells, uint64_t cells_words) {
  if (!c || !grid_min || !grid_dim) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->maps.find(map_id);
  if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
  const MapRec& r = it->second;
  if (r.dm.layout != kLayoutGrid) return RMP_ERR_INVALID_ARG;
  const uint64_t words = 8ull * (uint64_t)r.dm.gdim[0] * r.dm.gdim[1] * r.dm.gdim[2];
  if (cells && (!r.cells || cells_words < words)) return RMP_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) {
    grid_min[a] = r.dm.gmin[a];
    grid_dim[a] = r.dm.gdim[a];
  }
  if (!cells) return RMP_OK;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  RMP_CUDA(cudaMemcpy(cells, r.cells, words * 4, cudaMemcpyDeviceToHost));
  return RMP_OK;
}

size_t rmp_workspace_bytes(void) { return workspace_bytes(); }

int rmp_tune_set(rmp_ctx* c, int knob, int value) {
  if (!c) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (knob == RMP_TUNE_BLOCK) {
    if (value != 0 && value != 64 && value != 128 && value != 256) return RMP_ERR_INVALID_ARG;
    c->tune_block = value;
  } else if (knob == RMP_TUNE_LG_SEGMENTS) {
    if (value < -1 || value > (int)kMaxSingleLgSegs) return RMP_ERR_INVALID_ARG;
    c->tune_lg_segs = value;
  } else if (knob == RMP_TUNE_RAY_ORDER) {
    if (value < 0 || value > 1) return RMP_ERR_INVALID_ARG;
    c->tune_ray_order = value;
  } else if (knob == RMP_TUNE_SPLIT_BUDGET) {
    if (value < -1 || value > 65536) return RMP_ERR_INVALID_ARG;
    c->tune_split = value;
  } else if (knob == RMP_TUNE_CELL_SKIP) {
    if (value < -1 || value > 1) return RMP_ERR_INVALID_ARG;
    c->tune_cells = value;
  } else {
    return RMP_ERR_INVALID_ARG;
  }
  return RMP_OK;
}

int rmp_eval_launch_info(rmp_ctx* c, uint32_t map_id, uint32_t n_rays, const rmp_params_t* params,
                         rmp_launch_info_t* out) {
  if (!c || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->maps.find(map_id);
  if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
  const DevMap dm = it->second.dm;
  EvalConsts k;
  const Tuning t = tuning_of(c);
  int st = make_consts(params, dm.vs, n_rays, false, &k, t);
  if (st != RMP_OK) return st;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  const uint64_t wave = it->second.wave256[k.reduce_mode];
  auto_segments(t, n_rays, wave, &k);
  int block, grid;
  launch_shape(t, (uint64_t)n_rays << k.lg_segs, wave, &block, &grid);
  out->block = block;
  out->grid = grid;
  out->lg_segments = (int)k.lg_segs;
  out->ctas_per_sm = raycast_occupancy(dm, k.reduce_mode, block);
  out->sm_count = c->sm_count;
  out->smem_bytes = (int)raycast_smem_bytes(dm);
  out->ray_cells = (int)k.perm_M;
  return RMP_OK;
}

int rmp_tune_get(rmp_ctx* c, int knob, int* value) {
  if (!c || !value) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (knob == RMP_TUNE_BLOCK) *value = c->tune_block;
  else if (knob == RMP_TUNE_LG_SEGMENTS) *value = c->tune_lg_segs;
  else if (knob == RMP_TUNE_RAY_ORDER) *value = c->tune_ray_order;
  else if (knob == RMP_TUNE_SPLIT_BUDGET) *value = c->tune_split;
  else if (knob == RMP_TUNE_CELL_SKIP) *value = c->tune_cells;
  else return RMP_ERR_INVALID_ARG;
  return RMP_OK;
}

int rmp_workspace_init(void* ws, size_t bytes, rmp_stream_t stream) {
  if (!ws || bytes < workspace_bytes()) return RMP_ERR_INVALID_ARG;
  RMP_CUDA(workspace_reset(ws, (cudaStream_t)stream));
  return RMP_OK;
}

int rmp_raycast_eval_async(rmp_ctx* c, uint32_t map_id, const double* state_dev, uint32_t n_rays,
                           const rmp_params_t* params, void* ws, size_t ws_bytes,
                           rmp_stream_t stream, rmp_result_t* out_dev, rmp_ray_hit_t* hits_dev,
                           float* per_ray_dev) {
  if (!c || !state_dev || !ws || !out_dev || ws_bytes < workspace_bytes())
    return RMP_ERR_INVALID_ARG;
  MapRec mr;
  Tuning t;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->maps.find(map_id);
    if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
    mr = it->second;
    t = tuning_of(c);
  }
  EvalConsts k;
  int st = make_consts(params, mr.dm.vs, n_rays, false, &k, t);
  if (st != RMP_OK) return st;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  RMP_CUDA(launch_single(mr, t, k, state_dev, ws, out_dev, hits_dev, per_ray_dev,
                         (cudaStream_t)stream));
  return RMP_OK;
}

int rmp_raycast_eval(rmp_ctx* c, uint32_t map_id, const double x[3], const double xdot[3],
                     uint32_t n_rays, const rmp_params_t* params, rmp_stream_t stream,
                     rmp_result_t* out, rmp_ray_hit_t* hits_dev, float* per_ray_dev) {
  if (!c || !x || !xdot || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);      // held until the result is back
  auto it = c->maps.find(map_id);
  if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
  EvalConsts k;
  const Tuning t = tuning_of(c);
  int st = make_consts(params, it->second.dm.vs, n_rays, false, &k, t);
  if (st != RMP_OK) return st;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  for (int a = 0; a < 3; ++a) {        // x, xdot go to the device inside the launch
    k.x0[a] = x[a];
    k.x0[3 + a] = xdot[a];
  }
  RMP_CUDA(launch_single(it->second, t, k, nullptr, c->ws, c->result_map, hits_dev, per_ray_dev,
                         s));
  RMP_CUDA(cudaStreamSynchronize(s));
  *out = *c->result_host;
  if (out->status == RMP_ERR_TIMEOUT) RMP_CUDA(refresh_ws(c, s));
  return RMP_OK;
}

int rmp_scan_eval_async(rmp_ctx* c, const float* points_dev, uint32_t n, const double* state_dev,
                        const rmp_params_t* params, void* ws, size_t ws_bytes,
                        rmp_stream_t stream, rmp_result_t* out_dev, float* per_ray_dev) {
  if (!c || !points_dev || !state_dev || !ws || !out_dev || ws_bytes < workspace_bytes())
    return RMP_ERR_INVALID_ARG;
  EvalConsts k;
  int st = make_consts(params, 1.0, n, true, &k);
  if (st != RMP_OK) return st;
  Tuning t;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    t = tuning_of(c);
  }
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  int block, grid;
  scan_shape(t, c->sm_count, n, &block, &grid);
  RMP_CUDA(launch_scan(points_dev, k, state_dev, ws, out_dev, per_ray_dev, block, grid,
                       (cudaStream_t)stream));
  return RMP_OK;
}

int rmp_scan_eval(rmp_ctx* c, const float* points_dev, uint32_t n, const double x[3],
                  const double xdot[3], const rmp_params_t* params, rmp_stream_t stream,
                  rmp_result_t* out, float* per_ray_dev) {
  if (!c || !points_dev || !x || !xdot || !out) return RMP_ERR_INVALID_ARG;
  EvalConsts k;
  int st = make_consts(params, 1.0, n, true, &k);
  if (st != RMP_OK) return st;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  for (int a = 0; a < 3; ++a) {
    k.x0[a] = x[a];
    k.x0[3 + a] = xdot[a];
  }
  int block, grid;
  scan_shape(tuning_of(c), c->sm_count, n, &block, &grid);
  RMP_CUDA(launch_scan(points_dev, k, nullptr, c->ws, c->result_map, per_ray_dev, block, grid,
                       s));
  RMP_CUDA(cudaStreamSynchronize(s));
  *out = *c->result_host;
  if (out->status == RMP_ERR_TIMEOUT) RMP_CUDA(refresh_ws(c, s));
  return RMP_OK;
}

// ------------------------------------------------------------------ batched evaluation
}  // extern "C"

int rmp::ctx_device(const rmp_ctx* c) { return c->device; }

extern "C" {

size_t rmp_batch_workspace_bytes(uint32_t n_states, uint32_t max_rays) {
  if (n_states == 0 || n_states > kMaxBatchStates || max_rays == 0) return 0;
  return batch_layout(n_states, max_rays).total;
}

namespace {

// Constants and launch shape of a batch; grid = every CTA that fits on the device at once.
int batch_setup(rmp_ctx* c, uint32_t map_id, uint32_t n_states, uint32_t max_rays,
                const rmp_params_t* params, DevMap* dm, EvalConsts* k, int* block, int* grid) {
  if (n_states == 0 || n_states > kMaxBatchStates || max_rays == 0) return RMP_ERR_INVALID_ARG;
  Tuning t;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->maps.find(map_id);
    if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
    *dm = it->second.dm;
    t = tuning_of(c);
    if (t.cells == 0) dm->cells = nullptr;        // batches: on unless switched off
    *block = t.block != 0 ? t.block : 128;
  }
  int st = make_consts(params, dm->vs, max_rays, false, k, t);
  if (st != RMP_OK) return st;
  // segments per ray: a fixed tuned value for every state (at most kMaxBatchSegs, which the
  // batch workspace is sized for), or (default) the batch rule applied per state by the
  // prep kernel
  if (t.lg_segs < 0) k->lg_segs = 0xffffffffu;
  else if ((1u << k->lg_segs) > kMaxBatchSegs) k->lg_segs = 2;
  const int occ = batch_occupancy(*dm, k->reduce_mode, *block);
  if (occ <= 0) return RMP_ERR_CUDA;
  *grid = c->sm_count * occ;
  k->seg_threads = (uint32_t)*grid * (uint32_t)*block;
  return RMP_OK;
}

}  // namespace

namespace {

int batch_async_impl(rmp_ctx* c, uint32_t map_id, const double* states_dev,
                     const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                     const rmp_params_t* params, void* ws, size_t ws_bytes, rmp_stream_t stream,
                     rmp_result_t* out_dev, rmp_ray_hit_t* hits_dev, float* per_ray_dev,
                     const double* goals_dev, double alpha, double beta, int metric_mean = 0) {
  if (!c || !states_dev || !n_rays_dev || !ws || !out_dev) return RMP_ERR_INVALID_ARG;
  if (n_states == 0 || n_states > kMaxBatchStates || max_rays == 0 ||
      ws_bytes < batch_layout(n_states, max_rays).total)
    return RMP_ERR_INVALID_ARG;
  if (goals_dev && !(std::isfinite(alpha) && alpha >= 0.0 && std::isfinite(beta) && beta >= 0.0))
    return RMP_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  DevMap dm;
  EvalConsts k;
  int block, grid;
  int st = batch_setup(c, map_id, n_states, max_rays, params, &dm, &k, &block, &grid);
  if (st != RMP_OK) return st;
  k.att_alpha = alpha;
  k.att_beta = beta;
  k.att_mean = metric_mean ? 1 : 0;
  RMP_CUDA(launch_batch(dm, k, states_dev, n_rays_dev, n_states, max_rays, ws, out_dev, hits_dev,
                        per_ray_dev, block, grid, (cudaStream_t)stream, goals_dev));
  return RMP_OK;
}

}  // namespace

int rmp_combined_eval_batch_async(rmp_ctx* c, uint32_t map_id, const double* states_dev,
                                  const uint32_t* n_rays_dev, uint32_t n_states,
                                  uint32_t max_rays, const rmp_params_t* params,
                                  const double* goals_dev, double alpha, double beta,
                                  uint32_t metric_mean, void* ws, size_t ws_bytes,
                                  rmp_stream_t stream, rmp_result_t* out_dev) {
  if (!goals_dev || metric_mean > 1) return RMP_ERR_INVALID_ARG;
  return batch_async_impl(c, map_id, states_dev, n_rays_dev, n_states, max_rays, params, ws,
                          ws_bytes, stream, out_dev, nullptr, nullptr, goals_dev, alpha, beta,
                          (int)metric_mean);
}

}  // extern "C"

namespace {

// Constants of the ESDF policy from rmp_params_t (validated as for the ray policy).
int make_esdf_consts(const rmp_params_t* p, double alpha, double beta, EsdfConsts* k) {
  EvalConsts e;
  const int st = make_consts(p, 1.0, 1, true, &e);
  if (st != RMP_OK) return st;
  if (!(std::isfinite(alpha) && alpha >= 0.0 && std::isfinite(beta) && beta >= 0.0))
    return RMP_ERR_INVALID_ARG;
  std::memset(k, 0, sizeof(*k));
  k->eta_rep = p->eta_rep;
  k->nu_rep = p->nu_rep;
  k->eta_damp = p->eta_damp;
  k->nu_damp = p->nu_damp;
  k->r = p->r;
  k->c = p->c;
  k->eps = p->eps;
  k->alpha = alpha;
  k->beta = beta;
  k->w_mode = (int)p->w_mode;
  return RMP_OK;
}

// Closed loop of rmp_rollout (esdf null: the raycasting policy) and rmp_rollout_esdf.
int rollout_impl(rmp_ctx* c, uint32_t map_id, const EsdfRec* esdf, const double* robots,
                 uint32_t n, const rmp_params_t* params, const rmp_rollout_params_t* rp,
                 rmp_stream_t stream, rmp_rollout_result_t* out) {
  if (!c || !robots || !params || !rp || !out || n == 0 || n > kMaxBatchStates)
    return RMP_ERR_INVALID_ARG;
  if (!(rp->dt > 0.0 && std::isfinite(rp->dt)) || !(rp->goal_tol >= 0.0) || rp->max_steps == 0 ||
      (!esdf && (rp->n_rays == 0 || rp->metric_mean > 1)))
    return RMP_ERR_INVALID_ARG;
  EsdfConsts ek;
  if (esdf) {
    const int st = make_esdf_consts(params, rp->alpha, rp->beta, &ek);
    if (st != RMP_OK) return st;
  }
  DevMap dm;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->maps.find(map_id);
    if (it == c->maps.end()) return RMP_ERR_UNKNOWN_MAP;
    dm = it->second.dm;
  }
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t wsb = esdf ? 0 : batch_layout(n, rp->n_rays).total;
  const size_t o_st = 0, o_goal = align256(48 * (size_t)n), o_nr = o_goal + align256(24 * (size_t)n),
               o_res = o_nr + align256(4 * (size_t)n),
               o_rs = o_res + align256(sizeof(rmp_result_t) * n),
               o_cnt = o_rs + align256(sizeof(RolloutDev) * n), o_ws = o_cnt + 256;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, o_ws + wsb);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<double> st(6 * (size_t)n), goal(3 * (size_t)n);
  std::vector<uint32_t> nr(n, rp->n_rays);
  std::vector<RolloutDev> rs(n);
  for (uint32_t b = 0; b < n; ++b) {
    for (int a = 0; a < 6; ++a) st[6 * b + a] = robots[9 * (size_t)b + a];
    for (int a = 0; a < 3; ++a) goal[3 * b + a] = robots[9 * (size_t)b + 6 + a];
    std::memset(&rs[b], 0, sizeof(RolloutDev));
    for (int a = 0; a < 3; ++a) rs[b].seg_start[a] = st[6 * b + a];
  }
  double* d_st = (double*)(buf + o_st);
  double* d_goal = (double*)(buf + o_goal);
  uint32_t* d_nr = (uint32_t*)(buf + o_nr);
  rmp_result_t* d_res = (rmp_result_t*)(buf + o_res);
  RolloutDev* d_rs = (RolloutDev*)(buf + o_rs);
  uint32_t* d_cnt = (uint32_t*)(buf + o_cnt);
  RolloutConsts rc;
  rc.dt = rp->dt;
  rc.goal_tol = rp->goal_tol;
  rc.max_steps = rp->max_steps;
  rc.seg_steps = rp->seg_steps;
  rc.n_rays = rp->n_rays;
  rc.pad = 0;
  int status = RMP_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_st, st.data(), 48 * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_goal, goal.data(), 24 * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_nr, nr.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rs, rs.data(), sizeof(RolloutDev) * n, cudaMemcpyHostToDevice, s);
  // steps in rounds of 32; after each round the running count decides whether to go on
  const uint32_t kRound = 32;
  uint32_t running = n;
  for (uint32_t step = 0; e == cudaSuccess && status == RMP_OK && running > 0 &&
                          step < rp->max_steps;) {
    e = cudaMemsetAsync(d_cnt, 0, 4, s);
    for (uint32_t i = 0; i < kRound && step < rp->max_steps && e == cudaSuccess; ++i, ++step) {
      if (esdf) {
        e = launch_esdf_eval(esdf->prims, esdf->n, ek, d_st, d_goal, n, d_res, nullptr, s);
        if (e != cudaSuccess) break;
      } else {
        status = batch_async_impl(c, map_id, d_st, d_nr, n, rp->n_rays, params, buf + o_ws, wsb,
                                  stream, d_res, nullptr, nullptr, d_goal, rp->alpha, rp->beta,
                                  (int)rp->metric_mean);
        if (status != RMP_OK) break;
      }
      e = launch_rollout_step(dm, rc, d_res, d_st, d_goal, d_nr, d_rs, n,
                              i + 1 == kRound || step + 1 == rp->max_steps ? d_cnt : nullptr, s);
    }
    if (e == cudaSuccess && status == RMP_OK) {
      e = cudaMemcpyAsync(&running, d_cnt, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  if (e == cudaSuccess && status == RMP_OK) {
    e = cudaMemcpyAsync(st.data(), d_st, 48 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rs.data(), d_rs, sizeof(RolloutDev) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(buf);
  if (status != RMP_OK) return status;
  if (e != cudaSuccess) return cuda_status(e);
  for (uint32_t b = 0; b < n; ++b) {
    rmp_rollout_result_t& r = out[b];
    std::memset(&r, 0, sizeof(r));
    for (int a = 0; a < 3; ++a) {
      r.x[a] = st[6 * b + a];
      r.xdot[a] = st[6 * b + 3 + a];
    }
    r.path_length = rs[b].path_length;
    r.smoothness = rs[b].smooth_n ? rs[b].smooth_sum / rs[b].smooth_n : 1.0;
    r.status = rs[b].status;
    r.steps = rs[b].steps;
    r.smooth_segments = rs[b].smooth_n;
  }
  return RMP_OK;
}

}  // namespace

extern "C" {

int rmp_rollout(rmp_ctx* c, uint32_t map_id, const double* robots, uint32_t n,
                const rmp_params_t* params, const rmp_rollout_params_t* rp, rmp_stream_t stream,
                rmp_rollout_result_t* out) {
  return rollout_impl(c, map_id, nullptr, robots, n, params, rp, stream, out);
}

int rmp_probe_l2_read(rmp_ctx* c, const void* buf_dev, size_t bytes, uint32_t passes,
                      rmp_stream_t stream, uint64_t* checksum_dev) {
  if (!c || !buf_dev || !checksum_dev || bytes == 0 || bytes % 16 != 0 ||
      ((uintptr_t)buf_dev & 15u) != 0 || passes == 0)
    return RMP_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  RMP_CUDA(launch_probe_l2((const uint4*)buf_dev, bytes / 16, passes, c->sm_count * 4,
                           checksum_dev, (cudaStream_t)stream));
  return RMP_OK;
}

int rmp_esdf_upload(rmp_ctx* c, const rmp_primitive_t* prims, uint32_t n, uint32_t* esdf_id) {
  if (!c || !esdf_id || (n > 0 && !prims) || n > (1u << 20)) return RMP_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < n; ++i) {
    const rmp_primitive_t& p = prims[i];
    if (p.kind > RMP_PRIM_BOX || p.reserved != 0) return RMP_ERR_INVALID_ARG;
    const int ns = p.kind == RMP_PRIM_SPHERE ? 1 : 3;
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(p.center[a])) return RMP_ERR_INVALID_ARG;
    for (int a = 0; a < ns; ++a)
      if (!finite_pos(p.size[a])) return RMP_ERR_INVALID_ARG;
  }
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  EsdfRec r;
  r.n = n;
  if (n > 0) {
    RMP_CUDA(cudaMalloc((void**)&r.prims, sizeof(rmp_primitive_t) * n));
    const cudaError_t e = cudaMemcpy(r.prims, prims, sizeof(rmp_primitive_t) * n,
                                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(r.prims);
      return cuda_status(e);
    }
  }
  std::lock_guard<std::mutex> lk(c->mu);
  const uint32_t id = c->next_id++;
  c->esdfs[id] = r;
  *esdf_id = id;
  return RMP_OK;
}

int rmp_esdf_release(rmp_ctx* c, uint32_t esdf_id) {
  if (!c) return RMP_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->esdfs.find(esdf_id);
  if (it == c->esdfs.end()) return RMP_ERR_UNKNOWN_MAP;
  if (it->second.prims) cudaFree(it->second.prims);
  c->esdfs.erase(it);
  return RMP_OK;
}

int rmp_esdf_eval_async(rmp_ctx* c, uint32_t esdf_id, const double* states_dev,
                        const double* goals_dev, uint32_t n_states, const rmp_params_t* params,
                        double alpha, double beta, rmp_stream_t stream, rmp_result_t* out_dev,
                        double* query_dev) {
  if (!c || !states_dev || !out_dev || n_states == 0) return RMP_ERR_INVALID_ARG;
  EsdfConsts k;
  const int st = make_esdf_consts(params, alpha, beta, &k);
  if (st != RMP_OK) return st;
  EsdfRec r;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->esdfs.find(esdf_id);
    if (it == c->esdfs.end()) return RMP_ERR_UNKNOWN_MAP;
    r = it->second;
  }
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  RMP_CUDA(launch_esdf_eval(r.prims, r.n, k, states_dev, goals_dev, n_states, out_dev, query_dev,
                            (cudaStream_t)stream));
  return RMP_OK;
}

int rmp_rollout_esdf(rmp_ctx* c, uint32_t map_id, uint32_t esdf_id, const double* robots,
                     uint32_t n, const rmp_params_t* params, const rmp_rollout_params_t* rp,
                     rmp_stream_t stream, rmp_rollout_result_t* out) {
  if (!c) return RMP_ERR_INVALID_ARG;
  EsdfRec r;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->esdfs.find(esdf_id);
    if (it == c->esdfs.end()) return RMP_ERR_UNKNOWN_MAP;
    r = it->second;
  }
  return rollout_impl(c, map_id, &r, robots, n, params, rp, stream, out);
}

int rmp_raycast_eval_batch_async(rmp_ctx* c, uint32_t map_id, const double* states_dev,
                                 const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                                 const rmp_params_t* params, void* ws, size_t ws_bytes,
                                 rmp_stream_t stream, rmp_result_t* out_dev,
                                 rmp_ray_hit_t* hits_dev, float* per_ray_dev) {
  return batch_async_impl(c, map_id, states_dev, n_rays_dev, n_states, max_rays, params, ws,
                          ws_bytes, stream, out_dev, hits_dev, per_ray_dev, nullptr, 0.0, 0.0);
}

int rmp_raycast_eval_batch(rmp_ctx* c, uint32_t map_id, const double* states, const uint32_t* n_rays,
                           uint32_t n_states, const rmp_params_t* params, rmp_stream_t stream,
                           rmp_result_t* out) {
  if (!c || !states || !n_rays || !out || n_states == 0 || n_states > kMaxBatchStates)
    return RMP_ERR_INVALID_ARG;
  uint32_t max_rays = 1;
  for (uint32_t b = 0; b < n_states; ++b) max_rays = n_rays[b] > max_rays ? n_rays[b] : max_rays;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  const size_t wsb = batch_layout(n_states, max_rays).total;
  const size_t sb = 6 * sizeof(double) * n_states, nb = 4 * (size_t)n_states,
               ob = sizeof(rmp_result_t) * n_states;
  char* buf = nullptr;
  const size_t o_states = 0, o_n = align256(sb), o_out = o_n + align256(nb),
               o_ws = o_out + align256(ob);
  cudaError_t e = cudaMalloc((void**)&buf, o_ws + wsb);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t s = (cudaStream_t)stream;
  int st = RMP_OK;
  e = cudaMemcpyAsync(buf + o_states, states, sb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_n, n_rays, nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    st = rmp_raycast_eval_batch_async(c, map_id, (const double*)(buf + o_states),
                                      (const uint32_t*)(buf + o_n), n_states, max_rays, params,
                                      buf + o_ws, wsb, stream, (rmp_result_t*)(buf + o_out),
                                      nullptr, nullptr);
  }
  if (e == cudaSuccess && st == RMP_OK)
    e = cudaMemcpyAsync(out, buf + o_out, ob, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (st != RMP_OK) return st;
  return e == cudaSuccess ? RMP_OK : cuda_status(e);
}

int rmp_batch_autotune(rmp_ctx* c, uint32_t map_id, const double* states_dev,
                       const uint32_t* n_rays_dev, uint32_t n_states, uint32_t max_rays,
                       const rmp_params_t* params, void* ws, size_t ws_bytes, rmp_stream_t stream,
                       rmp_result_t* out_dev, int reps, float* times_ms, int n_times) {
  if (!c || reps < 1 || reps > 1000) return RMP_ERR_INVALID_ARG;
  static const int kBlocks[3] = {64, 128, 256};
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(c->device);
  if (!g.ok()) return RMP_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RMP_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RMP_ERR_CUDA;
  }
  float best = 3.0e38f;
  int best_b = 128, best_l = 0, idx = 0, st = RMP_OK;
  for (int bi = 0; bi < 3 && st == RMP_OK; ++bi)
    for (int l = 0; l <= 2 && st == RMP_OK; ++l, ++idx) {
        {
          std::lock_guard<std::mutex> lk(c->mu);
          c->tune_block = kBlocks[bi];
          c->tune_lg_segs = l;
        }
        // one untimed launch, then the median of `reps` timed ones
        st = rmp_raycast_eval_batch_async(c, map_id, states_dev, n_rays_dev, n_states, max_rays,
                                          params, ws, ws_bytes, stream, out_dev, nullptr, nullptr);
        float t[1000];
        for (int r = 0; r < reps && st == RMP_OK; ++r) {
          if (cudaEventRecord(e0, s) != cudaSuccess) st = RMP_ERR_CUDA;
          if (st == RMP_OK)
            st = rmp_raycast_eval_batch_async(c, map_id, states_dev, n_rays_dev, n_states,
                                              max_rays, params, ws, ws_bytes, stream, out_dev,
                                              nullptr, nullptr);
          if (st == RMP_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                               cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess))
            st = RMP_ERR_CUDA;
        }
        if (st != RMP_OK) break;
        std::sort(t, t + reps);
        const float med = t[reps / 2];
        if (times_ms && idx < n_times) times_ms[idx] = med;
        if (med < best) {
          best = med;
          best_b = kBlocks[bi];
          best_l = l;
        }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(c->mu);
  c->tune_block = best_b;
  c->tune_lg_segs = best_l;
  return st;
}

}  // extern "C"
