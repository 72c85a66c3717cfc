// rmp_static.cu -- batched evaluation with library-owned scratch: the batch workspace lives
// in a file-scope __device__ array instead of caller-provided device memory, so a call
// allocates nothing (see rmp_raycast_eval_batch_static in include/rmp.h).
#include <mutex>

#include "rmp_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;   // 4 MiB per device

// Batch workspace of the static entry point.  Nothing in it has to start at zero: the
// batch's prep kernel clears the tickets and the work counter at the start of every call.
static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

std::mutex g_mu;
// Device address of g_batch_scratch, per device id, looked up once per process: it stays
// valid for the life of the device's primary context (a cudaDeviceReset ends it, and this
// entry point must not be used after one).
void* g_scratch[64];
bool g_have[64];

}  // namespace

extern "C" int rmp_raycast_eval_batch_static(rmp_ctx* ctx, uint32_t map_id,
                                             const double* states_dev,
                                             const uint32_t* n_rays_dev, uint32_t n_states,
                                             uint32_t max_rays, const rmp_params_t* params,
                                             rmp_stream_t stream, rmp_result_t* out_dev) {
  if (!ctx || !states_dev || !n_rays_dev || !out_dev || n_states == 0 ||
      n_states > rmp::kMaxBatchStates || max_rays == 0)
    return RMP_ERR_INVALID_ARG;
  if (rmp::batch_layout(n_states, max_rays).total > kStaticScratchBytes)
    return RMP_ERR_NO_MEMORY;                     // batch larger than the static scratch
  const int dev = rmp::ctx_device(ctx);
  if (dev < 0 || dev >= 64) return RMP_ERR_INVALID_ARG;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_have[dev]) {
      // first call on this device: look up the array's device address with the device
      // current (may load the module's data on the device)
      int prev = 0;
      if (cudaGetDevice(&prev) != cudaSuccess) return RMP_ERR_CUDA;
      if (cudaSetDevice(dev) != cudaSuccess) return RMP_ERR_CUDA;
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
      const cudaError_t e_restore = cudaSetDevice(prev);
      if (e != cudaSuccess || !p || e_restore != cudaSuccess) return RMP_ERR_CUDA;
      g_scratch[dev] = p;
      g_have[dev] = true;
    }
    scratch = g_scratch[dev];
  }
  return rmp_raycast_eval_batch_async(ctx, map_id, states_dev, n_rays_dev, n_states, max_rays,
                                      params, scratch, kStaticScratchBytes, stream, out_dev,
                                      nullptr, nullptr);
}
