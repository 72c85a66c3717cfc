// rmp_stream.cu -- streamed LiDAR scans with host-to-device copies overlapped with the
// evaluation of the previous scan (host runtime; the evaluation is the scan kernel).
//
// A pipeline owns `slots` scan slots, each with device points, a workspace, a device and a
// pinned result, and two events.  Submitting a scan (points in the caller's pinned host
// memory) takes the next slot in turn -- waiting for that slot's previous scan to finish --
// enqueues the copy on the copy stream, makes the compute stream wait for it, enqueues the
// scan kernel and the 144-byte result copy on the compute stream, and returns a ticket.
// While scan k is being evaluated, the copy of scan k + 1 runs on the other stream.
#include <cstring>
#include <mutex>
#include <vector>

#include "rmp_internal.h"

namespace {

struct ScanSlot {
  float* pts = nullptr;           // device, max_points x 3
  void* ws = nullptr;             // workspace of the scan kernel
  double* state = nullptr;        // device x, xdot
  double* state_host = nullptr;   // pinned
  rmp_result_t* res = nullptr;    // device
  rmp_result_t* res_host = nullptr;
  cudaEvent_t copied = nullptr, done = nullptr;
  uint64_t ticket = 0;            // scan currently (or last) in this slot
  bool used = false;
};

}  // namespace

struct rmp_scan_pipeline {
  rmp_ctx* ctx = nullptr;
  int device = 0;
  uint32_t max_points = 0;
  cudaStream_t copy = nullptr, compute = nullptr;
  std::vector<ScanSlot> slots;
  std::mutex mu;
  uint64_t next = 1;
};

extern "C" {

int rmp_scan_pipeline_create(rmp_ctx* ctx, uint32_t max_points, uint32_t slots,
                             rmp_scan_pipeline** out) {
  if (!ctx || !out || max_points == 0 || slots < 2 || slots > 8) return RMP_ERR_INVALID_ARG;
  rmp_scan_pipeline* p = new (std::nothrow) rmp_scan_pipeline;
  if (!p) return RMP_ERR_NO_MEMORY;
  p->ctx = ctx;
  p->device = rmp::ctx_device(ctx);
  p->max_points = max_points;
  p->slots.resize(slots);
  int st = RMP_OK;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(p->device) != cudaSuccess)
    st = RMP_ERR_CUDA;
  if (st == RMP_OK && (cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking) != cudaSuccess))
    st = RMP_ERR_CUDA;
  const size_t wsb = rmp_workspace_bytes();
  for (ScanSlot& s : p->slots) {
    if (st != RMP_OK) break;
    if (cudaMalloc((void**)&s.pts, 12 * (size_t)max_points) != cudaSuccess ||
        cudaMalloc(&s.ws, wsb) != cudaSuccess ||
        cudaMalloc((void**)&s.state, 6 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&s.res, sizeof(rmp_result_t)) != cudaSuccess ||
        cudaMallocHost((void**)&s.state_host, 6 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&s.res_host, sizeof(rmp_result_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
        rmp::workspace_reset(s.ws, p->compute) != cudaSuccess)
      st = RMP_ERR_NO_MEMORY;
  }
  if (st != RMP_OK) {
    for (ScanSlot& s : p->slots) {
      if (s.pts) cudaFree(s.pts);
      if (s.ws) cudaFree(s.ws);
      if (s.state) cudaFree(s.state);
      if (s.res) cudaFree(s.res);
      if (s.state_host) cudaFreeHost(s.state_host);
      if (s.res_host) cudaFreeHost(s.res_host);
      if (s.copied) cudaEventDestroy(s.copied);
      if (s.done) cudaEventDestroy(s.done);
    }
    if (p->copy) cudaStreamDestroy(p->copy);
    if (p->compute) cudaStreamDestroy(p->compute);
    delete p;
  } else {
    *out = p;
  }
  cudaSetDevice(prev);
  return st;
}

int rmp_scan_pipeline_destroy(rmp_scan_pipeline* p) {
  if (!p) return RMP_ERR_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->copy);
  cudaStreamSynchronize(p->compute);
  for (ScanSlot& s : p->slots) {
    cudaFree(s.pts);
    cudaFree(s.ws);
    cudaFree(s.state);
    cudaFree(s.res);
    cudaFreeHost(s.state_host);
    cudaFreeHost(s.res_host);
    cudaEventDestroy(s.copied);
    cudaEventDestroy(s.done);
  }
  cudaStreamDestroy(p->copy);
  cudaStreamDestroy(p->compute);
  cudaSetDevice(prev);
  delete p;
  return RMP_OK;
}

int rmp_scan_pipeline_submit(rmp_scan_pipeline* p, const float* points_host, uint32_t n,
                             const double x[3], const double xdot[3], const rmp_params_t* params,
                             uint64_t* ticket) {
  if (!p || !points_host || !x || !xdot || !params || !ticket || n == 0 || n > p->max_points)
    return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(p->device) != cudaSuccess)
    return RMP_ERR_CUDA;
  const uint64_t t = p->next;
  ScanSlot& s = p->slots[(t - 1) % p->slots.size()];
  int st = RMP_OK;
  // the slot's previous scan must be done before its buffers are reused
  if (s.used && cudaEventSynchronize(s.done) != cudaSuccess) st = RMP_ERR_CUDA;
  if (st == RMP_OK) {
    for (int a = 0; a < 3; ++a) {
      s.state_host[a] = x[a];
      s.state_host[3 + a] = xdot[a];
    }
    if (cudaMemcpyAsync(s.pts, points_host, 12 * (size_t)n, cudaMemcpyHostToDevice, p->copy) !=
            cudaSuccess ||
        cudaMemcpyAsync(s.state, s.state_host, 6 * sizeof(double), cudaMemcpyHostToDevice,
                        p->copy) != cudaSuccess ||
        cudaEventRecord(s.copied, p->copy) != cudaSuccess ||
        cudaStreamWaitEvent(p->compute, s.copied, 0) != cudaSuccess)
      st = RMP_ERR_CUDA;
  }
  if (st == RMP_OK)
    st = rmp_scan_eval_async(p->ctx, s.pts, n, s.state, params, s.ws, rmp_workspace_bytes(),
                             p->compute, s.res, nullptr);
  if (st == RMP_OK &&
      (cudaMemcpyAsync(s.res_host, s.res, sizeof(rmp_result_t), cudaMemcpyDeviceToHost,
                       p->compute) != cudaSuccess ||
       cudaEventRecord(s.done, p->compute) != cudaSuccess))
    st = RMP_ERR_CUDA;
  cudaSetDevice(prev);
  if (st != RMP_OK) return st;
  s.ticket = t;
  s.used = true;
  p->next = t + 1;
  *ticket = t;
  return RMP_OK;
}

int rmp_scan_pipeline_wait(rmp_scan_pipeline* p, uint64_t ticket, rmp_result_t* out) {
  if (!p || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  if (ticket == 0 || ticket >= p->next) return RMP_ERR_INVALID_ARG;
  ScanSlot& s = p->slots[(ticket - 1) % p->slots.size()];
  if (s.ticket != ticket) return RMP_ERR_BUSY;     // the slot has been reused since
  if (cudaEventSynchronize(s.done) != cudaSuccess) return RMP_ERR_CUDA;
  *out = *s.res_host;
  return RMP_OK;
}

}  // extern "C"
