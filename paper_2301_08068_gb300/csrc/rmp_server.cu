// rmp_server.cu -- continuous-batching request server over the batched evaluation (host
// runtime; no kernels of its own).
//
// Clients submit single-state requests (map, state, ray count, params) from any thread.  A
// worker thread keeps up to `slots` batches in flight, each on its own CUDA stream: as
// soon as a slot is free it admits the oldest pending request and every later pending
// request with the same map and parameters (FIFO order, up to max_batch_states), as long
// as the batch's device memory (workspace, states, counts, results) fits in what is left
// of the server's budget, and launches one rmp_raycast_eval_batch_async.  Batches on
// different streams overlap on the device; a finished batch (event) returns its memory
// and completes its requests, which frees room for the requests that arrived meanwhile.
// A request whose batch alone would exceed the budget is completed with
// RMP_ERR_NO_MEMORY; a CUDA error completes the batch's requests with RMP_ERR_CUDA.
// The worker sleeps whenever it can launch nothing: a host function enqueued after each
// batch marks its slot done and wakes it, as do submissions (no polling of the GPU from the
// host).  The wake-up has its own mutex and condition variable, so the host function never
// takes the server lock.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "rmp_arena.h"
#include "rmp_internal.h"

namespace rmp {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id;
  uint32_t map_id;
  uint32_t n_rays;
  rmp_params_t params;
  double state[6];
  double t_submit;
};

struct Finished {
  rmp_result_t result;
  double latency;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::atomic<bool> finished{false};   // set by the batch's host function
  rmp_server* owner = nullptr;
  std::vector<uint64_t> ids;
  std::vector<double> t_submit;
  size_t off = 0, bytes = 0;
  double* h_states = nullptr;       // pinned staging, max_batch_states entries each
  uint32_t* h_counts = nullptr;
  rmp_result_t* h_out = nullptr;
};

bool same_key(const Request& a, const Request& b) {
  return a.map_id == b.map_id && std::memcmp(&a.params, &b.params, sizeof(rmp_params_t)) == 0;
}

struct BatchBytes {
  size_t ws, states, counts, out, total;
};

BatchBytes batch_bytes(uint32_t n, uint32_t max_rays) {
  BatchBytes b;
  b.ws = batch_layout(n, max_rays).total;
  b.states = Arena::round(6 * sizeof(double) * n);
  b.counts = Arena::round(4 * (size_t)n);
  b.out = Arena::round(sizeof(rmp_result_t) * n);
  b.total = b.ws + b.states + b.counts + b.out;
  return b;
}

rmp_result_t failed_result(uint32_t n_rays, int status) {
  rmp_result_t r;
  std::memset(&r, 0, sizeof(r));
  r.n_rays = n_rays;
  r.status = status;
  return r;
}

}  // namespace
}  // namespace rmp

using namespace rmp;

struct rmp_server {
  rmp_ctx* ctx = nullptr;
  // wake-up of the worker: bumped by every event it waits for (a batch's host function, a
  // submission, stop); the worker sleeps until it changes
  std::atomic<uint64_t> wake{0};
  std::mutex wake_mu;
  std::condition_variable wake_cv;
  int device = 0;
  rmp_server_config_t cfg;
  char* arena_dev = nullptr;
  Arena* arena = nullptr;
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Finished> finished;
  std::unordered_set<uint64_t> outstanding;      // issued tickets not yet collected
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  rmp_server_stats_t stats;
};

namespace {

// Complete every request of a finished (or failed) slot and give its memory back.
void reap(rmp_server* s, Slot& sl, int status) {
  const double t = now_s();
  for (size_t i = 0; i < sl.ids.size(); ++i) {
    Finished f;
    f.result = status == RMP_OK ? sl.h_out[i] : failed_result(sl.h_counts[i], status);
    f.latency = t - sl.t_submit[i];
    s->finished[sl.ids[i]] = f;
  }
  s->stats.completed += sl.ids.size();
  s->arena->release(sl.off, sl.bytes);
  sl.busy = false;
  sl.ids.clear();
  sl.t_submit.clear();
  s->cv_done.notify_all();
}

void complete_now(rmp_server* s, const Request& r, int status) {
  Finished f;
  f.result = failed_result(r.n_rays, status);
  f.latency = now_s() - r.t_submit;
  s->finished[r.id] = f;
  s->stats.completed += 1;
  s->stats.rejected += 1;
  s->cv_done.notify_all();
}

void wake_worker(rmp_server* s) {
  s->wake.fetch_add(1, std::memory_order_acq_rel);
  { std::lock_guard<std::mutex> lk(s->wake_mu); }   // orders the bump with the worker's wait
  s->wake_cv.notify_all();
}

// Host function enqueued after a batch's result copy: marks the slot finished and wakes the
// worker.  It calls no CUDA function and takes only the wake-up mutex.
void CUDART_CB batch_done(void* arg) {
  Slot* sl = static_cast<Slot*>(arg);
  sl->finished.store(true, std::memory_order_release);
  wake_worker(sl->owner);
}

// Form and launch one batch on free slot `sl` from the pending queue.  Returns false if
// nothing could be launched (the oldest request waits for memory).
bool launch_batch_on(rmp_server* s, Slot& sl) {
  const Request first = s->pending.front();
  const uint32_t cap = s->cfg.max_batch_states;
  BatchBytes need = batch_bytes(1, first.n_rays);
  if (need.total > s->arena->size()) {           // can never fit: fail it, keep going
    s->pending.pop_front();
    complete_now(s, first, RMP_ERR_NO_MEMORY);
    return true;
  }
  const size_t room = s->arena->largest_free();
  if (need.total > room) return false;
  // members: the oldest request, then later ones with the same key while the batch fits
  std::vector<size_t> take{0};
  uint32_t max_rays = first.n_rays;
  const size_t scan = s->pending.size() < 65536 ? s->pending.size() : 65536;
  for (size_t i = 1; i < scan && take.size() < cap; ++i) {
    const Request& r = s->pending[i];
    if (!same_key(r, first)) continue;
    const uint32_t mr = r.n_rays > max_rays ? r.n_rays : max_rays;
    const BatchBytes nb = batch_bytes((uint32_t)take.size() + 1, mr);
    if (nb.total > room) break;
    take.push_back(i);
    max_rays = mr;
    need = nb;
  }
  const uint32_t n = (uint32_t)take.size();
  const size_t off = s->arena->alloc(need.total);
  if (off == Arena::kFail) return false;
  sl.off = off;
  sl.bytes = need.total;
  sl.ids.resize(n);
  sl.t_submit.resize(n);
  for (uint32_t j = 0; j < n; ++j) {
    const Request& r = s->pending[take[j]];
    sl.ids[j] = r.id;
    sl.t_submit[j] = r.t_submit;
    std::memcpy(sl.h_states + 6 * j, r.state, sizeof(r.state));
    sl.h_counts[j] = r.n_rays;
  }
  // remove the members from the queue (indices ascending)
  std::deque<Request> rest;
  size_t t = 0;
  for (size_t i = 0; i < s->pending.size(); ++i) {
    if (t < take.size() && take[t] == i) {
      ++t;
      continue;
    }
    rest.push_back(s->pending[i]);
  }
  s->pending.swap(rest);
  char* base = s->arena_dev + off;
  void* ws = base;
  double* d_states = (double*)(base + need.ws);
  uint32_t* d_counts = (uint32_t*)(base + need.ws + need.states);
  rmp_result_t* d_out = (rmp_result_t*)(base + need.ws + need.states + need.counts);
  sl.busy = true;
  s->stats.batches += 1;
  s->stats.batched_states += n;
  cudaError_t e = cudaMemcpyAsync(d_states, sl.h_states, 6 * sizeof(double) * n,
                                  cudaMemcpyHostToDevice, sl.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_counts, sl.h_counts, 4 * (size_t)n, cudaMemcpyHostToDevice, sl.stream);
  int st = e == cudaSuccess ? RMP_OK : RMP_ERR_CUDA;
  if (st == RMP_OK)
    st = rmp_raycast_eval_batch_async(s->ctx, first.map_id, d_states, d_counts, n, max_rays,
                                      &first.params, ws, need.ws, sl.stream, d_out, nullptr,
                                      nullptr);
  if (st == RMP_OK &&
      cudaMemcpyAsync(sl.h_out, d_out, sizeof(rmp_result_t) * n, cudaMemcpyDeviceToHost,
                      sl.stream) != cudaSuccess)
    st = RMP_ERR_CUDA;
  if (st == RMP_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = RMP_ERR_CUDA;
  sl.finished.store(false, std::memory_order_relaxed);
  if (st == RMP_OK && cudaLaunchHostFunc(sl.stream, batch_done, &sl) != cudaSuccess)
    st = RMP_ERR_CUDA;
  if (st != RMP_OK) {
    // nothing usable was enqueued after the failure: wait for what was, then fail the batch
    cudaStreamSynchronize(sl.stream);
    reap(s, sl, st);
    s->stats.rejected += n;
    return true;
  }
  uint32_t inflight = 0;
  for (const Slot& o : s->slots) inflight += o.busy ? 1u : 0u;
  if (inflight > s->stats.max_inflight) s->stats.max_inflight = inflight;
  if (s->arena->high_water() > s->stats.mem_high_water) s->stats.mem_high_water = s->arena->high_water();
  return true;
}

void worker_main(rmp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    const uint64_t seen = s->wake.load(std::memory_order_acquire);
    bool progress = false;
    bool busy = false;
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      if (!sl.finished.load(std::memory_order_acquire)) {
        busy = true;
        continue;
      }
      // the host function ran after the batch's last operation: the event has completed,
      // and its status carries any error of the batch
      const cudaError_t q = cudaEventQuery(sl.done);
      reap(s, sl, q == cudaSuccess ? RMP_OK : RMP_ERR_CUDA);
      progress = true;
    }
    while (!s->pending.empty()) {
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (!sl.busy) {
          free_slot = &sl;
          break;
        }
      if (!free_slot || !launch_batch_on(s, *free_slot)) break;
      progress = true;
      busy = busy || free_slot->busy;
    }
    for (const Slot& sl : s->slots) busy = busy || sl.busy;
    if (s->stop && s->pending.empty() && !busy) break;
    if (progress) continue;
    // nothing to launch or reap: sleep, without the server lock, until a batch's host
    // function, a submission or stop bumps the wake-up count; the timed wait is a backstop
    // only (a host function that never ran would otherwise stall the server)
    lk.unlock();
    bool woken;
    {
      std::unique_lock<std::mutex> wl(s->wake_mu);
      woken = s->wake_cv.wait_for(wl, std::chrono::milliseconds(50), [s, seen] {
        return s->wake.load(std::memory_order_acquire) != seen;
      });
    }
    lk.lock();
    if (!woken) {
      for (Slot& sl : s->slots)                    // backstop: look at the events directly
        if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess)
          sl.finished.store(true, std::memory_order_release);
    }
  }
}

}  // namespace

extern "C" {

int rmp_server_config_default(rmp_server_config_t* cfg) {
  if (!cfg) return RMP_ERR_INVALID_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->slots = 4;
  cfg->max_batch_states = 256;
  cfg->max_rays = 262144;
  cfg->mem_budget_bytes = 1ull << 30;
  return RMP_OK;
}

int rmp_server_create(rmp_ctx* ctx, const rmp_server_config_t* cfg, rmp_server** out) {
  if (!ctx || !cfg || !out) return RMP_ERR_INVALID_ARG;
  if (cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch_states < 1 ||
      cfg->max_batch_states > kMaxBatchStates || cfg->max_rays < 1 ||
      cfg->mem_budget_bytes < Arena::kAlign)
    return RMP_ERR_INVALID_ARG;
  rmp_server* s = new (std::nothrow) rmp_server;
  if (!s) return RMP_ERR_NO_MEMORY;
  s->ctx = ctx;
  s->device = ctx_device(ctx);
  s->cfg = *cfg;
  std::memset(&s->stats, 0, sizeof(s->stats));
  int st = RMP_OK;
  if (cudaSetDevice(s->device) != cudaSuccess) st = RMP_ERR_CUDA;
  if (st == RMP_OK && cudaMalloc((void**)&s->arena_dev, cfg->mem_budget_bytes) != cudaSuccess)
    st = RMP_ERR_NO_MEMORY;
  s->slots = std::vector<Slot>(cfg->slots);
  for (Slot& sl : s->slots) {
    sl.owner = s;
    if (st != RMP_OK) break;
    const size_t n = cfg->max_batch_states;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&sl.h_states, 6 * sizeof(double) * n) != cudaSuccess ||
        cudaMallocHost((void**)&sl.h_counts, 4 * n) != cudaSuccess ||
        cudaMallocHost((void**)&sl.h_out, sizeof(rmp_result_t) * n) != cudaSuccess)
      st = RMP_ERR_CUDA;
  }
  if (st == RMP_OK) {
    s->arena = new (std::nothrow) Arena(cfg->mem_budget_bytes);
    if (!s->arena) st = RMP_ERR_NO_MEMORY;
  }
  if (st == RMP_OK) {
    try {
      s->worker = std::thread(worker_main, s);
    } catch (...) {
      st = RMP_ERR_NO_MEMORY;
    }
  }
  if (st != RMP_OK) {
    for (Slot& sl : s->slots) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.h_states) cudaFreeHost(sl.h_states);
      if (sl.h_counts) cudaFreeHost(sl.h_counts);
      if (sl.h_out) cudaFreeHost(sl.h_out);
    }
    if (s->arena_dev) cudaFree(s->arena_dev);
    delete s->arena;
    delete s;
    return st;
  }
  *out = s;
  return RMP_OK;
}

int rmp_server_destroy(rmp_server* s) {
  if (!s) return RMP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  wake_worker(s);
  if (s->worker.joinable()) s->worker.join();     // drains pending and in-flight work
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
    cudaFreeHost(sl.h_states);
    cudaFreeHost(sl.h_counts);
    cudaFreeHost(sl.h_out);
  }
  cudaFree(s->arena_dev);
  delete s->arena;
  delete s;
  return RMP_OK;
}

int rmp_server_submit(rmp_server* s, uint32_t map_id, const double x[3], const double xdot[3],
                      uint32_t n_rays, const rmp_params_t* params, uint64_t* ticket) {
  if (!s || !x || !xdot || !params || !ticket || n_rays == 0 || n_rays > s->cfg.max_rays)
    return RMP_ERR_INVALID_ARG;
  Request r;
  r.map_id = map_id;
  r.n_rays = n_rays;
  r.params = *params;
  for (int a = 0; a < 3; ++a) {
    r.state[a] = x[a];
    r.state[3 + a] = xdot[a];
  }
  r.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return RMP_ERR_BUSY;
    r.id = s->next_id++;
    s->pending.push_back(r);
    s->outstanding.insert(r.id);
    s->stats.submitted += 1;
  }
  wake_worker(s);
  *ticket = r.id;
  return RMP_OK;
}

int rmp_server_poll(rmp_server* s, uint64_t ticket, rmp_result_t* out, double* latency_s) {
  if (!s || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->outstanding.count(ticket)) return RMP_ERR_INVALID_ARG;   // never issued or collected
  auto it = s->finished.find(ticket);
  if (it == s->finished.end()) return RMP_ERR_NOT_READY;
  *out = it->second.result;
  if (latency_s) *latency_s = it->second.latency;
  s->finished.erase(it);
  s->outstanding.erase(ticket);
  return RMP_OK;
}

int rmp_server_wait(rmp_server* s, uint64_t ticket, uint32_t timeout_ms, rmp_result_t* out,
                    double* latency_s) {
  if (!s || !out) return RMP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    // never issued, or collected (also by another thread while this one waited)
    if (!s->outstanding.count(ticket)) return RMP_ERR_INVALID_ARG;
    auto it = s->finished.find(ticket);
    if (it != s->finished.end()) {
      *out = it->second.result;
      if (latency_s) *latency_s = it->second.latency;
      s->finished.erase(it);
      s->outstanding.erase(ticket);
      return RMP_OK;
    }
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->finished.find(ticket) == s->finished.end())
      return RMP_ERR_TIMEOUT;
  }
}

int rmp_server_stats(rmp_server* s, rmp_server_stats_t* out) {
  if (!s || !out) return RMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->pending = s->pending.size();
  return RMP_OK;
}

}  // extern "C"
