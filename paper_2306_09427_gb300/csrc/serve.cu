// Continuous-batching request loop over an RVE batch.
//
// The paper's RVE batch manager (Sec. 4.3) marshals the deformation
// increments of a macroscale iteration into one batched microscale solve.
// Here requests (rve id, F) arrive one by one, as from many macroscale
// Newton iterations in flight, and are served without waiting for a whole
// batch to finish:
//   * requests wait in a FIFO queue on the host;
//   * the server owns n_slots CUDA streams; whenever a slot is free, it
//     takes up to max_wave queued requests (skipping RVEs that are already
//     on the GPU, so each RVE's warm-start state is updated by one solve at
//     a time) and launches them as one wave (rve_solve_subset on the slot's
//     stream, inputs and outputs staged through pinned buffers);
//   * waves on different slots overlap on the device; a finished wave is
//     detected by its event and its results become available to poll;
//   * latency = completion detected - request submitted (host clock).
// Admission: the batch and the server's buffers must fit under the HBM
// byte cap given at creation (RVE_EADMIT otherwise).
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include "batch.h"

namespace rvegpu {
namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t rve;
  int64_t tag;
  double F[9];
  clk::time_point t0;
};

struct Done {
  int64_t tag;
  double sigma[9];
  int32_t iters, status;
  double latency;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double *dF = nullptr, *dS = nullptr;
  int32_t *dI = nullptr, *dSt = nullptr;
  double *hF = nullptr, *hS = nullptr;
  int32_t *hI = nullptr, *hSt = nullptr;
  std::vector<Request> reqs;
  std::vector<int64_t> ids;
  SubsetBuffers work;  // this slot's own work lists: waves in flight share nothing mutable
  bool busy = false;
};

}  // namespace
}  // namespace rvegpu

struct rve_server {
  rve_batch* b = nullptr;
  int max_wave = 0;
  std::vector<rvegpu::Slot> slots;
  std::deque<rvegpu::Request> queue;
  std::deque<rvegpu::Done> done;
  std::vector<uint8_t> on_gpu;  // per RVE
  int64_t completed = 0, waves = 0;
  size_t device_bytes = 0;
};

using namespace rvegpu;

namespace {

int retire(rve_server* s, Slot& sl) {
  const cudaError_t q = cudaEventQuery(sl.done);
  if (q == cudaErrorNotReady) return RVE_OK;
  if (q != cudaSuccess) return fail(RVE_ECUDA, std::string("wave failed: ") + cudaGetErrorString(q));
  const auto now = clk::now();
  for (size_t k = 0; k < sl.reqs.size(); ++k) {
    Done d;
    d.tag = sl.reqs[k].tag;
    std::memcpy(d.sigma, sl.hS + 9 * k, sizeof(d.sigma));
    d.iters = sl.hI[k];
    d.status = sl.hSt[k];
    d.latency = std::chrono::duration<double>(now - sl.reqs[k].t0).count();
    s->done.push_back(d);
    s->on_gpu[sl.reqs[k].rve] = 0;
  }
  s->completed += int64_t(sl.reqs.size());
  sl.reqs.clear();
  sl.busy = false;
  return RVE_OK;
}

int launch(rve_server* s, Slot& sl) {
  sl.reqs.clear();
  sl.ids.clear();
  // FIFO order, but an RVE already on the GPU (or already in this wave) waits
  std::deque<Request> keep;
  while (!s->queue.empty() && int(sl.reqs.size()) < s->max_wave) {
    Request r = s->queue.front();
    s->queue.pop_front();
    if (s->on_gpu[r.rve]) {
      keep.push_back(r);
      continue;
    }
    s->on_gpu[r.rve] = 1;
    sl.reqs.push_back(r);
  }
  while (!keep.empty()) {
    s->queue.push_front(keep.back());
    keep.pop_back();
  }
  if (sl.reqs.empty()) return RVE_OK;
  const size_t m = sl.reqs.size();
  for (size_t k = 0; k < m; ++k) {
    std::memcpy(sl.hF + 9 * k, sl.reqs[k].F, 9 * sizeof(double));
    sl.ids.push_back(sl.reqs[k].rve);
  }
  RVE_CUDA_TRY(cudaStreamWaitEvent(sl.stream, s->b->ev_last, 0));  // after the batch's last public call
  RVE_CUDA_TRY(cudaMemcpyAsync(sl.dF, sl.hF, 9 * m * sizeof(double), cudaMemcpyHostToDevice, sl.stream));
  const int rc =
      solve_subset(s->b, sl.ids.data(), int64_t(m), sl.dF, 0.0, 0, sl.dS, sl.dI, sl.dSt, sl.stream, false, &sl.work);
  if (rc != RVE_OK) return rc;
  RVE_CUDA_TRY(cudaMemcpyAsync(sl.hS, sl.dS, 9 * m * sizeof(double), cudaMemcpyDeviceToHost, sl.stream));
  RVE_CUDA_TRY(cudaMemcpyAsync(sl.hI, sl.dI, m * sizeof(int32_t), cudaMemcpyDeviceToHost, sl.stream));
  RVE_CUDA_TRY(cudaMemcpyAsync(sl.hSt, sl.dSt, m * sizeof(int32_t), cudaMemcpyDeviceToHost, sl.stream));
  RVE_CUDA_TRY(cudaEventRecord(sl.done, sl.stream));
  sl.busy = true;
  s->waves++;
  return RVE_OK;
}

}  // namespace

extern "C" {

void rve_server_destroy(rve_server* s) {
  if (!s) return;
  cudaSetDevice(s->b->device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFree(sl.dF);
    cudaFree(sl.dS);
    cudaFree(sl.dI);
    cudaFree(sl.dSt);
    cudaFreeHost(sl.hF);
    cudaFreeHost(sl.hS);
    cudaFreeHost(sl.hI);
    cudaFreeHost(sl.hSt);
    cudaFree(sl.work.d_work);
    cudaFree(sl.work.d_sorted);
    cudaFreeHost(sl.work.h_stage);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

int rve_server_create(rve_server** out, rve_batch* b, int32_t n_slots, int32_t max_wave, double hbm_cap_bytes) {
  if (!out || !b) return fail(RVE_EINVAL, "null argument");
  *out = nullptr;
  if (n_slots < 1 || n_slots > 64) return fail(RVE_EINVAL, "n_slots must be in 1..64");
  if (max_wave < 1) return fail(RVE_EINVAL, "max_wave must be >= 1");
  if (b->opt.precision == RVE_PREC_PLAIN_F64 && n_slots > 1)
    return fail(RVE_EINVAL, "the plain FP64 path shares one scratch area: use n_slots = 1");
  const size_t per_slot = size_t(max_wave) * (18 * sizeof(double) + 2 * sizeof(int32_t) + 2 * sizeof(Work));
  const double need = double(b->device_bytes) + double(per_slot) * n_slots;
  if (hbm_cap_bytes > 0.0 && need > hbm_cap_bytes)
    return fail(RVE_EADMIT, "batch and server buffers need " + std::to_string(need / 1e9) + " GB, over the cap of " +
                                std::to_string(hbm_cap_bytes / 1e9) + " GB");
  RVE_CUDA_TRY(cudaSetDevice(b->device));
  rve_server* s = new rve_server();
  s->b = b;
  s->max_wave = max_wave;
  s->on_gpu.assign(size_t(b->n_rve), 0);
  s->slots.resize(n_slots);
  for (Slot& sl : s->slots) {
    const size_t m = size_t(max_wave);
    bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&sl.dF, 9 * m * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&sl.dS, 9 * m * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&sl.dI, m * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&sl.dSt, m * sizeof(int32_t)) == cudaSuccess &&
              cudaMallocHost(&sl.hF, 9 * m * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&sl.hS, 9 * m * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&sl.hI, m * sizeof(int32_t)) == cudaSuccess &&
              cudaMallocHost(&sl.hSt, m * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&sl.work.d_work, m * sizeof(Work)) == cudaSuccess &&
              cudaMalloc(&sl.work.d_sorted, m * sizeof(Work)) == cudaSuccess &&
              cudaMallocHost(&sl.work.h_stage, m * sizeof(Work)) == cudaSuccess;
    sl.work.cap = m;
    if (!ok) {
      (void)cudaGetLastError();
      rve_server_destroy(s);
      return fail(RVE_ENOMEM, "server buffer allocation failed");
    }
    s->device_bytes += per_slot;
  }
  *out = s;
  return RVE_OK;
}

int rve_server_submit(rve_server* s, int64_t rve_id, const double* F, int64_t tag) {
  if (!s || !F) return fail(RVE_EINVAL, "null argument");
  if (rve_id < 0 || rve_id >= s->b->n_rve) return fail(RVE_EINVAL, "rve_id out of range");
  Request r;
  r.rve = rve_id;
  r.tag = tag;
  std::memcpy(r.F, F, sizeof(r.F));
  r.t0 = clk::now();
  s->queue.push_back(r);
  return RVE_OK;
}

int rve_server_step(rve_server* s) {
  if (!s) return fail(RVE_EINVAL, "null server");
  RVE_CUDA_TRY(cudaSetDevice(s->b->device));
  for (Slot& sl : s->slots)
    if (sl.busy) {
      const int rc = retire(s, sl);
      if (rc != RVE_OK) return rc;
    }
  for (Slot& sl : s->slots) {
    if (s->queue.empty()) break;
    if (!sl.busy) {
      const int rc = launch(s, sl);
      if (rc != RVE_OK) return rc;
    }
  }
  return RVE_OK;
}

int rve_server_drain(rve_server* s) {
  if (!s) return fail(RVE_EINVAL, "null server");
  for (;;) {
    bool busy = false;
    for (Slot& sl : s->slots)
      if (sl.busy) {
        RVE_CUDA_TRY(cudaEventSynchronize(sl.done));
        busy = true;
      }
    const int rc = rve_server_step(s);
    if (rc != RVE_OK) return rc;
    if (!busy && s->queue.empty()) return RVE_OK;
  }
}

int64_t rve_server_poll(rve_server* s, int64_t max, int64_t* tags, double* sigma, int32_t* iters, int32_t* status,
                        double* latency_s) {
  if (!s || max < 0) return fail(RVE_EINVAL, "bad poll arguments");
  int64_t n = 0;
  while (n < max && !s->done.empty()) {
    const Done& d = s->done.front();
    if (tags) tags[n] = d.tag;
    if (sigma) std::memcpy(sigma + 9 * n, d.sigma, sizeof(d.sigma));
    if (iters) iters[n] = d.iters;
    if (status) status[n] = d.status;
    if (latency_s) latency_s[n] = d.latency;
    s->done.pop_front();
    ++n;
  }
  return n;
}

int rve_server_get_stats(const rve_server* s, rve_server_stats* st) {
  if (!s || !st) return fail(RVE_EINVAL, "null argument");
  st->queued = int64_t(s->queue.size());
  int64_t inflight = 0;
  for (const Slot& sl : s->slots) inflight += sl.busy ? int64_t(sl.reqs.size()) : 0;
  st->in_flight = inflight;
  st->completed = s->completed;
  st->ready = int64_t(s->done.size());
  st->waves = s->waves;
  st->device_bytes = int64_t(s->device_bytes);
  return RVE_OK;
}

}  // extern "C"
