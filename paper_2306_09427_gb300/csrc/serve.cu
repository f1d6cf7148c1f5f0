// Continuous-batching request loop over a resident, growable pool of RVEs.
//
// The paper's RVE batch manager (Sec. 4.3) marshals the deformation
// increments of a macroscale iteration into one batched microscale solve.
// Here requests (rve id, F) arrive one by one, as from many macroscale
// Newton iterations in flight, and are served at the granularity of DR
// iterations:
//   * requests wait in a FIFO queue on the host;
//   * the server owns n_slots wave groups, each a CUDA stream with up to
//     max_wave request slots; a group launches one wave at a time, and a
//     wave advances every occupied slot by wave_iters DR iterations (the
//     fused kernel parks an unfinished solve: state h, velocity and loop
//     scalars stay on the device, Algorithm 2 resumes where it stopped);
//   * between two waves of a group, finished requests retire (their
//     results become available to poll) and queued requests take the free
//     slots, so a long solve never holds up the short ones behind it;
//     groups overlap on the device;
//   * an RVE is in at most one slot at a time, so its warm-start state is
//     advanced by one request at a time; every request's DR trajectory
//     depends only on its own F, its start state and the wave length, so
//     its result is bit-identical alone and in any mix;
//   * latency = completion detected - request submitted (host clock).
// wave_iters = 0 runs each request to the end within its first wave.
//
// Pool and admission: segment 0 is the batch given at creation; more RVE
// topologies are admitted at run time (rve_server_add_rves) as further
// segments when their device footprint fits under the HBM byte cap
// (RVE_EADMIT otherwise), and an idle segment can be removed to free its
// memory.  Global RVE ids are assigned in admission order and never reused.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include "batch.h"

namespace rvegpu {
namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t id;     // global RVE id
  int seg;        // segment index
  int64_t local;  // RVE index inside the segment's batch
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

struct Segment {
  rve_batch* b = nullptr;
  bool owned = false;    // admitted by rve_server_add_rves (removable)
  bool live = true;
  int64_t first = 0;     // global id of the segment's RVE 0
  int64_t n = 0;
  int64_t busy = 0;      // requests queued or in flight
  size_t bytes = 0;      // device bytes charged to the cap
  ResumeRec* d_resume = nullptr;
  void* d_vel = nullptr;
};

struct Group {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int cap = 0;
  double *dF = nullptr, *dS = nullptr;
  int32_t *dI = nullptr, *dSt = nullptr;
  double *hF = nullptr, *hS = nullptr;
  int32_t *hI = nullptr, *hSt = nullptr;
  std::vector<Request> slot;
  std::vector<uint8_t> used;
  std::vector<uint8_t> fresh;          // slot filled since the last wave (its F not yet uploaded)
  int n_used = 0;
  bool busy = false;
  std::vector<SubsetBuffers> work;     // per segment: work lists of this group's waves
  std::vector<int64_t> ids;
  std::vector<int32_t> outs;
};

size_t group_bytes(int cap) {
  return size_t(cap) * (18 * sizeof(double) + 2 * sizeof(int32_t));
}
size_t work_bytes(int cap) { return 2 * size_t(cap) * sizeof(Work); }

}  // namespace
}  // namespace rvegpu

struct rve_server {
  int device = 0;
  int precision = RVE_PREC_MIXED;
  rve_options opt{};
  int max_wave = 0;
  int32_t wave_iters = 0;
  double cap_bytes = 0.0;
  std::vector<rvegpu::Segment> segs;
  std::vector<rvegpu::Group> groups;
  std::deque<rvegpu::Request> queue;
  std::deque<rvegpu::Done> done;
  std::vector<uint8_t> on_gpu;  // per global id
  int64_t next_id = 0;
  int64_t completed = 0, waves = 0;
  size_t buffer_bytes = 0;      // the groups' own buffers
  size_t pool_bytes = 0;        // segments (batches + resume state)
};

using namespace rvegpu;

namespace {

int find_segment(const rve_server* s, int64_t id, int* seg, int64_t* local) {
  for (size_t k = 0; k < s->segs.size(); ++k) {
    const Segment& g = s->segs[k];
    if (g.live && id >= g.first && id < g.first + g.n) {
      *seg = int(k);
      *local = id - g.first;
      return RVE_OK;
    }
  }
  return fail(RVE_EINVAL, "rve_id " + std::to_string(id) + " is not in the pool");
}

void free_work(SubsetBuffers& w) {
  if (w.d_work) cudaFree(w.d_work);
  if (w.d_sorted) cudaFree(w.d_sorted);
  if (w.h_stage) cudaFreeHost(w.h_stage);
  w = SubsetBuffers{};
}

// Resume records and velocities of a segment, and the batched path of its
// precision; returns the device bytes the segment holds.
int attach_segment(rve_server* s, Segment& g) {
  for (Group& gr : s->groups) gr.work.emplace_back();  // this segment's work-list slot in every group
  const int rc = ensure_batched_path(g.b);
  if (rc != RVE_OK) return rc;
  const size_t vel_elem = s->precision == RVE_PREC_MIXED ? sizeof(float) : sizeof(double);
  const size_t n_rec = size_t(std::max<int64_t>(g.n, 1)) * sizeof(ResumeRec);
  const size_t n_vel = 4 * vel_elem * size_t(std::max<int64_t>(g.b->total_nf, 1));
  if (cudaMalloc(reinterpret_cast<void**>(&g.d_resume), n_rec) != cudaSuccess ||
      cudaMalloc(&g.d_vel, n_vel) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(RVE_ENOMEM, "server resume buffers: cudaMalloc failed");
  }
  RVE_CUDA_TRY(cudaMemset(g.d_resume, 0, n_rec));
  RVE_CUDA_TRY(cudaMemset(g.d_vel, 0, n_vel));
  g.bytes = g.b->device_bytes + n_rec + n_vel;
  return RVE_OK;
}

void release_segment(rve_server* s, size_t k) {
  Segment& g = s->segs[k];
  for (Group& gr : s->groups)
    if (k < gr.work.size()) free_work(gr.work[k]);
  if (g.d_resume) cudaFree(g.d_resume);
  if (g.d_vel) cudaFree(g.d_vel);
  g.d_resume = nullptr;
  g.d_vel = nullptr;
  if (g.owned && g.b) rve_batch_destroy(g.b);
  g.b = nullptr;
  g.live = false;
}

int ensure_work(rve_server* s, Group& gr, size_t seg) {
  SubsetBuffers& w = gr.work[seg];
  if (w.cap >= size_t(gr.cap)) return RVE_OK;
  const size_t m = size_t(gr.cap);
  if (cudaMalloc(&w.d_work, m * sizeof(Work)) != cudaSuccess ||
      cudaMalloc(&w.d_sorted, m * sizeof(Work)) != cudaSuccess ||
      cudaMallocHost(&w.h_stage, m * sizeof(Work)) != cudaSuccess) {
    (void)cudaGetLastError();
    free_work(w);
    return fail(RVE_ENOMEM, "server work buffers: allocation failed");
  }
  w.cap = m;
  s->buffer_bytes += work_bytes(gr.cap);
  return RVE_OK;
}

// A finished wave: retire the slots whose solve ended; parked ones stay.
int retire(rve_server* s, Group& gr) {
  const cudaError_t q = cudaEventQuery(gr.done);
  if (q == cudaErrorNotReady) return RVE_OK;
  if (q != cudaSuccess) return fail(RVE_ECUDA, std::string("wave failed: ") + cudaGetErrorString(q));
  const auto now = clk::now();
  for (int k = 0; k < gr.cap; ++k) {
    if (!gr.used[k] || gr.hSt[k] == RVE_STATUS_RUNNING) continue;
    const Request& r = gr.slot[k];
    Done d;
    d.tag = r.tag;
    std::memcpy(d.sigma, gr.hS + 9 * size_t(k), sizeof(d.sigma));
    d.iters = gr.hI[k];
    d.status = gr.hSt[k];
    d.latency = std::chrono::duration<double>(now - r.t0).count();
    s->done.push_back(d);
    s->on_gpu[r.id] = 0;
    s->segs[r.seg].busy--;
    gr.used[k] = 0;
    gr.n_used--;
    s->completed++;
  }
  gr.busy = false;
  return RVE_OK;
}

// Fill free slots from the queue (FIFO; an RVE already in a slot waits),
// then launch one wave over the occupied slots.
int launch(rve_server* s, Group& gr) {
  std::deque<Request> keep;
  int k = 0;
  while (!s->queue.empty() && gr.n_used < gr.cap) {
    Request r = s->queue.front();
    s->queue.pop_front();
    if (s->on_gpu[r.id]) {
      keep.push_back(r);
      continue;
    }
    while (gr.used[k]) ++k;
    s->on_gpu[r.id] = 1;
    gr.slot[k] = r;
    gr.used[k] = 1;
    gr.fresh[k] = 1;
    gr.n_used++;
    std::memcpy(gr.hF + 9 * size_t(k), r.F, 9 * sizeof(double));
  }
  while (!keep.empty()) {
    s->queue.push_front(keep.back());
    keep.pop_back();
  }
  if (gr.n_used == 0) return RVE_OK;
  int hi = 0, lo = gr.cap, fresh_lo = gr.cap, fresh_hi = -1;
  for (int j = 0; j < gr.cap; ++j) {
    if (!gr.used[j]) continue;
    lo = std::min(lo, j);
    hi = j;
    if (gr.fresh[j]) {
      fresh_lo = std::min(fresh_lo, j);
      fresh_hi = j;
      gr.fresh[j] = 0;
    }
  }
  // this group's waves run after the last public call's GPU work on each batch
  for (const Segment& g : s->segs)
    if (g.live && g.busy > 0) RVE_CUDA_TRY(cudaStreamWaitEvent(gr.stream, g.b->ev_last, 0));
  if (fresh_hi >= 0)
    RVE_CUDA_TRY(cudaMemcpyAsync(gr.dF + 9 * size_t(fresh_lo), gr.hF + 9 * size_t(fresh_lo),
                                 9 * sizeof(double) * size_t(fresh_hi - fresh_lo + 1), cudaMemcpyHostToDevice,
                                 gr.stream));
  for (size_t sg = 0; sg < s->segs.size(); ++sg) {
    Segment& g = s->segs[sg];
    if (!g.live || g.busy == 0) continue;
    gr.ids.clear();
    gr.outs.clear();
    for (int j = lo; j <= hi; ++j)
      if (gr.used[j] && gr.slot[j].seg == int(sg)) {
        gr.ids.push_back(gr.slot[j].local);
        gr.outs.push_back(int32_t(j));
      }
    if (gr.ids.empty()) continue;
    const int rw = ensure_work(s, gr, sg);
    if (rw != RVE_OK) return rw;
    WaveParams wp;
    wp.wave_iters = s->wave_iters;
    wp.resume = g.d_resume;
    wp.vel = g.d_vel;
    const int rc = solve_items(g.b, gr.ids.data(), gr.outs.data(), int64_t(gr.ids.size()), gr.dF, 0.0, 0, gr.dS,
                               gr.dI, gr.dSt, gr.stream, false, &gr.work[sg], &wp);
    if (rc != RVE_OK) return rc;
  }
  const size_t n = size_t(hi - lo + 1);
  RVE_CUDA_TRY(cudaMemcpyAsync(gr.hS + 9 * size_t(lo), gr.dS + 9 * size_t(lo), 9 * n * sizeof(double),
                               cudaMemcpyDeviceToHost, gr.stream));
  RVE_CUDA_TRY(cudaMemcpyAsync(gr.hI + lo, gr.dI + lo, n * sizeof(int32_t), cudaMemcpyDeviceToHost, gr.stream));
  RVE_CUDA_TRY(cudaMemcpyAsync(gr.hSt + lo, gr.dSt + lo, n * sizeof(int32_t), cudaMemcpyDeviceToHost, gr.stream));
  RVE_CUDA_TRY(cudaEventRecord(gr.done, gr.stream));
  gr.busy = true;
  s->waves++;
  return RVE_OK;
}

bool any_busy(const rve_server* s) {
  for (const Group& gr : s->groups)
    if (gr.busy || gr.n_used > 0) return true;
  return false;
}

}  // namespace

extern "C" {

void rve_server_destroy(rve_server* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  for (Group& gr : s->groups)
    if (gr.stream) cudaStreamSynchronize(gr.stream);
  for (size_t k = 0; k < s->segs.size(); ++k)
    if (s->segs[k].live) release_segment(s, k);
  for (Group& gr : s->groups) {
    cudaFree(gr.dF);
    cudaFree(gr.dS);
    cudaFree(gr.dI);
    cudaFree(gr.dSt);
    cudaFreeHost(gr.hF);
    cudaFreeHost(gr.hS);
    cudaFreeHost(gr.hI);
    cudaFreeHost(gr.hSt);
    for (SubsetBuffers& w : gr.work) free_work(w);
    if (gr.done) cudaEventDestroy(gr.done);
    if (gr.stream) cudaStreamDestroy(gr.stream);
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
  RVE_CUDA_TRY(cudaSetDevice(b->device));
  // admission of the base batch and the server's own buffers, before allocating them
  const double buffers = double(group_bytes(max_wave)) * n_slots;
  if (hbm_cap_bytes > 0.0 && double(b->device_bytes) + buffers > hbm_cap_bytes)
    return fail(RVE_EADMIT, "batch and server buffers need " + std::to_string((b->device_bytes + buffers) / 1e9) +
                                " GB, over the cap of " + std::to_string(hbm_cap_bytes / 1e9) + " GB");
  rve_server* s = new rve_server();
  s->device = b->device;
  s->precision = b->opt.precision;
  s->opt = b->opt;
  s->max_wave = max_wave;
  s->cap_bytes = hbm_cap_bytes;
  s->groups.resize(n_slots);
  for (Group& gr : s->groups) {
    const size_t m = size_t(max_wave);
    gr.cap = max_wave;
    gr.slot.resize(m);
    gr.used.assign(m, 0);
    gr.fresh.assign(m, 0);
    const bool ok = cudaStreamCreateWithFlags(&gr.stream, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&gr.done, cudaEventDisableTiming) == cudaSuccess &&
                    cudaMalloc(&gr.dF, 9 * m * sizeof(double)) == cudaSuccess &&
                    cudaMalloc(&gr.dS, 9 * m * sizeof(double)) == cudaSuccess &&
                    cudaMalloc(&gr.dI, m * sizeof(int32_t)) == cudaSuccess &&
                    cudaMalloc(&gr.dSt, m * sizeof(int32_t)) == cudaSuccess &&
                    cudaMallocHost(&gr.hF, 9 * m * sizeof(double)) == cudaSuccess &&
                    cudaMallocHost(&gr.hS, 9 * m * sizeof(double)) == cudaSuccess &&
                    cudaMallocHost(&gr.hI, m * sizeof(int32_t)) == cudaSuccess &&
                    cudaMallocHost(&gr.hSt, m * sizeof(int32_t)) == cudaSuccess;
    if (!ok) {
      (void)cudaGetLastError();
      rve_server_destroy(s);
      return fail(RVE_ENOMEM, "server buffer allocation failed");
    }
    s->buffer_bytes += group_bytes(max_wave);
  }
  Segment g;
  g.b = b;
  g.owned = false;
  g.first = 0;
  g.n = b->n_rve;
  s->segs.push_back(g);
  if (b->opt.precision != RVE_PREC_PLAIN_F64) {
    const int rc = attach_segment(s, s->segs.back());
    if (rc != RVE_OK) {
      rve_server_destroy(s);
      return rc;
    }
  } else {
    for (Group& gr : s->groups) gr.work.emplace_back();
    s->segs.back().bytes = b->device_bytes;
  }
  s->pool_bytes = s->segs.back().bytes;
  if (hbm_cap_bytes > 0.0 && double(s->pool_bytes + s->buffer_bytes) > hbm_cap_bytes) {
    rve_server_destroy(s);
    return fail(RVE_EADMIT, "batch state and server buffers exceed the cap of " +
                                std::to_string(hbm_cap_bytes / 1e9) + " GB");
  }
  s->next_id = b->n_rve;
  s->on_gpu.assign(size_t(b->n_rve), 0);
  *out = s;
  return RVE_OK;
}

int rve_server_set_wave_iters(rve_server* s, int32_t wave_iters) {
  if (!s) return fail(RVE_EINVAL, "null server");
  if (wave_iters < 0) return fail(RVE_EINVAL, "wave_iters must be >= 0");
  if (wave_iters > 0 && s->precision == RVE_PREC_PLAIN_F64)
    return fail(RVE_EINVAL, "iteration-level waves need a batched precision");
  if (any_busy(s)) return fail(RVE_EINVAL, "change the wave length only while no request is on the GPU");
  s->wave_iters = wave_iters;
  return RVE_OK;
}

int rve_server_add_rves(rve_server* s, int64_t n_rve, const int64_t* node_off, const double* X,
                        const int64_t* fiber_off, const int32_t* conn, const double* L0, const double* EA,
                        const double* B, const uint8_t* is_boundary, const double* V0, int64_t* first_id) {
  if (!s || !first_id) return fail(RVE_EINVAL, "null argument");
  if (n_rve < 1) return fail(RVE_EINVAL, "n_rve must be >= 1");
  if (s->precision == RVE_PREC_PLAIN_F64) return fail(RVE_EINVAL, "the pool grows on the batched precisions");
  if (!node_off || !fiber_off) return fail(RVE_EINVAL, "node_off and fiber_off are required");
  // a lower bound of the footprint from the input sizes (fiber records and
  // per-node state) rejects an obviously oversized admission before any allocation
  const double free_room = s->cap_bytes > 0.0 ? s->cap_bytes - double(s->pool_bytes + s->buffer_bytes) : 1e300;
  const double lower = 56.0 * double(fiber_off[n_rve] - fiber_off[0]) + 32.0 * double(node_off[n_rve] - node_off[0]);
  if (lower > free_room)
    return fail(RVE_EADMIT, "admitting " + std::to_string(n_rve) + " RVEs needs more than " +
                                std::to_string(lower / 1e9) + " GB; " + std::to_string(free_room / 1e9) +
                                " GB left under the cap");
  rve_batch* nb = nullptr;
  int rc = rve_batch_create(&nb, s->device, n_rve, node_off, X, fiber_off, conn, L0, EA, B, is_boundary, V0, &s->opt);
  if (rc != RVE_OK) return rc;
  Segment g;
  g.b = nb;
  g.owned = true;
  g.first = s->next_id;
  g.n = n_rve;
  s->segs.push_back(g);
  rc = attach_segment(s, s->segs.back());
  const double after = double(s->pool_bytes + s->segs.back().bytes + s->buffer_bytes);
  if (rc != RVE_OK || (s->cap_bytes > 0.0 && after > s->cap_bytes)) {
    const size_t need = s->segs.back().bytes;
    release_segment(s, s->segs.size() - 1);
    for (Group& gr : s->groups) gr.work.pop_back();
    s->segs.pop_back();
    if (rc != RVE_OK) return rc;
    return fail(RVE_EADMIT, "admitting " + std::to_string(n_rve) + " RVEs needs " + std::to_string(need / 1e9) +
                                " GB; " + std::to_string(free_room / 1e9) + " GB left under the cap");
  }
  s->pool_bytes += s->segs.back().bytes;
  s->next_id += n_rve;
  s->on_gpu.resize(size_t(s->next_id), 0);
  *first_id = g.first;
  return RVE_OK;
}

int rve_server_remove_rves(rve_server* s, int64_t first_id) {
  if (!s) return fail(RVE_EINVAL, "null server");
  for (size_t k = 0; k < s->segs.size(); ++k) {
    Segment& g = s->segs[k];
    if (!g.live || g.first != first_id) continue;
    if (!g.owned) return fail(RVE_EINVAL, "the batch given at creation stays in the pool");
    if (g.busy > 0) return fail(RVE_EINVAL, "requests for these RVEs are queued or in flight");
    for (Group& gr : s->groups)
      if (gr.busy) RVE_CUDA_TRY(cudaStreamSynchronize(gr.stream));
    s->pool_bytes -= g.bytes;
    release_segment(s, k);
    return RVE_OK;
  }
  return fail(RVE_EINVAL, "no admitted RVE group starts at id " + std::to_string(first_id));
}

int rve_server_submit(rve_server* s, int64_t rve_id, const double* F, int64_t tag) {
  if (!s || !F) return fail(RVE_EINVAL, "null argument");
  Request r;
  const int rc = find_segment(s, rve_id, &r.seg, &r.local);
  if (rc != RVE_OK) return rc;
  r.id = rve_id;
  r.tag = tag;
  std::memcpy(r.F, F, sizeof(r.F));
  r.t0 = clk::now();
  s->queue.push_back(r);
  s->segs[r.seg].busy++;
  return RVE_OK;
}

int rve_server_step(rve_server* s) {
  if (!s) return fail(RVE_EINVAL, "null server");
  RVE_CUDA_TRY(cudaSetDevice(s->device));
  for (Group& gr : s->groups)
    if (gr.busy) {
      const int rc = retire(s, gr);
      if (rc != RVE_OK) return rc;
    }
  for (Group& gr : s->groups) {
    if (!gr.busy && (gr.n_used > 0 || !s->queue.empty())) {
      const int rc = launch(s, gr);
      if (rc != RVE_OK) return rc;
    }
  }
  return RVE_OK;
}

int rve_server_drain(rve_server* s) {
  if (!s) return fail(RVE_EINVAL, "null server");
  for (;;) {
    for (Group& gr : s->groups)
      if (gr.busy) RVE_CUDA_TRY(cudaEventSynchronize(gr.done));
    const int rc = rve_server_step(s);
    if (rc != RVE_OK) return rc;
    if (!any_busy(s) && s->queue.empty()) return RVE_OK;
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
  for (const Group& gr : s->groups) inflight += gr.n_used;
  st->in_flight = inflight;
  st->completed = s->completed;
  st->ready = int64_t(s->done.size());
  st->waves = s->waves;
  st->device_bytes = int64_t(s->buffer_bytes);
  int64_t rves = 0;
  for (const Segment& g : s->segs)
    if (g.live) rves += g.n;
  st->pool_rves = rves;
  st->pool_device_bytes = int64_t(s->pool_bytes);
  st->wave_iters = s->wave_iters;
  return RVE_OK;
}

}  // extern "C"
