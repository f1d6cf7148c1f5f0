// The library-owned batch object behind the opaque rve_batch handle.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "rve_internal.h"

namespace rvegpu {

#define RVE_CUDA_TRY(call)                                                              \
  do {                                                                                  \
    cudaError_t err__ = (call);                                                         \
    if (err__ != cudaSuccess)                                                           \
      return ::rvegpu::fail(RVE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(err__)); \
  } while (0)

// One launch configuration of the fused kernel and the work it runs.
struct Bin {
  int mode = 0;   // 0 resident, 1 streamed (SCR in shared), 2 streamed (SCR global)
  int nt = 256;   // threads per CTA
  int npt = 1;    // free nodes per thread
  int per_sm = 1; // CTAs per SM the footprint allows (bin key)
  int check_every = 0;  // 0: the batch option; > 0: set by the autotuner
  size_t smem = 0;
  size_t smem_node = 0;  // > 0: the node-centric kernel can run this bin with this much shared memory
  bool pdl = false;      // launched as a programmatic dependent of the launch before it on its stream
  int cl = 0;            // > 0: the cluster kernel runs this bin, cl CTAs per RVE ...
  int cl_npt = 1;        // ... with cl_npt free nodes per thread ...
  size_t smem_cluster = 0;  // ... and this much shared memory per CTA
  std::vector<Work> work;
  Work* d_work = nullptr;    // canonical order
  Work* d_sorted = nullptr;  // longest-first order written before each launch (bins up to LPT_MAX)
  int n = 0;
};
constexpr int LPT_MAX = 16384;  // bins up to this size are sorted on the device before launch

// Launch configuration chosen for one RVE.
struct BinKey {
  int mode, nt, npt, per_sm;
  size_t smem;
  int cl = 0, cl_npt = 1;  // cluster configuration (streamed RVEs, mixed precision): part of the key, so an
                           // RVE's cluster split does not depend on the other RVEs of its batch
  size_t smem_cl = 0;
  bool operator==(const BinKey& o) const {
    return mode == o.mode && nt == o.nt && npt == o.npt && per_sm == o.per_sm && cl == o.cl && cl_npt == o.cl_npt;
  }
};

// Batched-path state of one arithmetic type (float: mixed, double: FP64).
struct PathState {
  bool ready = false;
  std::vector<BinKey> key_of;   // per RVE
  std::vector<Bin> bins;        // all-RVE solve
  std::vector<Bin> tan_bins;    // tangent: 18 perturbed solves per RVE
  std::vector<Bin> man_bins;    // six-solve (Mandel) tangent: direction slots 0..5 of the above
  void* d_state = nullptr;      // 4 doubles per free node (fluctuation h, FP64 for both paths)
  uint8_t* d_valid = nullptr;   // per RVE: state holds a previous solve
  int32_t* d_last_iters = nullptr;  // per RVE: iterations of its last solve (scheduling cost)
  void* d_gP0 = nullptr;        // streamed-bin scratch (4 T per active fiber)
  void* d_gP1 = nullptr;
  void* d_gSCR = nullptr;
  double* d_energy = nullptr;   // energy_check: 6 doubles per RVE of the last all-RVE solve
  void* d_tan_state = nullptr;  // 18 x 4 doubles per free node
  void* d_tan_g[3] = {};        // streamed-bin scratch of the tangent directions
  std::vector<int> bin_of;      // per RVE: index into bins
  std::vector<Work> work_of;    // per RVE: its work item in the all-RVE solve
  Work* d_sub_work = nullptr;   // subset solves
  Work* d_sub_sorted = nullptr;
  size_t sub_cap = 0;
};

constexpr int N_SIDE_STREAMS = 6;

// Work-list buffers of one subset solve in flight.  Concurrent solves need
// their own (the server gives each slot one); the batch's own set is used
// by the public entry point, which orders itself after earlier GPU work.
struct SubsetBuffers {
  Work* d_work = nullptr;
  Work* d_sorted = nullptr;
  Work* h_stage = nullptr;  // pinned
  size_t cap = 0;
};

// Subset solve (rve_solve_subset); fork = false keeps every launch on `s`.
int solve_subset(rve_batch* b, const int64_t* ids, int64_t m, const double* F, double tol, int32_t max_iter,
                 double* sigma, int32_t* iters, int32_t* status, cudaStream_t s, bool fork,
                 const SubsetBuffers* ext);
// Iteration-level waves: solves stop after wave_iters iterations and park
// (resume: one record per RVE of the batch; vel: 4 T per free node).
struct WaveParams {
  int32_t wave_iters = 0;
  ResumeRec* resume = nullptr;
  void* vel = nullptr;
};
// Subset solve writing item k's outputs (and reading its F) at index outs[k]
// (k when outs is null), optionally as one wave.
int solve_items(rve_batch* b, const int64_t* ids, const int32_t* outs, int64_t m, const double* F, double tol,
                int32_t max_iter, double* sigma, int32_t* iters, int32_t* status, cudaStream_t s, bool fork,
                const SubsetBuffers* ext, const WaveParams* wave);
// Bring up the batched path of the batch's precision (bins, state buffers).
int ensure_batched_path(rve_batch* b);
constexpr int N_DIRS = 18;  // 9 directions x (+h, -h)

}  // namespace rvegpu

namespace rvegpu {
// A captured rve_solve, replayed while its arguments stay the same.
struct GraphEntry {
  const double* F;
  double* sigma;
  int32_t* iters;
  int32_t* status;
  cudaStream_t stream;
  double tol;
  int32_t max_iter;
  cudaGraphExec_t exec;
};
}  // namespace rvegpu

struct rve_batch {
  int device = 0;
  int64_t n_rve = 0;
  rve_options opt{};
  rvegpu::HostTopology topo;
  int64_t total_nf = 0, total_na = 0, total_nb = 0;
  // device topology
  rvegpu::RveMeta* d_meta = nullptr;
  rvegpu::FibD* d_fa = nullptr;
  uint32_t* d_fij = nullptr;
  rvegpu::FibD* d_fb = nullptr;
  uint16_t* d_csr = nullptr;
  uint16_t* d_nord = nullptr;
  uint32_t* d_ncsr = nullptr;
  float* d_ncap = nullptr;
  rvegpu::PathState pf, pd;
  // plain FP64 path scratch (sized for the largest RVE)
  double* d_pl = nullptr;
  size_t pl_bytes = 0;
  double* h_pl = nullptr;  // pinned, reduction read-back
  int32_t* d_pdl_done = nullptr;  // CTAs finished of the dependent part of a split launch
  // streams for concurrent bins
  cudaStream_t side[rvegpu::N_SIDE_STREAMS] = {};
  cudaStream_t hstream = nullptr;  // host-buffer solves
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[rvegpu::N_SIDE_STREAMS] = {};
  // tangent scratch
  double* d_tanF = nullptr;
  double* d_tanS = nullptr;
  int32_t* d_tanI = nullptr;
  int32_t* d_tanSt = nullptr;
  // host-API staging
  double* d_hF = nullptr;
  double* d_hS = nullptr;
  int32_t* d_hI = nullptr;
  int32_t* d_hSt = nullptr;
  double* h_pin = nullptr;
  size_t h_pin_bytes = 0;
  rvegpu::Work* h_work_pin = nullptr;  // staging for subset work lists
  size_t h_work_cap = 0;
  cudaEvent_t ev_work = nullptr;       // last upload from h_work_pin done
  cudaEvent_t ev_last = nullptr;       // end of the last public call's GPU work on this batch
  size_t device_bytes = 0;
  std::vector<void*> allocations;
  std::vector<rvegpu::GraphEntry> graphs;  // rve_solve captures (option graphs = 1)
  // optional per-launch timing of the fused solve kernel (rve_set_kernel_timing)
  bool timing = false;
  std::vector<cudaEvent_t> kev;  // start/end pairs, reused across calls
  size_t n_kev = 0;              // pairs recorded by the last public call
};
