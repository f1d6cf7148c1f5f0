// C ABI of the batched RVE solver (declared in include/rve.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batch.h"
#include "dr_fused.cuh"
#include "mandel.cuh"

namespace rvegpu {

namespace {
thread_local std::string g_error;
}

void set_error(const std::string& msg) { g_error = msg; }
int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

int launch_bin_viscous(const DrArgs<float>& a, const Bin& bin, cudaStream_t s);
int launch_bin_viscous(const DrArgs<double>& a, const Bin& bin, cudaStream_t s);
int launch_bin_kinetic(const DrArgs<float>& a, const Bin& bin, cudaStream_t s);
int launch_bin_kinetic(const DrArgs<double>& a, const Bin& bin, cudaStream_t s);
int launch_bin_energy(const DrArgs<float>& a, const Bin& bin, cudaStream_t s);
int launch_bin_energy(const DrArgs<double>& a, const Bin& bin, cudaStream_t s);
template <typename T>
int launch_bin(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  if (a.kinetic) return launch_bin_kinetic(a, bin, s);
  return a.energy ? launch_bin_energy(a, bin, s) : launch_bin_viscous(a, bin, s);
}
int cluster_capacity_f32(int npt, int cl, size_t smem, int* n_clusters);
int plain_scratch_bytes(int nf_max, int na_max);
int plain_solve_one(rve_batch* b, int r, int out, const double* F, double tol, int max_iter, double* sigma,
                    int32_t* iters, int32_t* status, cudaStream_t s);

namespace {

#define TRY(x)                  \
  do {                          \
    const int rc__ = (x);       \
    if (rc__ != RVE_OK) return rc__; \
  } while (0)

int dalloc(rve_batch* b, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return fail(RVE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  b->allocations.push_back(*p);
  b->device_bytes += bytes;
  return RVE_OK;
}

template <class T>
int upload(rve_batch* b, T** d, const std::vector<T>& h) {
  TRY(dalloc(b, reinterpret_cast<void**>(d), h.size() * sizeof(T)));
  if (!h.empty()) RVE_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return RVE_OK;
}

int valid_options(const rve_options& o) {
  if (!(o.tol > 0.0) || !std::isfinite(o.tol)) return fail(RVE_EINVAL, "tol must be > 0");
  if (o.max_iter < 0) return fail(RVE_EINVAL, "max_iter must be >= 0");
  if (o.check_every < 1) return fail(RVE_EINVAL, "check_every must be >= 1");
  if (o.precision < RVE_PREC_PLAIN_F64 || o.precision > RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "unknown precision");
  if (o.warm_start != 0 && o.warm_start != 1) return fail(RVE_EINVAL, "warm_start must be 0 or 1");
  if (!std::isfinite(o.damping)) return fail(RVE_EINVAL, "damping must be finite");
  if (!std::isfinite(o.sigma_tol)) return fail(RVE_EINVAL, "sigma_tol must be finite");
  if (o.graphs != 0 && o.graphs != 1) return fail(RVE_EINVAL, "graphs must be 0 or 1");
  if (!(o.damping_scale >= 0.0 && o.damping_scale <= 1.0))
    return fail(RVE_EINVAL, "damping_scale must be in (0, 1] (0 = default)");
  if (o.damping_mode != RVE_DAMP_VISCOUS && o.damping_mode != RVE_DAMP_KINETIC)
    return fail(RVE_EINVAL, "damping_mode must be RVE_DAMP_VISCOUS or RVE_DAMP_KINETIC");
  if (o.damping_mode == RVE_DAMP_KINETIC && o.precision == RVE_PREC_PLAIN_F64)
    return fail(RVE_EINVAL, "kinetic damping runs on the batched precisions");
  if (o.energy_check != 0 && o.energy_check != 1) return fail(RVE_EINVAL, "energy_check must be 0 or 1");
  if (o.energy_check && (o.precision == RVE_PREC_PLAIN_F64 || o.damping_mode == RVE_DAMP_KINETIC))
    return fail(RVE_EINVAL, "the energy balance runs on the batched precisions with viscous damping");
  if (o.reserved_ != 0) return fail(RVE_EINVAL, "reserved_ must be 0");
  if (o.kernel != RVE_KERNEL_AUTO && o.kernel != RVE_KERNEL_TWO_PHASE && o.kernel != RVE_KERNEL_NODE)
    return fail(RVE_EINVAL, "kernel must be RVE_KERNEL_AUTO, RVE_KERNEL_TWO_PHASE or RVE_KERNEL_NODE");
  if (o.threads != 0 && o.threads != 64 && o.threads != 128 && o.threads != 256 && o.threads != 512 &&
      o.threads != 1024)
    return fail(RVE_EINVAL, "threads must be 0, 64, 128, 256, 512 or 1024");
  return RVE_OK;
}

// Launch configuration of one RVE in the fused kernel.
template <typename T>
int choose_key(int nf, int na, int csr_len, int threads, BinKey& k) {
  if (nf > 4 * MAX_THREADS) return fail(RVE_EINVAL, "the batched path holds at most 4096 free nodes per RVE");
  int nt;
  if (threads > 0) {
    nt = threads;
  } else {
    const int target = std::max(na / 5, (nf + 3) / 4);
    nt = 64;
    while (nt < target && nt < 1024) nt *= 2;
  }
  while (nf > 4 * nt && nt < 1024) nt *= 2;
  auto npt_of = [](int nf_, int nt_) {
    const int q = (nf_ + nt_ - 1) / nt_;
    return q <= 1 ? 1 : (q <= 2 ? 2 : 4);
  };
  int npt = npt_of(nf, nt);
  const size_t budget = SMEM_LIMIT - 1024;
  size_t sm = smem_resident<T>(nf, na, csr_len, nt);
  int mode = 0;
  if (sm > budget) {
    nt = 1024;
    npt = std::max(2, npt_of(nf, nt));
    const size_t s1 = smem_streamed<T>(nf, na, nt, true);
    if (s1 <= budget) {
      mode = 1;
      sm = s1;
    } else {
      mode = 2;
      sm = smem_streamed<T>(nf, na, nt, false);
      if (sm > budget) return fail(RVE_EINVAL, "RVE too large for the batched path");
    }
  }
  const int by_smem = int((228 * 1024) / (sm + 1024 + 512));
  const int by_thr = 2048 / nt;
  k = BinKey{mode, nt, npt, std::max(1, std::min(by_smem, by_thr)), sm};
  return RVE_OK;
}

// Incidence slots of the busiest thread of RVE r in the node-centric layout
// (nt threads, npt free nodes each, dealt by node_rank over the
// decreasing-degree order).
int node_slots(const rve_batch* b, int64_t r, int nt, int npt) {
  const RveMeta& M = b->topo.meta[size_t(r)];
  const uint16_t* csr = b->topo.csr.data() + M.csr_off;
  auto deg = [&](int a) {
    const uint32_t w = b->topo.ncsr[size_t(M.node_off + a)];
    int d = 0;
    for (uint32_t k = 0; k < (w & 0xffu); ++k) d += (uint32_t(csr[(w >> 8) + k]) >> 1) < uint32_t(M.na) ? 1 : 0;
    return d;
  };
  int best = 0;
  for (int t = 0; t < nt; ++t) {
    int sl = 0;
    for (int q = 0; q < npt; ++q) {
      const int k = node_rank(q, t, nt);
      if (k < M.nf) sl += deg(int(b->topo.nord[size_t(M.node_off + k)]));
    }
    best = std::max(best, sl);
  }
  return best;
}

// Shared memory the node-centric kernel needs for every RVE of a work list
// at (nt, npt); 0 when one of them does not fit or holds more free nodes
// than the threads own.
template <typename T>
size_t node_smem(const rve_batch* b, const std::vector<Work>& work, int nt, int npt) {
  size_t need = 0;
  for (const Work& w : work) {
    const RveMeta& M = b->topo.meta[size_t(w.rve)];
    if (M.nf > nt * npt) return 0;
    need = std::max(need, smem_node<T>(M.nf, node_slots(b, w.rve, nt, npt), nt));
  }
  return need <= SMEM_LIMIT - 1024 ? need : 0;
}

// Free nodes per thread preferred by the cluster kernel when both fit: 2
// (half the SMs per RVE of 1; each thread walks twice the slots).
#ifndef RVE_CLUSTER_NPT_PREF
#define RVE_CLUSTER_NPT_PREF 2
#endif

// Cluster configuration of a streamed RVE (mixed precision), from the RVE
// alone: the fewest CTAs of CLUSTER_NT threads that own every free node,
// with RVE_CLUSTER_NPT_PREF nodes per thread if that fits one CTA's shared
// memory, else the other choice; cl = 0 when neither fits.
void cluster_key(const rve_batch* b, int64_t r, BinKey& k) {
  k.cl = 0;
  k.cl_npt = 1;
  k.smem_cl = 0;
  const int nf = b->topo.meta[size_t(r)].nf;
  const int order[2] = {RVE_CLUSTER_NPT_PREF, 3 - RVE_CLUSTER_NPT_PREF};
  for (int npt : order) {
    const int cl = std::max(2, (nf + npt * CLUSTER_NT - 1) / (npt * CLUSTER_NT));
    if (cl > CLUSTER_MAX) continue;
    const size_t need = smem_cluster<float>(nf, node_slots(b, r, cl * CLUSTER_NT, npt), CLUSTER_NT);
    if (need > SMEM_LIMIT - 1024) continue;
    k.cl = cl;
    k.cl_npt = npt;
    k.smem_cl = need;
    return;
  }
}

// The device must hold at least one cluster of a bin's configuration;
// otherwise the bin runs the streamed two-phase kernel.
int check_cluster(Bin& bin) {
  if (bin.cl == 0) return RVE_OK;
  int n_clusters = 0;
  TRY(cluster_capacity_f32(bin.cl_npt, bin.cl, bin.smem_cluster, &n_clusters));
  if (n_clusters <= 0) bin.cl = 0;
  return RVE_OK;
}

template <typename T>
PathState& path(rve_batch* b);
template <>
PathState& path<float>(rve_batch* b) {
  return b->pf;
}
template <>
PathState& path<double>(rve_batch* b) {
  return b->pd;
}

int upload_bins(rve_batch* b, std::vector<Bin>& bins) {
  for (Bin& bin : bins) {
    bin.n = int(bin.work.size());
    TRY(upload(b, &bin.d_work, bin.work));
    if (bin.n > 0 && bin.n <= LPT_MAX) TRY(upload(b, &bin.d_sorted, bin.work));
  }
  return RVE_OK;
}

// Longest-first order of a bin's work items by learned cost: active fibers x
// (iterations of the RVE's last solve + 1); ties keep the canonical order.
// One CTA, bitonic sort of 64-bit keys (cost << 17 | reversed position).
__global__ void lpt_sort(const Work* __restrict__ in, Work* __restrict__ out, int n, const RveMeta* __restrict__ meta,
                         const int32_t* __restrict__ last_iters) {
  extern __shared__ unsigned long long key[];
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    unsigned long long k = 0ull;
    if (i < n) {
      const int r = in[i].rve;
      const unsigned long long cost =
          static_cast<unsigned long long>(meta[r].na) * static_cast<unsigned long long>(max(last_iters[r], 0) + 1);
      k = (cost << 17) | static_cast<unsigned long long>((1 << 17) - 1 - i);
    }
    key[i] = k;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], c = key[ixj];
          const bool desc = (i & k) == 0;
          if (desc ? (a < c) : (a > c)) {
            key[i] = c;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    out[i] = in[(1 << 17) - 1 - static_cast<int>(key[i] & 0x1ffffull)];
}

int launch_sorted(rve_batch* b, const Bin& bin, cudaStream_t s, const int32_t* last_iters, Bin& use) {
  use = bin;
  if (!bin.d_sorted || bin.n <= 1 || bin.n > LPT_MAX) return RVE_OK;
  int n2 = 1;
  while (n2 < bin.n) n2 <<= 1;
  static bool attr_set[64] = {};
  static std::mutex attr_mu;
  int dev = 0;
  RVE_CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(attr_mu);
    if (dev >= 64 || !attr_set[dev]) {
      RVE_CUDA_TRY(cudaFuncSetAttribute(lpt_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(LPT_MAX * sizeof(unsigned long long))));
      if (dev < 64) attr_set[dev] = true;
    }
  }
  lpt_sort<<<1, 1024, size_t(n2) * sizeof(unsigned long long), s>>>(bin.d_work, bin.d_sorted, bin.n, b->d_meta,
                                                                     last_iters);
  RVE_CUDA_TRY(cudaGetLastError());
  use.d_work = bin.d_sorted;
  return RVE_OK;
}

template <typename T>
int ensure_path(rve_batch* b) {
  PathState& P = path<T>(b);
  if (P.ready) return RVE_OK;
  const int64_t n = b->n_rve;
  P.key_of.resize(n);
  std::vector<BinKey> keys;
  std::vector<std::vector<int>> members;
  for (int64_t r = 0; r < n; ++r) {
    const RveMeta& M = b->topo.meta[r];
    BinKey k;
    TRY(choose_key<T>(M.nf, M.na, M.csr_len, b->opt.threads, k));
    if (k.mode != 0 && std::is_same<T, float>::value) cluster_key(b, r, k);
    P.key_of[r] = k;
    size_t j = 0;
    while (j < keys.size() && !(keys[j] == k)) ++j;
    if (j == keys.size()) {
      keys.push_back(k);
      members.emplace_back();
    }
    keys[j].smem = std::max(keys[j].smem, k.smem);
    keys[j].smem_cl = std::max(keys[j].smem_cl, k.smem_cl);
    members[j].push_back(int(r));
  }
  // streamed-bin scratch offsets (main solves and tangent directions)
  int64_t scr_main = 0, scr_tan = 0;
  std::vector<int32_t> scr_of(n, 0), scr_tan_of(n, 0);
  for (int64_t r = 0; r < n; ++r) {
    if (P.key_of[r].mode == 0) continue;
    scr_of[r] = int32_t(scr_main);
    scr_main += b->topo.meta[r].na + 1;  // + the zero slot
    scr_tan_of[r] = int32_t(scr_tan);
    scr_tan += int64_t(N_DIRS) * (b->topo.meta[r].na + 1);
  }
  if (scr_tan > INT32_MAX) return fail(RVE_EINVAL, "streamed scratch exceeds 32-bit offsets");
  P.bins.clear();
  P.tan_bins.clear();
  P.man_bins.clear();
  for (size_t j = 0; j < keys.size(); ++j) {
    std::vector<int>& mem = members[j];
    std::stable_sort(mem.begin(), mem.end(),
                     [&](int x, int y) { return b->topo.meta[x].na > b->topo.meta[y].na; });
    Bin bin;
    bin.mode = keys[j].mode;
    bin.nt = keys[j].nt;
    bin.npt = keys[j].npt;
    bin.per_sm = keys[j].per_sm;
    bin.smem = keys[j].smem;
    Bin tb = bin;
    Bin mb = bin;
    for (int r : mem) bin.work.push_back(Work{r, r, b->topo.meta[r].node_off, 0, scr_of[r], 0});
    if (bin.mode == 0) {
      bin.smem_node = node_smem<T>(b, bin.work, bin.nt, bin.npt);
    } else {
      bin.cl = keys[j].cl;
      bin.cl_npt = keys[j].cl_npt;
      bin.smem_cluster = keys[j].smem_cl;
      TRY(check_cluster(bin));
    }
    tb.smem_node = mb.smem_node = bin.smem_node;
    tb.cl = mb.cl = bin.cl;
    tb.cl_npt = mb.cl_npt = bin.cl_npt;
    tb.smem_cluster = mb.smem_cluster = bin.smem_cluster;
    for (int r : mem)
      for (int d = 0; d < N_DIRS; ++d) {
        const Work w{r, int32_t(d * n + r), int32_t(d * b->total_nf + b->topo.meta[r].node_off), 1,
                     int32_t(scr_tan_of[r] + d * (b->topo.meta[r].na + 1)), 0};
        tb.work.push_back(w);
        if (d < N_MANDEL) mb.work.push_back(w);
      }
    P.bins.push_back(std::move(bin));
    P.tan_bins.push_back(std::move(tb));
    P.man_bins.push_back(std::move(mb));
  }
  // largest total work first so the long bins start early
  auto work_of = [&](const Bin& x) {
    int64_t w = 0;
    for (const Work& wk : x.work) w += b->topo.meta[wk.rve].na;
    return w;
  };
  std::stable_sort(P.bins.begin(), P.bins.end(), [&](const Bin& x, const Bin& y) { return work_of(x) > work_of(y); });
  std::stable_sort(P.tan_bins.begin(), P.tan_bins.end(),
                   [&](const Bin& x, const Bin& y) { return work_of(x) > work_of(y); });
  std::stable_sort(P.man_bins.begin(), P.man_bins.end(),
                   [&](const Bin& x, const Bin& y) { return work_of(x) > work_of(y); });
  P.bin_of.assign(size_t(n), -1);
  P.work_of.assign(size_t(n), Work{});
  for (size_t j = 0; j < P.bins.size(); ++j)
    for (const Work& w : P.bins[j].work) {
      P.bin_of[w.rve] = int(j);
      P.work_of[w.rve] = w;
    }
  TRY(upload_bins(b, P.bins));
  TRY(upload_bins(b, P.tan_bins));
  TRY(upload_bins(b, P.man_bins));
  TRY(dalloc(b, &P.d_state, sizeof(double) * 4 * size_t(std::max<int64_t>(b->total_nf, 1))));
  RVE_CUDA_TRY(cudaMemset(P.d_state, 0, sizeof(double) * 4 * size_t(std::max<int64_t>(b->total_nf, 1))));
  TRY(dalloc(b, reinterpret_cast<void**>(&P.d_valid), size_t(std::max<int64_t>(n, 1))));
  RVE_CUDA_TRY(cudaMemset(P.d_valid, 0, size_t(std::max<int64_t>(n, 1))));
  TRY(dalloc(b, reinterpret_cast<void**>(&P.d_last_iters), sizeof(int32_t) * size_t(std::max<int64_t>(n, 1))));
  RVE_CUDA_TRY(cudaMemset(P.d_last_iters, 0, sizeof(int32_t) * size_t(std::max<int64_t>(n, 1))));
  if (scr_main > 0) {
    TRY(dalloc(b, &P.d_gP0, sizeof(T) * 4 * size_t(scr_main)));
    TRY(dalloc(b, &P.d_gP1, sizeof(T) * 4 * size_t(scr_main)));
    TRY(dalloc(b, &P.d_gSCR, sizeof(T) * 4 * size_t(scr_main)));
  }
  P.ready = true;
  return RVE_OK;
}

// Run a list of bins on `s`, concurrently on side streams when there are several.
constexpr size_t KERNEL_TIMING_MAX = 65536;  // launches recorded per rve_set_kernel_timing

// The costliest RVEs of a large resident bin (the head of the longest-first
// list) run in a launch of their own whose shared-memory request leaves no
// room for another CTA on their SM: an RVE alone on an SM takes ~25 % less
// time per DR iteration than two sharing one, and these RVEs set the end of
// the solve.  The rest of the bin follows on the same stream as a
// programmatic dependent launch, which starts as soon as every CTA of the
// first has begun (so those are resident first) and runs beside it on the
// other SMs.  Same kernel and arithmetic, so the results do not change.
#ifndef RVE_EXCL_MAX
#define RVE_EXCL_MAX 8
#endif
constexpr int EXCL_MAX = RVE_EXCL_MAX;     // RVEs given SMs of their own, per bin
constexpr size_t EXCL_SMEM = 224 * 1024;   // dynamic shared memory of their CTAs
int excl_count(const Bin& use) {
  if (use.mode != 0 || use.per_sm < 2 || use.n < 64) return 0;
  return std::min(EXCL_MAX, use.n / 64);
}

template <typename T>
int launch_split(rve_batch* b, const Bin& use, const DrArgs<T>& a, cudaStream_t s) {
  const int k = excl_count(use);
  if (k == 0) return launch_bin(a, use, s);
  Bin heavy = use, light = use;
  heavy.n = k;
  heavy.smem = std::max(use.smem, EXCL_SMEM);
  if (use.smem_node > 0) heavy.smem_node = std::max(use.smem_node, EXCL_SMEM);
  light.d_work = use.d_work + k;
  light.n = use.n - k;
  light.pdl = true;
  DrArgs<T> al = a;
  al.pdl_done = b->d_pdl_done;
  TRY(launch_bin(a, heavy, s));
  return launch_bin(al, light, s);
}

template <typename T>
int run_one(rve_batch* b, const Bin& bin, const DrArgs<T>& a, cudaStream_t s, bool split = false) {
  Bin use;
  TRY(launch_sorted(b, bin, s, a.last_iters, use));
  auto launch = [&]() { return split ? launch_split(b, use, a, s) : launch_bin(a, use, s); };
  if (!b->timing || b->n_kev >= KERNEL_TIMING_MAX) return launch();
  // events on the launching stream bracket the fused kernel alone
  if (2 * b->n_kev + 2 > b->kev.size()) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RVE_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return fail(RVE_ECUDA, "cudaEventCreate failed");
    }
    b->kev.push_back(e0);
    b->kev.push_back(e1);
  }
  const size_t k = 2 * b->n_kev++;
  RVE_CUDA_TRY(cudaEventRecord(b->kev[k], s));
  TRY(launch());
  RVE_CUDA_TRY(cudaEventRecord(b->kev[k + 1], s));
  return RVE_OK;
}

template <typename T>
// split: a lone bin may give its costliest RVEs SMs of their own (whole-
// batch solves; subset solves, whose concurrent calls would queue on the
// one high-priority stream, keep one launch per bin)
int run_bins(rve_batch* b, const std::vector<Bin>& bins, const DrArgs<T>& a, cudaStream_t s, bool fork = true,
             bool split = false) {
  std::vector<const Bin*> live;
  for (const Bin& x : bins)
    if (x.n > 0) live.push_back(&x);
  if (live.empty()) return RVE_OK;
  if (live.size() == 1 || !fork) {
    // one bin (or one stream): its costliest RVEs may take SMs of their own
    for (const Bin* x : live) TRY(run_one(b, *x, a, s, split && live.size() == 1));
    return RVE_OK;
  }
  RVE_CUDA_TRY(cudaEventRecord(b->ev_fork, s));
  const int ns = std::min<int>(N_SIDE_STREAMS, int(live.size()));
  for (int k = 0; k < ns; ++k) RVE_CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->ev_fork, 0));
  for (size_t i = 0; i < live.size(); ++i) TRY(run_one(b, *live[i], a, b->side[i % ns]));
  for (int k = 0; k < ns; ++k) {
    RVE_CUDA_TRY(cudaEventRecord(b->ev_join[k], b->side[k]));
    RVE_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_join[k], 0));
  }
  return RVE_OK;
}

template <typename T>
DrArgs<T> make_args(rve_batch* b, const double* F, double tol, int max_iter, double* sigma, int32_t* iters,
                    int32_t* status, void* state, int warm_start) {
  PathState& P = path<T>(b);
  DrArgs<T> a;
  a.meta = b->d_meta;
  a.fa = b->d_fa;
  a.fij = b->d_fij;
  a.fb = b->d_fb;
  a.csr = b->d_csr;
  a.ncsr = b->d_ncsr;
  a.nord = b->d_nord;
  a.node_kernel = b->opt.kernel == RVE_KERNEL_NODE ? 1 : 0;
  a.ncap = b->d_ncap;
  a.work = nullptr;
  a.n_work = 0;
  a.F = F;
  a.sigma = sigma;
  a.iters = iters;
  a.status = status;
  a.state = static_cast<double*>(state);
  a.valid = P.d_valid;
  a.last_iters = P.d_last_iters;
  a.warm_start = warm_start;
  a.gP0 = static_cast<T*>(P.d_gP0);
  a.gP1 = static_cast<T*>(P.d_gP1);
  a.gSCR = static_cast<T*>(P.d_gSCR);
  a.tol = tol;
  a.max_iter = max_iter;
  a.check_every = b->opt.check_every;
  a.damping = b->opt.damping;
  a.kinetic = b->opt.damping_mode == RVE_DAMP_KINETIC ? 1 : 0;
  a.damping_scale = b->opt.damping_scale > 0.0 ? b->opt.damping_scale : DAMP_SCALE;
  a.sigma_tol = b->opt.sigma_tol;
  a.wave_iters = 0;
  a.resume = nullptr;
  a.vel = nullptr;
  a.energy = nullptr;
  a.pdl_done = nullptr;
  return a;
}

int set_device(rve_batch* b) {
  RVE_CUDA_TRY(cudaSetDevice(b->device));
  return RVE_OK;
}

// Public calls share the batch's state and scratch: each one's GPU work
// starts after the previous call's, whatever streams they use.
void clear_graphs(rve_batch* b) {
  for (GraphEntry& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

int order_after_last(rve_batch* b, cudaStream_t s) {
  RVE_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_last, 0));
  return RVE_OK;
}

// Per-RVE energy records of the all-RVE solve (option energy_check).
int energy_buffer(rve_batch* b, PathState& P, double** out) {
  if (!P.d_energy) {
    TRY(dalloc(b, reinterpret_cast<void**>(&P.d_energy), sizeof(double) * 6 * size_t(std::max<int64_t>(b->n_rve, 1))));
    RVE_CUDA_TRY(cudaMemset(P.d_energy, 0, sizeof(double) * 6 * size_t(std::max<int64_t>(b->n_rve, 1))));
  }
  *out = P.d_energy;
  return RVE_OK;
}

int solve_all(rve_batch* b, const double* F, double tol, int max_iter, double* sigma, int32_t* iters,
              int32_t* status, cudaStream_t s) {
  const int prec = b->opt.precision;
  if (prec == RVE_PREC_MIXED) {
    TRY(ensure_path<float>(b));
    DrArgs<float> a = make_args<float>(b, F, tol, max_iter, sigma, iters, status, b->pf.d_state, b->opt.warm_start);
    if (b->opt.energy_check) TRY(energy_buffer(b, b->pf, &a.energy));
    return run_bins(b, b->pf.bins, a, s, true, true);
  }
  if (prec == RVE_PREC_BATCHED_F64) {
    TRY(ensure_path<double>(b));
    DrArgs<double> a = make_args<double>(b, F, tol, max_iter, sigma, iters, status, b->pd.d_state, b->opt.warm_start);
    if (b->opt.energy_check) TRY(energy_buffer(b, b->pd, &a.energy));
    return run_bins(b, b->pd.bins, a, s, true, true);
  }
  TRY(ensure_path<double>(b));  // state buffer shared with the FP64 batched path
  for (int64_t r = 0; r < b->n_rve; ++r)
    TRY(plain_solve_one(b, int(r), int(r), F, tol, max_iter, sigma, iters, status, s));
  return RVE_OK;
}

__global__ void tan_copy_state(const double* __restrict__ st, double* __restrict__ tan, int64_t total_nf,
                               int n_dirs) {
  const int64_t n4 = 4 * total_nf;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(n_dirs) * n4;
       i += int64_t(gridDim.x) * blockDim.x)
    tan[i] = st[i % n4];
}

__global__ void tan_make_F(const double* __restrict__ F, double* __restrict__ Fp, int64_t n, double h) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(N_DIRS) * n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = i / n, r = i % n;
    const int dir = int(d / 2);
    const double sgn = (d % 2 == 0) ? 1.0 : -1.0;
    for (int k = 0; k < 9; ++k) Fp[9 * i + k] = F[9 * r + k] + (k == dir ? sgn * h : 0.0);
  }
}

__global__ void tan_finish(const double* __restrict__ S, const int32_t* __restrict__ St, int64_t n, double h,
                           double* __restrict__ D, int32_t* __restrict__ status) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < 81 * n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / 81;
    const int ij = int(i % 81) / 9, kl = int(i % 81) % 9;
    const double sp = S[9 * ((2 * kl) * n + r) + ij];
    const double sm = S[9 * ((2 * kl + 1) * n + r) + ij];
    D[i] = (sp - sm) / (2.0 * h);
    if (status && i % 81 == 0) {
      int w = status[r];
      for (int d = 0; d < N_DIRS; ++d) w = max(w, St[d * n + r] == RVE_STATUS_EMPTY ? 0 : St[d * n + r]);
      status[r] = w;
    }
  }
}

// Orientation tensor Omega = <n (x) n> of every RVE at the state of its last
// solve (x = F X + h; h = 0 for an RVE not yet solved in that precision),
// over the active and the boundary-to-boundary fibers (the fibers kept after
// pruning); Sec. 4 sends it to the macroscale, Sec. 5's alignment measure is
// P2(a) = (3 a.Omega.a - 1)/2.  One CTA per RVE; per-thread sums in FP32 of
// unit dyads, per-warp partials summed in FP64.
constexpr int ORIENT_THREADS = 128;

__global__ void __launch_bounds__(ORIENT_THREADS) orient_kernel(const RveMeta* __restrict__ meta,
                                                               const FibD* __restrict__ fa,
                                                               const uint32_t* __restrict__ fij,
                                                               const FibD* __restrict__ fb,
                                                               const double* __restrict__ state,
                                                               const uint8_t* __restrict__ valid,
                                                               const double* __restrict__ F, double* __restrict__ omega,
                                                               int64_t r0) {
  __shared__ double part[ORIENT_THREADS / 32][6];
  const int64_t r = r0 + blockIdx.x;
  const RveMeta M = meta[r];
  const int tid = threadIdx.x;
  float f[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) f[k] = float(F[9 * r + k]);
  const bool warm = state && valid && valid[r];
  const double* st = warm ? state + 4 * size_t(M.node_off) : nullptr;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto add = [&](float dx, float dy, float dz) {
    const float inv = 1.0f / (dx * dx + dy * dy + dz * dz);
    acc[0] += dx * dx * inv;
    acc[1] += dy * dy * inv;
    acc[2] += dz * dz * inv;
    acc[3] += dy * dz * inv;
    acc[4] += dx * dz * inv;
    acc[5] += dx * dy * inv;
  };
  for (int e = tid; e < M.na; e += ORIENT_THREADS) {
    const FibD& q = fa[M.fa_off + e];
    const float X0 = float(q.dx), X1 = float(q.dy), X2 = float(q.dz);
    float dx = f[0] * X0 + f[1] * X1 + f[2] * X2;
    float dy = f[3] * X0 + f[4] * X1 + f[5] * X2;
    float dz = f[6] * X0 + f[7] * X1 + f[8] * X2;
    if (st) {
      const uint32_t ij = fij[M.fa_off + e];
      const uint32_t i = ij & 0xffffu, j = ij >> 16;
      double hx = 0.0, hy = 0.0, hz = 0.0;
      if (j < uint32_t(M.nf)) {
        hx += st[4 * j];
        hy += st[4 * j + 1];
        hz += st[4 * j + 2];
      }
      if (i < uint32_t(M.nf)) {
        hx -= st[4 * i];
        hy -= st[4 * i + 1];
        hz -= st[4 * i + 2];
      }
      dx += float(hx);
      dy += float(hy);
      dz += float(hz);
    }
    add(dx, dy, dz);
  }
  for (int e = tid; e < M.nb; e += ORIENT_THREADS) {
    const FibD& q = fb[M.fb_off + e];
    const float X0 = float(q.dx), X1 = float(q.dy), X2 = float(q.dz);
    add(f[0] * X0 + f[1] * X1 + f[2] * X2, f[3] * X0 + f[4] * X1 + f[5] * X2, f[6] * X0 + f[7] * X1 + f[8] * X2);
  }
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[warp][k] = double(v);
  }
  __syncthreads();
  if (tid < 9) {
    const int i = tid / 3, j = tid % 3;
    const int k = (i == j) ? i : 6 - i - j;  // xx yy zz yz xz xy
    double t = 0.0;
    for (int w = 0; w < ORIENT_THREADS / 32; ++w) t += part[w][k];
    const int cnt = M.na + M.nb;
    omega[9 * r + tid] = cnt > 0 ? t / double(cnt) : 0.0;
  }
}

// Buffers of the perturbed solves (both tangents): F, sigma, iterations and
// status per direction slot, the slots' warm-start states, and the streamed
// bins' scratch (laid out for all 18 slots; the six-solve tangent uses 0..5).
template <typename T>
int tangent_buffers(rve_batch* b, PathState& P, DrArgs<T>& a1) {
  const int64_t n = b->n_rve;
  if (!b->d_tanF) {
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_tanF), sizeof(double) * 9 * N_DIRS * size_t(n)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_tanS), sizeof(double) * 9 * N_DIRS * size_t(n)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_tanI), sizeof(int32_t) * (N_DIRS + 1) * size_t(n)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_tanSt), sizeof(int32_t) * (N_DIRS + 1) * size_t(n)));
  }
  if (!P.d_tan_state)
    TRY(dalloc(b, &P.d_tan_state, sizeof(double) * 4 * N_DIRS * size_t(std::max<int64_t>(b->total_nf, 1))));
  int64_t scr = 0;
  for (const Bin& bin : P.tan_bins)
    if (bin.mode != 0)
      for (const Work& w : bin.work) scr += b->topo.meta[w.rve].na + 1;
  if (scr > 0) {
    if (!P.d_tan_g[0])
      for (int k = 0; k < 3; ++k) TRY(dalloc(b, &P.d_tan_g[k], sizeof(T) * 4 * size_t(scr)));
    a1.gP0 = static_cast<T*>(P.d_tan_g[0]);
    a1.gP1 = static_cast<T*>(P.d_tan_g[1]);
    a1.gSCR = static_cast<T*>(P.d_tan_g[2]);
  }
  return RVE_OK;
}

// The paper's six-solve tangent (Sec. 3.2): base solve at F, six probing
// solves at R (U + h T_p) warm-started from it, then the FP64 algebra of
// mandel_finish.  C: 36 doubles per RVE (Mandel [I][J]).
template <typename T>
int mandel_batched(rve_batch* b, const double* F, double h, double tol, int max_iter, double* sigma, double* C,
                   int32_t* status, cudaStream_t s) {
  TRY(ensure_path<T>(b));
  PathState& P = path<T>(b);
  const int64_t n = b->n_rve;
  DrArgs<T> a1 = make_args<T>(b, nullptr, tol, max_iter, nullptr, nullptr, nullptr, nullptr, 1);
  TRY(tangent_buffers<T>(b, P, a1));
  int32_t* st_base = status ? status : b->d_tanSt + N_DIRS * n;
  int32_t* it_base = b->d_tanI + N_DIRS * n;
  const DrArgs<T> a0 = make_args<T>(b, F, tol, max_iter, sigma, it_base, st_base, P.d_state, b->opt.warm_start);
  TRY(run_bins(b, P.bins, a0, s));
  if (b->total_nf > 0) {
    tan_copy_state<<<1024, 256, 0, s>>>(static_cast<const double*>(P.d_state), static_cast<double*>(P.d_tan_state),
                                        b->total_nf, N_MANDEL);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  if (n > 0) {
    mandel_make_F<<<int((n + 127) / 128 < 4096 ? (n + 127) / 128 : 4096), 128, 0, s>>>(F, b->d_tanF, n, h);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  a1.F = b->d_tanF;
  a1.sigma = b->d_tanS;
  a1.iters = b->d_tanI;
  a1.status = b->d_tanSt;
  a1.state = static_cast<double*>(P.d_tan_state);
  TRY(run_bins(b, P.man_bins, a1, s, true, true));
  if (n > 0) {
    mandel_finish<<<int((n + 127) / 128 < 4096 ? (n + 127) / 128 : 4096), 128, 0, s>>>(
        F, sigma, b->d_tanS, b->d_tanSt, n, h, C, status);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  return RVE_OK;
}

template <typename T>
int tangent_batched(rve_batch* b, const double* F, double h, double tol, int max_iter, double* sigma,
                    double* dsdF, int32_t* status, cudaStream_t s) {
  TRY(ensure_path<T>(b));
  PathState& P = path<T>(b);
  const int64_t n = b->n_rve;
  DrArgs<T> a1 = make_args<T>(b, nullptr, tol, max_iter, nullptr, nullptr, nullptr, nullptr, 1);
  TRY(tangent_buffers<T>(b, P, a1));
  int32_t* st_base = status ? status : b->d_tanSt + N_DIRS * n;
  int32_t* it_base = b->d_tanI + N_DIRS * n;
  // base solve
  const DrArgs<T> a0 = make_args<T>(b, F, tol, max_iter, sigma, it_base, st_base, P.d_state, b->opt.warm_start);
  TRY(run_bins(b, P.bins, a0, s));
  // perturbed solves, warm-started from the base fluctuation
  if (b->total_nf > 0) {
    tan_copy_state<<<1024, 256, 0, s>>>(static_cast<const double*>(P.d_state), static_cast<double*>(P.d_tan_state),
                                        b->total_nf, N_DIRS);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  if (n > 0) {
    tan_make_F<<<256, 256, 0, s>>>(F, b->d_tanF, n, h);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  a1.F = b->d_tanF;
  a1.sigma = b->d_tanS;
  a1.iters = b->d_tanI;
  a1.status = b->d_tanSt;
  a1.state = static_cast<double*>(P.d_tan_state);
  TRY(run_bins(b, P.tan_bins, a1, s, true, true));
  if (n > 0) {
    tan_finish<<<512, 256, 0, s>>>(b->d_tanS, b->d_tanSt, n, h, dsdF, status);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  return RVE_OK;
}

// Autotuner: per bin, time the bin's RVEs under each launch configuration
// their sizes allow and keep the fastest.
template <typename T>
int autotune_path(rve_batch* b, const double* F, int reps, cudaStream_t s, double* ms_before, double* ms_after) {
  TRY(ensure_path<T>(b));
  PathState& P = path<T>(b);
  double* d_sig = nullptr;
  int32_t *d_it = nullptr, *d_st = nullptr;
  RVE_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_sig), sizeof(double) * 9 * size_t(b->n_rve), s));
  RVE_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_it), sizeof(int32_t) * size_t(b->n_rve), s));
  RVE_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_st), sizeof(int32_t) * size_t(b->n_rve), s));
  cudaEvent_t e0, e1;
  RVE_CUDA_TRY(cudaEventCreate(&e0));
  RVE_CUDA_TRY(cudaEventCreate(&e1));
  DrArgs<T> a = make_args<T>(b, F, b->opt.tol, b->opt.max_iter, d_sig, d_it, d_st, P.d_state, 0);
  auto time_bin = [&](const Bin& bin, float& ms) -> int {
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
      RVE_CUDA_TRY(cudaEventRecord(e0, s));
      TRY(run_one(b, bin, a, s));
      RVE_CUDA_TRY(cudaEventRecord(e1, s));
      RVE_CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.f;
      RVE_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    ms = best;
    return RVE_OK;
  };
  double before = 0.0, after = 0.0;
  for (Bin& bin : P.bins) {
    if (bin.n == 0) continue;
    int nf_max = 0, na_max = 0, csr_max = 0;
    for (const Work& w : bin.work) {
      nf_max = std::max(nf_max, b->topo.meta[w.rve].nf);
      na_max = std::max(na_max, b->topo.meta[w.rve].na);
      csr_max = std::max(csr_max, b->topo.meta[w.rve].csr_len);
    }
    float t_cur = 0.f;
    TRY(run_one(b, bin, a, s));  // warm-up (attributes, caches)
    TRY(time_bin(bin, t_cur));
    before += t_cur;
    Bin best = bin;
    float t_best = t_cur;
    for (int nt : {64, 128, 256, 512, 1024}) {
      BinKey k;
      if (choose_key<T>(nf_max, na_max, csr_max, nt, k) != RVE_OK) continue;
      if (k.mode != bin.mode || k.nt != nt) continue;  // same storage mode, the asked thread count
      for (int kc : {25, 50, 100}) {
        Bin cand = bin;
        cand.nt = k.nt;
        cand.npt = k.npt;
        cand.per_sm = k.per_sm;
        cand.smem = std::max(k.smem, size_t(0));
        cand.smem_node = cand.mode == 0 ? node_smem<T>(b, bin.work, k.nt, k.npt) : 0;
        cand.check_every = kc;
        float t = 0.f;
        TRY(run_one(b, cand, a, s));
        TRY(time_bin(cand, t));
        if (t < t_best) {
          t_best = t;
          best = cand;
        }
      }
    }
    bin.nt = best.nt;
    bin.npt = best.npt;
    bin.per_sm = best.per_sm;
    bin.smem = best.smem;
    bin.smem_node = best.smem_node;
    bin.check_every = best.check_every;
    after += t_best;
  }
  // the tangent bins mirror the solve bins' configurations
  for (std::vector<Bin>* tb : {&P.tan_bins, &P.man_bins})
    for (size_t j = 0; j < tb->size() && j < P.bins.size(); ++j) {
      (*tb)[j].nt = P.bins[j].nt;
      (*tb)[j].npt = P.bins[j].npt;
      (*tb)[j].per_sm = P.bins[j].per_sm;
      (*tb)[j].smem = P.bins[j].smem;
      (*tb)[j].smem_node = P.bins[j].smem_node;
      (*tb)[j].cl = P.bins[j].cl;
      (*tb)[j].cl_npt = P.bins[j].cl_npt;
      (*tb)[j].smem_cluster = P.bins[j].smem_cluster;
      (*tb)[j].check_every = P.bins[j].check_every;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RVE_CUDA_TRY(cudaFreeAsync(d_sig, s));
  RVE_CUDA_TRY(cudaFreeAsync(d_it, s));
  RVE_CUDA_TRY(cudaFreeAsync(d_st, s));
  RVE_CUDA_TRY(cudaStreamSynchronize(s));
  if (ms_before) *ms_before = before;
  if (ms_after) *ms_after = after;
  return RVE_OK;
}

}  // namespace
}  // namespace rvegpu

using namespace rvegpu;

extern "C" {

void rve_options_default(rve_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 3e-7;
  o->sigma_tol = 0.0;
  o->max_iter = 200000;
  o->check_every = 50;
  o->precision = RVE_PREC_MIXED;
  o->warm_start = 0;
  o->damping = 0.0;
  o->threads = 0;
  o->damping_mode = RVE_DAMP_VISCOUS;
  o->damping_scale = DAMP_SCALE;
  o->kernel = RVE_KERNEL_AUTO;
}

const char* rve_last_error(void) { return g_error.c_str(); }

int rve_set_options(rve_batch* b, const rve_options* opt) {
  if (!b || !opt) return fail(RVE_EINVAL, "null argument");
  TRY(valid_options(*opt));
  const bool retune = opt->threads != b->opt.threads;
  b->opt = *opt;
  clear_graphs(b);  // options are baked into captured launches
  if (retune) {
    b->pf.ready = false;  // bins depend on the thread count; rebuilt lazily
    b->pd.ready = false;
  }
  return RVE_OK;
}

int rve_batch_create(rve_batch** out, int device, int64_t n_rve, const int64_t* node_off, const double* X,
                     const int64_t* fiber_off, const int32_t* conn, const double* L0, const double* EA,
                     const double* B, const uint8_t* is_boundary, const double* V0, const rve_options* opt) {
  if (!out) return fail(RVE_EINVAL, "out is null");
  *out = nullptr;
  rve_options o;
  rve_options_default(&o);
  if (opt) o = *opt;
  TRY(valid_options(o));
  // host-side validation and layout first: malformed input fails without touching a GPU
  rve_batch* b = new rve_batch();
  b->n_rve = n_rve;
  b->opt = o;
  int rc = build_topology(n_rve, node_off, X, fiber_off, conn, L0, EA, B, is_boundary, V0, b->topo);
  if (rc != RVE_OK) {
    delete b;
    return rc;
  }
  int ndev = 0;
  const cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || device < 0 || device >= ndev) {
    delete b;
    (void)cudaGetLastError();
    return fail(ce != cudaSuccess ? RVE_ECUDA : RVE_EINVAL,
                ce != cudaSuccess ? std::string("no usable CUDA device: ") + cudaGetErrorString(ce)
                                  : std::string("device ordinal out of range"));
  }
  b->device = device;
  auto bail = [&](int rc_) {
    rve_batch_destroy(b);
    return rc_;
  };
  for (const RveMeta& M : b->topo.meta) {
    b->total_nf += M.nf;
    b->total_na += M.na;
    b->total_nb += M.nb;
  }
  if ((rc = set_device(b)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_meta, b->topo.meta)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_fa, b->topo.fa)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_fij, b->topo.fij)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_fb, b->topo.fb)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_csr, b->topo.csr)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_ncsr, b->topo.ncsr)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_nord, b->topo.nord)) != RVE_OK) return bail(rc);
  if ((rc = upload(b, &b->d_ncap, b->topo.ncap)) != RVE_OK) return bail(rc);
  int nf_max = 0, na_max = 0;
  for (const RveMeta& M : b->topo.meta) {
    nf_max = std::max(nf_max, M.nf);
    na_max = std::max(na_max, M.na);
  }
  b->pl_bytes = size_t(plain_scratch_bytes(nf_max, na_max)) + 16 * 256;
  if ((rc = dalloc(b, reinterpret_cast<void**>(&b->d_pl), b->pl_bytes)) != RVE_OK) return bail(rc);
  if ((rc = dalloc(b, reinterpret_cast<void**>(&b->d_pdl_done), sizeof(int32_t))) != RVE_OK) return bail(rc);
  if (cudaMemset(b->d_pdl_done, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(RVE_ECUDA, "cudaMemset failed"));
  if (cudaMallocHost(reinterpret_cast<void**>(&b->h_pl), 64 * sizeof(double)) != cudaSuccess)
    return bail(fail(RVE_ENOMEM, "cudaMallocHost failed"));
  for (int k = 0; k < N_SIDE_STREAMS; ++k) {
    if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(RVE_ECUDA, "stream/event creation failed"));
  }
  if (cudaStreamCreateWithFlags(&b->hstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_work, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_last, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(RVE_ECUDA, "event creation failed"));
  *out = b;
  return RVE_OK;
}

int rve_solve(rve_batch* b, const double* F, double tol, int32_t max_iter, double* sigma, int32_t* iters,
              int32_t* status, void* stream) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (b->n_rve == 0) return RVE_OK;
  if (!F || !sigma) return fail(RVE_EINVAL, "F and sigma are required");
  TRY(set_device(b));
  if (!(tol > 0.0)) tol = b->opt.tol;
  if (max_iter <= 0) max_iter = b->opt.max_iter;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(order_after_last(b, s));
  // graphs need a created stream (the legacy and per-thread default streams cannot be captured);
  // kernel timing records events between launches, so it runs uncaptured
  const bool graphable = b->opt.graphs && !b->timing && b->opt.precision != RVE_PREC_PLAIN_F64 && s != nullptr &&
                         s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (graphable) {
    for (const GraphEntry& g : b->graphs)
      if (g.F == F && g.sigma == sigma && g.iters == iters && g.status == status && g.stream == s && g.tol == tol &&
          g.max_iter == max_iter) {
        RVE_CUDA_TRY(cudaGraphLaunch(g.exec, s));
        RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
        return RVE_OK;
      }
  }
  TRY(solve_all(b, F, tol, max_iter, sigma, iters, status, s));
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  if (graphable && b->graphs.size() < 16) {
    // record the same launch sequence (nothing runs during capture) for replay
    // relaxed mode: only stream work is recorded; the host-side calls of the
    // launch path (error queries, attributes) stay legal during capture
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      (void)cudaGetLastError();  // not capturable: the solve above already ran uncaptured
      return RVE_OK;
    }
    const int rc = solve_all(b, F, tol, max_iter, sigma, iters, status, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &g);  // always leave capture mode
    if (rc != RVE_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();  // do not leak the capture's error into later calls
      if (rc != RVE_OK) return rc;
      return fail(RVE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(RVE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    b->graphs.push_back(GraphEntry{F, sigma, iters, status, s, tol, max_iter, exec});
  }
  return RVE_OK;
}

int rve_solve_subset(rve_batch* b, const int64_t* ids, int64_t m, const double* F, double tol, int32_t max_iter,
                     double* sigma, int32_t* iters, int32_t* status, void* stream) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  TRY(set_device(b));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(order_after_last(b, s));
  TRY(rvegpu::solve_subset(b, ids, m, F, tol, max_iter, sigma, iters, status, s, true, nullptr));
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

}  // extern "C"

namespace rvegpu {
int solve_subset(rve_batch* b, const int64_t* ids, int64_t m, const double* F, double tol, int32_t max_iter,
                 double* sigma, int32_t* iters, int32_t* status, cudaStream_t s, bool fork,
                 const SubsetBuffers* ext) {
  return solve_items(b, ids, nullptr, m, F, tol, max_iter, sigma, iters, status, s, fork, ext, nullptr);
}

int solve_items(rve_batch* b, const int64_t* ids, const int32_t* outs, int64_t m, const double* F, double tol,
                int32_t max_iter, double* sigma, int32_t* iters, int32_t* status, cudaStream_t s, bool fork,
                const SubsetBuffers* ext, const WaveParams* wave) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (m == 0) return RVE_OK;
  if (m < 0 || !ids || !F || !sigma) return fail(RVE_EINVAL, "bad subset arguments");
  if (m > INT32_MAX) return fail(RVE_EINVAL, "subset too large");
  TRY(set_device(b));
  if (!(tol > 0.0)) tol = b->opt.tol;
  if (max_iter <= 0) max_iter = b->opt.max_iter;
  std::vector<uint8_t> seen(size_t(b->n_rve), 0);
  for (int64_t k = 0; k < m; ++k) {
    if (ids[k] < 0 || ids[k] >= b->n_rve) return fail(RVE_EINVAL, "subset id out of range");
    if (seen[ids[k]]++) return fail(RVE_EINVAL, "subset ids must be distinct");
  }
  const int prec = b->opt.precision;
  if (prec == RVE_PREC_PLAIN_F64) {
    if (wave && wave->wave_iters > 0) return fail(RVE_EINVAL, "iteration-level waves need a batched precision");
    TRY(ensure_path<double>(b));
    for (int64_t k = 0; k < m; ++k)
      TRY(plain_solve_one(b, int(ids[k]), outs ? outs[k] : int(k), F, tol, max_iter, sigma, iters, status, s));
    return RVE_OK;
  }
  const bool f32 = prec == RVE_PREC_MIXED;
  if (f32) TRY(ensure_path<float>(b));
  else TRY(ensure_path<double>(b));
  PathState& P = f32 ? b->pf : b->pd;
  // group ids by bin of the all-RVE solve
  std::vector<Bin> bins(P.bins.size());
  for (size_t j = 0; j < bins.size(); ++j) {
    bins[j].mode = P.bins[j].mode;
    bins[j].nt = P.bins[j].nt;
    bins[j].npt = P.bins[j].npt;
    bins[j].per_sm = P.bins[j].per_sm;
    bins[j].smem = P.bins[j].smem;
    bins[j].smem_node = P.bins[j].smem_node;
    bins[j].cl = P.bins[j].cl;
    bins[j].cl_npt = P.bins[j].cl_npt;
    bins[j].smem_cluster = P.bins[j].smem_cluster;
  }
  for (int64_t k = 0; k < m; ++k) {
    const int r = int(ids[k]);
    Work w = P.work_of[r];
    w.out = outs ? outs[k] : int32_t(k);
    bins[P.bin_of[r]].work.push_back(w);
  }
  for (Bin& x : bins)
    std::stable_sort(x.work.begin(), x.work.end(),
                     [&](const Work& p, const Work& q) { return b->topo.meta[p.rve].na > b->topo.meta[q.rve].na; });
  // stage the work lists: caller-provided buffers, or the batch's own set
  SubsetBuffers buf;
  if (ext) {
    if (size_t(m) > ext->cap) return fail(RVE_EINVAL, "subset larger than the caller's work buffers");
    buf = *ext;
  } else {
    RVE_CUDA_TRY(cudaEventSynchronize(b->ev_work));  // previous upload from the pinned staging done
    if (size_t(m) > b->h_work_cap) {
      if (b->h_work_pin) cudaFreeHost(b->h_work_pin);
      b->h_work_pin = nullptr;
      const size_t cap = std::max<size_t>(size_t(m), 1024);
      RVE_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&b->h_work_pin), cap * sizeof(Work)));
      b->h_work_cap = cap;
    }
    if (size_t(m) > P.sub_cap) {
      void* p = nullptr;
      void* q = nullptr;
      TRY(dalloc(b, &p, std::max<size_t>(size_t(m), 1024) * sizeof(Work)));
      TRY(dalloc(b, &q, std::max<size_t>(size_t(m), 1024) * sizeof(Work)));
      P.d_sub_work = static_cast<Work*>(p);
      P.d_sub_sorted = static_cast<Work*>(q);
      P.sub_cap = std::max<size_t>(size_t(m), 1024);
    }
    buf.d_work = P.d_sub_work;
    buf.d_sorted = P.d_sub_sorted;
    buf.h_stage = b->h_work_pin;
    buf.cap = P.sub_cap;
  }
  size_t off = 0;
  for (Bin& x : bins) {
    std::copy(x.work.begin(), x.work.end(), buf.h_stage + off);
    x.d_work = buf.d_work + off;
    x.d_sorted = buf.d_sorted + off;
    x.n = int(x.work.size());
    off += x.work.size();
  }
  RVE_CUDA_TRY(cudaMemcpyAsync(buf.d_work, buf.h_stage, off * sizeof(Work), cudaMemcpyHostToDevice, s));
  if (!ext) RVE_CUDA_TRY(cudaEventRecord(b->ev_work, s));
  if (f32) {
    DrArgs<float> a = make_args<float>(b, F, tol, max_iter, sigma, iters, status, b->pf.d_state, b->opt.warm_start);
    if (wave) {
      a.wave_iters = wave->wave_iters;
      a.resume = wave->resume;
      a.vel = static_cast<float*>(wave->vel);
    }
    return run_bins(b, bins, a, s, fork);
  }
  DrArgs<double> a = make_args<double>(b, F, tol, max_iter, sigma, iters, status, b->pd.d_state, b->opt.warm_start);
  if (wave) {
    a.wave_iters = wave->wave_iters;
    a.resume = wave->resume;
    a.vel = static_cast<double*>(wave->vel);
  }
  return run_bins(b, bins, a, s, fork);
}

int ensure_batched_path(rve_batch* b) {
  if (b->opt.precision == RVE_PREC_MIXED) return ensure_path<float>(b);
  return ensure_path<double>(b);
}
}  // namespace rvegpu

extern "C" {

int rve_solve_host(rve_batch* b, const double* F, double tol, int32_t max_iter, double* sigma, int32_t* iters,
                   int32_t* status) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (b->n_rve == 0) return RVE_OK;
  if (!F || !sigma) return fail(RVE_EINVAL, "F and sigma are required");
  TRY(set_device(b));
  const size_t n = size_t(b->n_rve);
  if (!b->d_hF) {
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_hF), 9 * n * sizeof(double)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_hS), 9 * n * sizeof(double)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_hI), n * sizeof(int32_t)));
    TRY(dalloc(b, reinterpret_cast<void**>(&b->d_hSt), n * sizeof(int32_t)));
    const size_t bytes = 9 * n * sizeof(double) * 2 + 2 * n * sizeof(int32_t);
    RVE_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&b->h_pin), bytes));
    b->h_pin_bytes = bytes;
  }
  double* pF = b->h_pin;
  double* pS = b->h_pin + 9 * n;
  int32_t* pI = reinterpret_cast<int32_t*>(b->h_pin + 18 * n);
  int32_t* pSt = pI + n;
  std::memcpy(pF, F, 9 * n * sizeof(double));
  cudaStream_t s = b->hstream;
  RVE_CUDA_TRY(cudaMemcpyAsync(b->d_hF, pF, 9 * n * sizeof(double), cudaMemcpyHostToDevice, s));
  TRY(rve_solve(b, b->d_hF, tol, max_iter, b->d_hS, b->d_hI, b->d_hSt, s));
  RVE_CUDA_TRY(cudaMemcpyAsync(pS, b->d_hS, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  RVE_CUDA_TRY(cudaMemcpyAsync(pI, b->d_hI, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RVE_CUDA_TRY(cudaMemcpyAsync(pSt, b->d_hSt, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RVE_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(sigma, pS, 9 * n * sizeof(double));
  if (iters) std::memcpy(iters, pI, n * sizeof(int32_t));
  if (status) std::memcpy(status, pSt, n * sizeof(int32_t));
  return RVE_OK;
}

int rve_tangent(rve_batch* b, const double* F, double h, double tol, int32_t max_iter, double* sigma,
                double* dsigma_dF, int32_t* status, void* stream) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (b->n_rve == 0) return RVE_OK;
  if (!F || !sigma || !dsigma_dF) return fail(RVE_EINVAL, "F, sigma and dsigma_dF are required");
  TRY(set_device(b));
  if (!(h > 0.0)) h = 1e-4;
  if (!(tol > 0.0)) tol = b->opt.tol;
  if (max_iter <= 0) max_iter = b->opt.max_iter;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->opt.precision != RVE_PREC_MIXED && b->opt.precision != RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "rve_tangent needs a batched precision (RVE_PREC_MIXED or RVE_PREC_BATCHED_F64)");
  TRY(order_after_last(b, s));
  if (b->opt.precision == RVE_PREC_MIXED) TRY(tangent_batched<float>(b, F, h, tol, max_iter, sigma, dsigma_dF, status, s));
  else TRY(tangent_batched<double>(b, F, h, tol, max_iter, sigma, dsigma_dF, status, s));
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

int rve_set_kernel_timing(rve_batch* b, int32_t on) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (on != 0 && on != 1) return fail(RVE_EINVAL, "on must be 0 or 1");
  b->timing = on != 0;
  b->n_kev = 0;
  return RVE_OK;
}

int rve_last_kernel_ms(rve_batch* b, int32_t max, double* ms) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (max > 0 && !ms) return fail(RVE_EINVAL, "ms is required when max > 0");
  TRY(set_device(b));
  const int32_t n = int32_t(b->n_kev);
  for (int32_t k = 0; k < n && k < max; ++k) {
    RVE_CUDA_TRY(cudaEventSynchronize(b->kev[2 * size_t(k) + 1]));
    float t = 0.0f;
    RVE_CUDA_TRY(cudaEventElapsedTime(&t, b->kev[2 * size_t(k)], b->kev[2 * size_t(k) + 1]));
    ms[k] = double(t);
  }
  return n;
}

int rve_energy(rve_batch* b, int32_t precision, double* energy, void* stream) {
  if (!b || !energy) return fail(RVE_EINVAL, "batch and energy are required");
  if (precision != RVE_PREC_MIXED && precision != RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "energy records exist on the batched precisions");
  const PathState& P = precision == RVE_PREC_MIXED ? b->pf : b->pd;
  if (!P.d_energy) return fail(RVE_EINVAL, "no energy records: solve with the option energy_check = 1 first");
  TRY(set_device(b));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(order_after_last(b, s));
  RVE_CUDA_TRY(cudaMemcpyAsync(energy, P.d_energy, sizeof(double) * 6 * size_t(b->n_rve), cudaMemcpyDeviceToDevice, s));
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

int rve_orientation(rve_batch* b, const double* F, int32_t precision, double* omega, void* stream) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (b->n_rve == 0) return RVE_OK;
  if (!F || !omega) return fail(RVE_EINVAL, "F and omega are required");
  if (precision != RVE_PREC_PLAIN_F64 && precision != RVE_PREC_MIXED && precision != RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "unknown precision");
  TRY(set_device(b));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(order_after_last(b, s));
  const PathState& P = precision == RVE_PREC_MIXED ? b->pf : b->pd;
  const double* state = P.ready ? static_cast<const double*>(P.d_state) : nullptr;
  const uint8_t* valid = P.ready ? P.d_valid : nullptr;
  const int64_t n = b->n_rve;
  for (int64_t r0 = 0; r0 < n; r0 += 65535) {  // grid.x limit of a launch over RVEs
    const int64_t m = std::min<int64_t>(65535, n - r0);
    orient_kernel<<<unsigned(m), ORIENT_THREADS, 0, s>>>(b->d_meta, b->d_fa, b->d_fij, b->d_fb, state, valid, F,
                                                          omega, r0);
    RVE_CUDA_TRY(cudaGetLastError());
  }
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

int rve_tangent_mandel(rve_batch* b, const double* F, double h, double tol, int32_t max_iter, double* sigma,
                       double* C, int32_t* status, void* stream) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  if (b->n_rve == 0) return RVE_OK;
  if (!F || !sigma || !C) return fail(RVE_EINVAL, "F, sigma and C are required");
  TRY(set_device(b));
  if (!(h > 0.0)) h = 1e-4;
  if (!(tol > 0.0)) tol = b->opt.tol;
  if (max_iter <= 0) max_iter = b->opt.max_iter;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->opt.precision != RVE_PREC_MIXED && b->opt.precision != RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "rve_tangent_mandel needs a batched precision (RVE_PREC_MIXED or RVE_PREC_BATCHED_F64)");
  TRY(order_after_last(b, s));
  if (b->opt.precision == RVE_PREC_MIXED) TRY(mandel_batched<float>(b, F, h, tol, max_iter, sigma, C, status, s));
  else TRY(mandel_batched<double>(b, F, h, tol, max_iter, sigma, C, status, s));
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

int rve_reset_state(rve_batch* b, const int64_t* ids, int64_t m) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  TRY(set_device(b));
  RVE_CUDA_TRY(cudaDeviceSynchronize());
  for (PathState* P : {&b->pf, &b->pd}) {
    if (!P->ready) continue;
    if (!ids) {
      RVE_CUDA_TRY(cudaMemset(P->d_valid, 0, size_t(std::max<int64_t>(b->n_rve, 1))));
      continue;
    }
    for (int64_t k = 0; k < m; ++k) {
      if (ids[k] < 0 || ids[k] >= b->n_rve) return fail(RVE_EINVAL, "reset id out of range");
      RVE_CUDA_TRY(cudaMemset(P->d_valid + ids[k], 0, 1));
    }
  }
  return RVE_OK;
}

int rve_autotune(rve_batch* b, const double* F, int32_t reps, void* stream, double* ms_before, double* ms_after) {
  if (!b || !F) return fail(RVE_EINVAL, "batch and F are required");
  if (b->n_rve == 0) return RVE_OK;
  if (reps < 1) reps = 1;
  TRY(set_device(b));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(order_after_last(b, s));
  int rc;
  clear_graphs(b);  // bin configurations are baked into captured launches
  if (b->opt.precision == RVE_PREC_MIXED) rc = autotune_path<float>(b, F, reps, s, ms_before, ms_after);
  else if (b->opt.precision == RVE_PREC_BATCHED_F64) rc = autotune_path<double>(b, F, reps, s, ms_before, ms_after);
  else return fail(RVE_EINVAL, "the autotuner tunes the batched precisions");
  if (rc != RVE_OK) return rc;
  RVE_CUDA_TRY(cudaEventRecord(b->ev_last, s));
  return RVE_OK;
}

int rve_batch_get_bins(const rve_batch* b, int32_t precision, int32_t max, rve_bin_info* out) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  const PathState& P = precision == RVE_PREC_BATCHED_F64 ? b->pd : b->pf;
  if (!P.ready) return 0;
  int n = 0;
  for (const Bin& x : P.bins) {
    if (n >= max) break;
    if (out) {
      out[n].n_rve = x.n;
      out[n].mode = x.mode;
      out[n].threads = x.nt;
      out[n].nodes_per_thread = x.npt;
      out[n].ctas_per_sm = x.per_sm;
      out[n].check_every = x.check_every > 0 ? x.check_every : b->opt.check_every;
      const bool alt = b->opt.kernel == RVE_KERNEL_NODE && !b->opt.energy_check &&
                       b->opt.damping_mode == RVE_DAMP_VISCOUS;
      out[n].kernel = 0;
      out[n].cluster = 0;
      out[n].exclusive = P.bins.size() == 1 ? excl_count(x) : 0;
      out[n].sorted = (x.d_sorted && x.n > 1 && x.n <= LPT_MAX) ? 1 : 0;
      out[n].smem_bytes = int64_t(x.smem);
      if (alt && x.mode == 0 && x.smem_node > 0) {
        out[n].kernel = 1;
        out[n].smem_bytes = int64_t(x.smem_node);
      } else if (alt && x.mode != 0 && x.cl > 0) {
        out[n].kernel = 2;
        out[n].cluster = x.cl;
        out[n].threads = CLUSTER_NT;
        out[n].nodes_per_thread = x.cl_npt;
        out[n].smem_bytes = int64_t(x.smem_cluster);
      }
    }
    ++n;
  }
  return n;
}

int rve_batch_get_info(const rve_batch* b, rve_batch_info* info) {
  if (!b || !info) return fail(RVE_EINVAL, "null argument");
  info->n_rve = b->n_rve;
  info->free_nodes = b->total_nf;
  info->active_fibers = b->total_na;
  info->fixed_fibers = b->total_nb;
  info->pruned_fibers = b->topo.pruned_fibers;
  info->n_bins = int64_t(std::max(b->pf.bins.size(), b->pd.bins.size()));
  info->device_bytes = int64_t(b->device_bytes);
  return RVE_OK;
}

int rve_batch_get_sizes(const rve_batch* b, int32_t* free_nodes, int32_t* active_fibers, int32_t* fixed_fibers) {
  if (!b) return fail(RVE_EINVAL, "null batch");
  for (int64_t r = 0; r < b->n_rve; ++r) {
    const RveMeta& M = b->topo.meta[r];
    if (free_nodes) free_nodes[r] = M.nf;
    if (active_fibers) active_fibers[r] = M.na;
    if (fixed_fibers) fixed_fibers[r] = M.nb;
  }
  return RVE_OK;
}

int rve_get_positions(rve_batch* b, int64_t r, const double* F, int32_t precision, double* x_out) {
  if (!b || !F || !x_out) return fail(RVE_EINVAL, "null argument");
  if (r < 0 || r >= b->n_rve) return fail(RVE_EINVAL, "RVE index out of range");
  TRY(set_device(b));
  const RveMeta& M = b->topo.meta[r];
  const int64_t n0 = b->topo.node_off_in[r];
  for (int i = 0; i < M.n_nodes; ++i)
    for (int k = 0; k < 3; ++k) {
      const double* X = &b->topo.X_in[3 * (n0 + i)];
      x_out[3 * i + k] = F[3 * k] * X[0] + F[3 * k + 1] * X[1] + F[3 * k + 2] * X[2];
    }
  const bool f32 = precision == RVE_PREC_MIXED;
  PathState& P = f32 ? b->pf : b->pd;
  if (!P.ready || M.nf == 0) return RVE_OK;
  RVE_CUDA_TRY(cudaDeviceSynchronize());
  uint8_t valid = 0;
  RVE_CUDA_TRY(cudaMemcpy(&valid, P.d_valid + r, 1, cudaMemcpyDeviceToHost));
  if (!valid) return RVE_OK;
  std::vector<double> h(4 * size_t(M.nf));
  RVE_CUDA_TRY(cudaMemcpy(h.data(), static_cast<double*>(P.d_state) + 4 * size_t(M.node_off),
                          h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int a = 0; a < M.nf; ++a) {
    const int i = b->topo.free_node_id[M.node_off + a];
    for (int k = 0; k < 3; ++k) x_out[3 * i + k] += h[4 * a + k];
  }
  return RVE_OK;
}

int rve_set_positions(rve_batch* b, int64_t r, const double* F, int32_t precision, const double* x) {
  if (!b || !F || !x) return fail(RVE_EINVAL, "null argument");
  if (r < 0 || r >= b->n_rve) return fail(RVE_EINVAL, "RVE index out of range");
  if (precision != RVE_PREC_MIXED && precision != RVE_PREC_BATCHED_F64)
    return fail(RVE_EINVAL, "set positions on a batched precision (the plain path shares the FP64 state)");
  TRY(set_device(b));
  if (precision == RVE_PREC_MIXED) TRY(ensure_path<float>(b));
  else TRY(ensure_path<double>(b));
  PathState& P = precision == RVE_PREC_MIXED ? b->pf : b->pd;
  const RveMeta& M = b->topo.meta[r];
  RVE_CUDA_TRY(cudaDeviceSynchronize());  // no solve may be using the state
  if (M.nf > 0) {
    const int64_t n0 = b->topo.node_off_in[r];
    std::vector<double> h(4 * size_t(M.nf), 0.0);
    for (int a = 0; a < M.nf; ++a) {
      const int i = b->topo.free_node_id[M.node_off + a];
      const double* X = &b->topo.X_in[3 * (n0 + i)];
      for (int k = 0; k < 3; ++k)
        h[4 * a + k] = x[3 * i + k] - (F[3 * k] * X[0] + F[3 * k + 1] * X[1] + F[3 * k + 2] * X[2]);
    }
    RVE_CUDA_TRY(cudaMemcpy(static_cast<double*>(P.d_state) + 4 * size_t(M.node_off), h.data(),
                            h.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  const uint8_t one = 1;
  RVE_CUDA_TRY(cudaMemcpy(P.d_valid + r, &one, 1, cudaMemcpyHostToDevice));
  return RVE_OK;
}

void rve_batch_destroy(rve_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  clear_graphs(b);
  for (cudaEvent_t e : b->kev) cudaEventDestroy(e);
  for (void* p : b->allocations) cudaFree(p);
  for (int k = 0; k < N_SIDE_STREAMS; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->hstream) cudaStreamDestroy(b->hstream);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_work) cudaEventDestroy(b->ev_work);
  if (b->ev_last) cudaEventDestroy(b->ev_last);
  if (b->h_pl) cudaFreeHost(b->h_pl);
  if (b->h_pin) cudaFreeHost(b->h_pin);
  if (b->h_work_pin) cudaFreeHost(b->h_work_pin);
  delete b;
}

}  // extern "C"
