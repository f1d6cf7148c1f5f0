// Internal data layout of an RVE batch (host and device).
//
// Storage is structure-of-arrays with per-RVE offsets: every RVE's free
// nodes, active fibers (at least one free end), boundary-to-boundary
// fibers and CSR entries sit in contiguous segments of batch-wide arrays
// (the packed row-offset/value layout of the paper's PackedView, Sec. 4.3).
// Free nodes are numbered 0..nf-1 inside an RVE; fixed (boundary) nodes
// are not stored at all: under the affine boundary condition their
// fluctuation h = x - F X is identically zero (Eq. affine-bc vs
// Eq. micro_coords), so a fiber end on the boundary reads the zero slot nf.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace rvegpu {

// Static per-fiber record, double precision (read once per solve).
struct FibD {
  double dx, dy, dz;  // X_j - X_i (reference chord)
  double L0, EA, B;
  double half_inv_L02;  // 1 / (2 L0^2): Green strain without a division on the device
};

// Per-RVE metadata, one per RVE on the device.
struct RveMeta {
  int32_t nf;       // free nodes kept
  int32_t na;       // active fibers
  int32_t nb;       // boundary-to-boundary fibers
  int32_t n_nodes;  // nodes in the input (for position export)
  int32_t node_off; // offset into per-free-node arrays
  int32_t fa_off;   // offset into active-fiber arrays
  int32_t fb_off;   // offset into boundary-fiber arrays
  int32_t csr_off;  // offset into CSR entries (a multiple of 4)
  int32_t csr_len;  // CSR entries of this RVE (each node's run padded to 4)
  int32_t pad_;
  double V0;        // reference volume
  double sum_EA;    // sum of EA over kept fibers (absolute residual floor)
};

// One unit of work of a batched launch: solve RVE `rve` with F[9*out..],
// write outputs at index `out`, keep the fluctuation state at
// state_off (in free nodes) of the state buffer.
struct Work {
  int32_t rve;
  int32_t out;
  int32_t state_off;
  int32_t kind;     // 0: the RVE's own state slot (warm start if enabled and
                    //    valid, marks it valid); 1: scratch slot, always warm
  int32_t scr_off;  // streamed bins: offset (in fibers) of this item's
                    // global P0/P1/SCR scratch
  int32_t pad;
};

// Loop state of a solve parked between the launches of an iteration-level
// serving wave (one per RVE; the velocity is kept per free node beside it).
struct ResumeRec {
  int32_t it;        // DR iterations done so far
  int32_t n_checks;  // convergence checks done (rebase schedule)
  double c;          // damping coefficient in use
  float ke_prev;     // kinetic damping: kinetic energy of the last step
  int32_t kin_half;  // kinetic damping: next step starts from rest
  int32_t active;    // 1: parked, resume from this record; 0: start afresh
  int32_t pad;
};
constexpr int RVE_STATUS_PARKED_INTERNAL = 4;  // == RVE_STATUS_RUNNING

// Loop variants of the fused kernel (template parameter VAR).
constexpr int VAR_VISCOUS = 0;
constexpr int VAR_KINETIC = 1;
constexpr int VAR_ENERGY = 2;

// Dynamic-relaxation constants of the explicit update (Sec. 3.2: the
// mass, damping and time step are fictitious and chosen for speed).
//   lumped mass   m_i = MASS_GAMMA * (dt^2/4) * sum_e 2 max(k_e, |N_e|/l_e),
//                 dt = 1, re-evaluated every iteration from the current state
//                 (a Gershgorin bound on the stiffness, so the central
//                 difference step stays stable as fibers stiffen);
//   step cap      |x_i^{n+1} - x_i^n| <= STEP_CAP * min_{e at i} L0_e;
//   damping       c0 at start, then c = DAMP_SCALE * 2 sqrt(lambda), c <= C_MAX,
//                 lambda the Rayleigh quotient v.K v / v.M v of the last
//                 step's velocity: critical damping of a mode with that
//                 eigenvalue.  The quotient sits above the slowest mode's
//                 eigenvalue, and a scale of 0.7 takes about 20 % fewer
//                 iterations, but with it one 16^3 uneven RVE solved in FP64
//                 to 1e-10 stopped on a weakly unstable equilibrium that the
//                 oracle could not certify stable; the default DAMP_SCALE is
//                 1.0 and the option damping_scale sets another.
#ifndef RVE_MASS_GAMMA
#define RVE_MASS_GAMMA 1.1
#endif
constexpr double MASS_GAMMA = RVE_MASS_GAMMA;
constexpr double MASS_COEF = MASS_GAMMA * 0.25 * 2.0;
constexpr double STEP_CAP = 0.1;
constexpr double DAMP_C0 = 0.1;
constexpr double DAMP_C_MAX = 1.9;
constexpr double DAMP_SCALE = 1.0;
constexpr double ABS_FLOOR = 1e-16;  // absolute residual floor per unit EA
#ifndef RVE_REBASE_EVERY
#define RVE_REBASE_EVERY 4
#endif
constexpr int REBASE_EVERY = RVE_REBASE_EVERY;  // FP32 path: rebase the reference state every 4 checks
// stress-convergence estimate: stress and residual compared SIG_WINDOW
// checks apart, contraction ratio capped at SIG_RHO_CAP
constexpr int SIG_WINDOW = 2;
constexpr double SIG_RHO_CAP = 0.95;

// Shared-memory footprint of one RVE held by the fused kernel.
// resident: P0, P1 (one 4-vector each per active fiber), SCR (na+1
// 4-vectors: slot na stays zero for CSR padding), H (nf+1 4-vectors), CSR
// entries (csr_len u16) and a reduction buffer.
// streamed: H and SCR only when they fit, otherwise H and the FP64
// reference copy.
__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline size_t red_bytes(int nt) { return align_up(size_t(nt / 32) * 12 * sizeof(double) + 256, 16); }  // >= 6 per warp + 32
// The fiber-scratch region also holds the FP64 reference state (3 doubles
// per node) during a rebase, so it is the larger of the two.
template <typename T>
__host__ __device__ inline size_t scr_region_bytes(int nf, int na) {
  const size_t a = size_t(na + 1) * 4 * sizeof(T), b = size_t(nf + 1) * 3 * sizeof(double);
  return a > b ? a : b;
}
template <typename T>
inline size_t smem_resident(int nf, int na, int csr_len, int nt) {
  const size_t v4 = 4 * sizeof(T);
  return 2 * align_up(size_t(na) * v4, 16) + align_up(scr_region_bytes<T>(nf, na), 16) +
         align_up(size_t(nf + 1) * v4, 16) + align_up(size_t(csr_len) * sizeof(uint16_t), 16) + red_bytes(nt);
}
template <typename T>
inline size_t smem_streamed(int nf, int na, int nt, bool scr_in_smem) {
  const size_t v4 = 4 * sizeof(T);
  return align_up(size_t(nf + 1) * v4, 16) +
         (scr_in_smem ? align_up(scr_region_bytes<T>(nf, na), 16)
                      : align_up(size_t(nf + 1) * 3 * sizeof(double), 16)) +
         red_bytes(nt);
}

// Node-centric layout (dr_node_kernel): two H buffers (nf+1 4-vectors each),
// the reduction buffer, then per incidence slot two 4-vectors (chord/strain
// and law parameters), `slots` slots per thread (the busiest thread's
// count) for nt threads.
template <typename T>
inline size_t smem_node(int nf, int slots, int nt) {
  const size_t v4 = 4 * sizeof(T);
  return 2 * align_up(size_t(nf + 1) * v4, 16) + red_bytes(nt) + size_t(slots) * 2 * size_t(nt) * v4;
}
// Cluster layout (dr_cluster_kernel), per CTA: two replicas of the H
// buffers (nf+1 4-vectors each), the reduction buffer, CTA 0's gather rows
// (8 x 12 doubles), then the incidence slots of the CTA's threads.
constexpr int CLUSTER_NT = 512;  // threads per CTA of the cluster kernel
constexpr int CLUSTER_MAX = 8;   // CTAs per cluster (the portable limit)
template <typename T>
inline size_t smem_cluster(int nf, int slots, int nt) {
  const size_t v4 = 4 * sizeof(T);
  return 2 * align_up(size_t(nf + 1) * v4, 16) + red_bytes(nt) + align_up(8 * 12 * sizeof(double), 16) +
         size_t(slots) * 2 * size_t(nt) * v4;
}
// Free node dealt to thread t as its q-th node: position in the
// decreasing-degree order, snaking (q even: q nt + t; q odd: (q+1) nt - 1 - t)
// so that each thread's total is balanced.
__host__ __device__ inline int node_rank(int q, int t, int nt) { return (q & 1) ? (q + 1) * nt - 1 - t : q * nt + t; }

constexpr int NODES_PER_THREAD = 4;  // free nodes owned per thread (registers)
constexpr int MAX_THREADS = 1024;
constexpr size_t SMEM_LIMIT = 232448;  // 227 KB opt-in per CTA

// Arguments of the fused batched kernel.
template <typename T>
struct DrArgs {
  const RveMeta* meta;
  const FibD* fa;          // active fibers
  const uint32_t* fij;     // packed endpoints i | j << 16 (nf = boundary zero slot)
  const FibD* fb;          // boundary-to-boundary fibers
  const uint16_t* csr;     // per free node: (active fiber << 1) | (node is endpoint j), runs padded to 4
                           // entries with (na << 1) (the zero scratch slot)
  const uint32_t* ncsr;    // per free node: (local CSR begin << 8) | count
  const float* ncap;       // per free node: STEP_CAP * min incident L0
  const uint16_t* nord;    // per RVE (node offsets): free nodes by decreasing degree
  int32_t node_kernel;     // 1: resident bins run dr_node_kernel, streamed bins with a cluster layout dr_cluster_kernel
  const Work* work;
  int32_t n_work;
  const double* F;         // 9 per output index
  double* sigma;           // 9 per output index
  int32_t* iters;          // per output index (may be null)
  int32_t* status;         // per output index (may be null)
  double* state;           // 4 per state node: FP64 fluctuation h (x, y, z, unused)
  uint8_t* valid;          // per RVE: own state slot holds a solve
  int32_t* last_iters;     // per RVE: iterations of its last own-slot solve (scheduling cost)
  int32_t warm_start;
  // streamed bins: per-solve scratch in global memory (Work::scr_off)
  T* gP0;
  T* gP1;
  T* gSCR;
  double tol;
  int32_t max_iter;
  int32_t check_every;
  double damping;          // > 0 fixed, <= 0 adaptive
  double sigma_tol;        // > 0: also require the estimated stress error <= sigma_tol
  int32_t kinetic;         // 1: kinetic damping (no viscous term, velocity reset after a kinetic-energy peak)
  double damping_scale;    // s in the adaptive damping c = s * 2 sqrt(lambda)
  // iteration-level waves (serving): with wave_iters > 0 a solve stops at the
  // first check at least wave_iters iterations after this launch took it up,
  // parks (state h, velocity, ResumeRec) and reports RVE_STATUS_RUNNING; the
  // next launch of the same RVE resumes it.  resume == nullptr: no parking.
  int32_t wave_iters;
  ResumeRec* resume;       // per RVE
  T* vel;                  // 4 T per state node (velocity of a parked solve)
  double* energy;          // non-null: energy-balance variant, 6 doubles per output index
  // non-null: this launch is a programmatic dependent of the launch before
  // it on its stream (the rest of a bin whose costliest RVEs run there); its
  // last CTA waits for that launch before it exits (counter, reset by it)
  int32_t* pdl_done;
};

}  // namespace rvegpu

// ---------------------------------------------------------------- host side
#include <string>
#include <vector>

#include "rve.h"

namespace rvegpu {

// Per-thread error message behind rve_last_error().
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// Host copy of one RVE's processed topology (after pruning/renumbering).
struct HostTopology {
  std::vector<RveMeta> meta;
  std::vector<FibD> fa, fb;
  std::vector<uint32_t> fij;
  std::vector<uint16_t> csr;
  std::vector<uint32_t> ncsr;
  std::vector<float> ncap;
  std::vector<uint16_t> nord;         // per RVE: free nodes by decreasing degree
  std::vector<int32_t> free_node_id;  // original RVE-local id of each free node
  std::vector<int64_t> node_off_in;   // input node offsets (position export)
  std::vector<double> X_in;           // input coordinates (position export)
  int64_t pruned_fibers = 0;
};

// Validate, prune and lay out the input networks.  Returns RVE_OK or RVE_EINVAL.
int build_topology(int64_t n_rve, const int64_t* node_off, const double* X, const int64_t* fiber_off,
                   const int32_t* conn, const double* L0, const double* EA, const double* B,
                   const uint8_t* is_boundary, const double* V0, HostTopology& out);

}  // namespace rvegpu
