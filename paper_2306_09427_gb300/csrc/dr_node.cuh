// Node-centric fused dynamic-relaxation kernel: one CTA solves one RVE, and
// every thread owns NPT free nodes and evaluates the fibers incident to them
// itself (resident RVEs, viscous damping).
//
// The arithmetic per DR iteration is that of dr_fused_kernel (Algorithm 2,
// Sec. 3.2, in the fluctuation form with the FP64 reference state and the
// rebase; see dr_fused.cuh): fiber force, damped central-difference update
// with the per-iteration Gershgorin mass and step cap, residual and damping
// checks every check_every iterations, compensated FP64 stress at the end.
// What differs is where the fiber forces are formed.  dr_fused_kernel runs
// a fiber phase (one thread per fiber, forces to a shared scratch), a
// barrier, a node phase (a CSR gather of that scratch) and a second
// barrier.  Here the owner of a free node walks its own incidence slots: per
// slot it reads the far end's correction, forms the fiber force and adds it
// to the node's force in registers.  A fiber with two free ends is then
// evaluated by both owners (about 1.8x the fiber arithmetic on these
// networks), but the scratch store, the CSR read, the scratch gather and one
// barrier per iteration are gone, and the two evaluations give exactly
// opposite forces: exchanging the ends negates the chord, the correction
// difference and every vector built from them, and leaves the strain, the
// length and the law unchanged, operation by operation in IEEE arithmetic.
//
// Shared memory per RVE:
//   H0, H1  correction d = h - h_ref of every free node and the zero slot nf
//           (boundary ends, h = 0 under the affine BC, Eq. affine-bc), held
//           at the node's rank in the decreasing-degree order, so that the
//           owners of consecutive positions are consecutive threads;
//           double-buffered: iteration n reads one and writes the other, so
//           one barrier per iteration orders the writes before the reads;
//   red     reduction partials;
//   PP      per incidence slot of a thread: the chord g = x_far - x_own at the
//           reference state and the reference Green strain, then the law
//           (1/(2 L0^2), EA/B, B, far end's position); slot s of thread t at
//           PP[(2 s) NT + t] and PP[(2 s + 1) NT + t], so a warp reads one
//           slot of its 32 threads as one contiguous 512-byte row.
// Free nodes are dealt to threads in decreasing-degree order (node_rank), so
// the nodes that a warp owns at one time have nearly equal degrees and the
// per-node slot loops do not diverge much, and the snake order balances
// each thread's total slot count.
#pragma once

#include "dr_fused.cuh"

namespace rvegpu {

// Owned nodes of a thread, passed by value to the out-of-line parts.
template <int NPT>
struct OwnSet {
  int own[NPT];  // free node, or -1
  int deg[NPT];  // incidence slots of the node
  int off[NPT];  // first slot of the node
};

// Rebase of a thread's incidence slots: chord g = +-F dX_e + h_ref,far -
// h_ref,own and the reference Green strain, in FP64, rounded to the loop
// type; h_ref is read from the FP64 state that the owners have just written
// (plain loads: the read-only path would not see writes of this launch).
// Walks the owned nodes' CSR runs in global memory (once per REBASE_EVERY
// checks).  Out of line, like rebase_fibers.
template <typename T, typename V4, int NT, int NPT>
__device__ __noinline__ void node_rebase_slots(const DrArgs<T>& A, const RveMeta& M, const OwnSet<NPT> os,
                                               const double* sF, const double* st, V4* PP) {
  const int tid = threadIdx.x;
  const FibD* __restrict__ fa = A.fa + M.fa_off;
  const uint32_t* __restrict__ fij = A.fij + M.fa_off;
  const uint16_t* __restrict__ csr = A.csr + M.csr_off;
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = os.own[q];
    if (a < 0) continue;
    const uint32_t w = A.ncsr[M.node_off + a];
    const uint32_t b0 = w >> 8, n = w & 0xffu;
    const double ax = st[4 * a + 0], ay = st[4 * a + 1], az = st[4 * a + 2];
    int s = os.off[q];
    for (uint32_t k = 0; k < n; ++k) {
      const uint32_t x = csr[b0 + k];
      const uint32_t e = x >> 1;
      if (e >= uint32_t(M.na)) continue;  // padding (zero slot)
      const uint32_t ij = fij[e];
      const uint32_t far = (x & 1u) ? (ij & 0xffffu) : (ij >> 16);
      const FibD f = fa[e];
      const double cx = sF[0] * f.dx + sF[1] * f.dy + sF[2] * f.dz;
      const double cy = sF[3] * f.dx + sF[4] * f.dy + sF[5] * f.dz;
      const double cz = sF[6] * f.dx + sF[7] * f.dy + sF[8] * f.dz;
      const bool is_j = (x & 1u) != 0;
      const bool fb = far == uint32_t(M.nf);  // boundary end: h_ref = 0
      const double fx = fb ? 0.0 : st[4 * far + 0], fy = fb ? 0.0 : st[4 * far + 1], fz = fb ? 0.0 : st[4 * far + 2];
      const double gx = (is_j ? -cx : cx) + (fx - ax);
      const double gy = (is_j ? -cy : cy) + (fy - ay);
      const double gz = (is_j ? -cz : cz) + (fz - az);
      V4 p0;
      p0.x = T(gx);
      p0.y = T(gy);
      p0.z = T(gz);
      p0.w = T((gx * gx + gy * gy + gz * gz - f.L0 * f.L0) * f.half_inv_L02);
      PP[size_t(2 * s) * NT + tid] = p0;
      ++s;
    }
  }
}

// Law parameters of a thread's incidence slots (once per solve) and the
// slot layout of its nodes.  Returns the owned-node set.
template <typename T, typename V4, int NT, int NPT>
__device__ __noinline__ OwnSet<NPT> node_setup_slots(const DrArgs<T>& A, const RveMeta& M, const uint16_t* rank_of,
                                                     V4* PP, int g = -1, int ntc = NT) {
  const int tid = threadIdx.x;
  if (g < 0) g = tid;
  const FibD* __restrict__ fa = A.fa + M.fa_off;
  const uint32_t* __restrict__ fij = A.fij + M.fa_off;
  const uint16_t* __restrict__ csr = A.csr + M.csr_off;
  OwnSet<NPT> os;
  int s = 0;
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int k = node_rank(q, g, ntc);
    const int a = k < M.nf ? int(A.nord[M.node_off + k]) : -1;
    os.own[q] = a;
    os.off[q] = s;
    if (a >= 0) {
      const uint32_t w = A.ncsr[M.node_off + a];
      const uint32_t b0 = w >> 8, n = w & 0xffu;
      for (uint32_t kk = 0; kk < n; ++kk) {
        const uint32_t x = csr[b0 + kk];
        const uint32_t e = x >> 1;
        if (e >= uint32_t(M.na)) continue;
        const uint32_t ij = fij[e];
        const uint32_t far = (x & 1u) ? (ij & 0xffffu) : (ij >> 16);
        const FibD f = fa[e];
        V4 p1;
        p1.x = T(f.half_inv_L02);
        p1.y = T(f.B > 0.0 ? f.EA / f.B : f.EA);
        p1.z = T(f.B);
        p1.w = k_pack_ij(far == uint32_t(M.nf) ? uint32_t(M.nf) : uint32_t(rank_of[far]), T(0));  // far end's H position
        PP[size_t(2 * s + 1) * NT + tid] = p1;
        ++s;
      }
    }
    os.deg[q] = s - os.off[q];
  }
  return os;
}

// FP64 partials of sum_e s_e d_e (x) d_e over the fibers a thread owns for
// the stress (a fiber counts at its free end when the other end is on the
// boundary, else at its lower-numbered end), at the state held in H.
// COMP: compensated (Neumaier) sums, lane 0 of each warp writes 6
// (sum, compensation) pairs to red[(warp * 6 + k) * 2 + {0, 1}]; otherwise
// plain FP64 sums written to red[warp * 9 + 3 + k] (the check's layout).
template <typename T, typename V4, int NT, int NPT, bool COMP>
__device__ __noinline__ void node_stress_partials(const V4* PP, const V4* H, const OwnSet<NPT> os, int nf,
                                                  double* red, int g = -1, int ntc = NT) {
  const int tid = threadIdx.x;
  if (g < 0) g = tid;  // the thread's index over the threads that share the RVE
  CSum s6[6];
  T ps[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};  // check partials in the loop type (see add_virial)
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    if (os.own[q] < 0) continue;
    const int a = node_rank(q, g, ntc);  // own H position
    const V4 hs = H[a];
    for (int k = 0; k < os.deg[q]; ++k) {
      const int s = os.off[q] + k;
      const V4 p0 = PP[size_t(2 * s) * NT + tid];
      const V4 p1 = PP[size_t(2 * s + 1) * NT + tid];
      const int far = int(k_unpack_ij(p1.w));
      if (!(far == nf || a < far)) continue;
      T Dx, Dy, Dz, sv, sbar;
      fiber_force<T>(p0, p1, hs, H[far], Dx, Dy, Dz, sv, sbar);
      const double sd = double(sv), dx = double(Dx), dy = double(Dy), dz = double(Dz);
      if (COMP) {
        s6[0].add(sd * dx * dx);
        s6[1].add(sd * dy * dy);
        s6[2].add(sd * dz * dz);
        s6[3].add(sd * dy * dz);
        s6[4].add(sd * dx * dz);
        s6[5].add(sd * dx * dy);
      } else {
        const T ox = sv * Dx, oy = sv * Dy, oz = sv * Dz;
        ps[0] += ox * Dx;
        ps[1] += oy * Dy;
        ps[2] += oz * Dz;
        ps[3] += oy * Dz;
        ps[4] += ox * Dz;
        ps[5] += ox * Dy;
      }
    }
  }
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (COMP) {
      double s = s6[k].s, cc = s6[k].c;
      warp_csum(s, cc);
      if (lane == 0) {
        red[(warp * 6 + k) * 2 + 0] = s;
        red[(warp * 6 + k) * 2 + 1] = cc;
      }
    } else {
      const double v = warp_sum(double(ps[k]));
      if (lane == 0) red[warp * 9 + 3 + k] = v;
    }
  }
}

// Rebase of the node-centric layout: fold each owned node's correction into
// the FP64 state in global memory, zero it in the buffer the next iteration
// reads (Hn) and in the registers, barrier, then recompute the thread's own
// slots from the FP64 state (private to the thread: no barrier after them).
template <typename T, int NT, int NPT, typename V4>
__device__ __forceinline__ void node_rebase(const DrArgs<T>& A, const Work& wk, const RveMeta& M, const double* sF,
                                            const OwnSet<NPT>& os, V4* Hn, V4* PP, bool init, bool warm,
                                            T (&hx)[NPT], T (&hy)[NPT], T (&hz)[NPT]) {
  double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = os.own[q];
    if (a >= 0) {
      double rx = 0.0, ry = 0.0, rz = 0.0;
      if (!init || warm) {
        rx = st[4 * a + 0];
        ry = st[4 * a + 1];
        rz = st[4 * a + 2];
      }
      if (!init) {
        rx += double(hx[q]);
        ry += double(hy[q]);
        rz += double(hz[q]);
      }
      st[4 * a + 0] = rx;
      st[4 * a + 1] = ry;
      st[4 * a + 2] = rz;
      st[4 * a + 3] = 0.0;
      hx[q] = hy[q] = hz[q] = T(0);
      V4 z;
      z.x = z.y = z.z = z.w = T(0);
      Hn[node_rank(q, threadIdx.x, NT)] = z;
    }
  }
  __syncthreads();  // the block's state writes are visible to the block after the barrier
  node_rebase_slots<T, V4, NT, NPT>(A, M, os, sF, st, PP);
}

template <typename T, int NT, int NPT>
__global__ void __launch_bounds__(NT, min_blocks<NT>()) dr_node_kernel(const DrArgs<T> A) {
  using V4 = typename Vec4<T>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sF[9], sE[9];
  __shared__ double sRes[8], sBB[12];
  __shared__ double sThr[2], sSig[SIG_WINDOW + 1][8];
  __shared__ int sFlag;
  __shared__ T sAB[2];
  __shared__ double sC;

  // a launch that follows this one as a programmatic dependent (the rest of a
  // bin whose costliest RVEs run here, one per SM) may start once every CTA
  // of this launch is resident; it reads nothing written here
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const Work wk = A.work[blockIdx.x];
  const RveMeta M = A.meta[wk.rve];
  const int tid = threadIdx.x;
  const int nf = M.nf, na = M.na, nb = M.nb;

  // ---- shared-memory carve-up (layout mirrored by smem_node)
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = smem + off;
    off += align_up(bytes, 16);
    return p;
  };
  V4* H0 = reinterpret_cast<V4*>(carve(size_t(nf + 1) * sizeof(V4)));
  V4* H1 = reinterpret_cast<V4*>(carve(size_t(nf + 1) * sizeof(V4)));
  double* red = reinterpret_cast<double*>(carve(size_t(NT / 32) * 12 * sizeof(double) + 256));
  V4* PP = reinterpret_cast<V4*>(smem + off);

  if (tid < 9) sF[tid] = A.F[9 * size_t(wk.out) + tid];
  __syncthreads();
  if (tid < 9) {
    const int k = tid / 3, l = tid % 3;
    sE[tid] = 0.5 * (sF[k] * sF[l] + sF[3 + k] * sF[3 + l] + sF[6 + k] * sF[6 + l] - (k == l ? 1.0 : 0.0));
  }
  __syncthreads();
  const double detF = sF[0] * (sF[4] * sF[8] - sF[5] * sF[7]) - sF[1] * (sF[3] * sF[8] - sF[5] * sF[6]) +
                      sF[2] * (sF[3] * sF[7] - sF[4] * sF[6]);
  const bool badF = !(detF > 0.0) || !(detF < 1e300);

  // ---- set-up: affine force scale (FP64) over the active fibers
  double raff2 = 0.0;
  for (int e = tid; e < na; e += NT) {
    const FibD q = A.fa[M.fa_off + e];
    const double ex = sE[0] * q.dx + sE[1] * q.dy + sE[2] * q.dz;
    const double ey = sE[3] * q.dx + sE[4] * q.dy + sE[5] * q.dz;
    const double ez = sE[6] * q.dx + sE[7] * q.dy + sE[8] * q.dz;
    const double L02 = q.L0 * q.L0;
    const double a = (q.dx * ex + q.dy * ey + q.dz * ez + 0.5 * (q.dx * q.dx + q.dy * q.dy + q.dz * q.dz - L02)) / L02;
    const T Na = law_t<T>(a, q.EA, q.B);
    raff2 += double(Na * Na);
  }
  raff2 += boundary_stress_partials(A.fb + M.fb_off, nb, tid, NT, sF, sE, red);
  // H positions are ranks in the decreasing-degree order (the owners of
  // consecutive ranks are consecutive threads: conflict-free H stores); the
  // inverse order is built in H1, which holds nothing before the first update
  uint16_t* rank_of = reinterpret_cast<uint16_t*>(H1);
  for (int k = tid; k < nf; k += NT) rank_of[A.nord[M.node_off + k]] = uint16_t(k);
  if (tid == 0) rank_of[nf] = uint16_t(nf);
  __syncthreads();
  const OwnSet<NPT> os = node_setup_slots<T, V4, NT, NPT>(A, M, rank_of, PP);
  __syncthreads();  // rank_of read by every thread before H1 is written
  if (tid == 0) {
    V4 z;
    z.x = z.y = z.z = z.w = T(0);
    H0[nf] = z;
    H1[nf] = z;
  }
  ResumeRec rr{};
  if (A.resume) rr = A.resume[wk.rve];
  const bool resumed = A.resume != nullptr && rr.active != 0;
  const bool warm = resumed || wk.kind == 1 || (A.warm_start && A.valid[wk.rve]);
  T hx[NPT], hy[NPT], hz[NPT], vx[NPT], vy[NPT], vz[NPT];
  float cap[NPT];
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = os.own[q];
    hx[q] = hy[q] = hz[q] = T(0);
    vx[q] = vy[q] = vz[q] = T(0);
    cap[q] = 0.f;
    if (a >= 0) {
      cap[q] = A.ncap[M.node_off + a];
      if (resumed) {
        const T* vv = A.vel + 4 * size_t(wk.state_off + a);
        vx[q] = vv[0];
        vy[q] = vv[1];
        vz[q] = vv[2];
      }
    }
  }
  {
    __syncthreads();
    if (tid < 6) {
      double s = 0.0, cc = 0.0;
      for (int w = 0; w < NT / 32; ++w) {
        double t, e;
        two_sum(s, red[(w * 6 + tid) * 2 + 0], t, e);
        s = t;
        cc += e + red[(w * 6 + tid) * 2 + 1];
      }
      sBB[2 * tid] = s;
      sBB[2 * tid + 1] = cc;
    }
    __syncthreads();
  }
  {
    double v1[1] = {raff2};
    block_allreduce<NT, 1>(v1, red);
    raff2 = v1[0];
  }
  const double thr = fmax(A.tol * sqrt(raff2), ABS_FLOOR * M.sum_EA);
  const double thr2 = thr * thr;
  __syncthreads();  // red read by every thread before it is reused
  // initial reference state (H0 is read first; H1 is zeroed at the first update)
  node_rebase<T, NT, NPT>(A, wk, M, sF, os, H0, PP, true, warm, hx, hy, hz);

  // ---- dynamic relaxation loop
  const int K = A.check_every;
  const bool adaptive = !(A.damping > 0.0);
  double c = adaptive ? DAMP_C0 : A.damping;
  if (resumed) c = rr.c;
  T alpha = T((2.0 - c) / (2.0 + c)), beta = T(2.0 / (2.0 + c));
  int it = resumed ? rr.it : 0, n_checks = resumed ? rr.n_checks : 0;
  const int it0 = it;
  const bool sig_test = A.sigma_tol > 0.0;
  if (tid == 0) {
    sAB[0] = alpha;
    sAB[1] = beta;
    sC = c;
    const double thr_tight = fmax(1e-3 * A.sigma_tol * sqrt(raff2), ABS_FLOOR * M.sum_EA);
    sThr[0] = thr2;
    sThr[1] = thr_tight * thr_tight;
    for (int k = 0; k <= SIG_WINDOW; ++k) sSig[k][7] = 0.0;
  }
  __syncthreads();
  double pre = 0.0, pm = 0.0;
  bool have_pre = false;
  int cur = 0;  // H buffer read by this iteration
  int status = RVE_STATUS_EMPTY;
  if (nf > 0 && !badF) {
    status = RVE_STATUS_MAX_ITER;
    int to_check = 0;
    for (;; ++it) {
      const bool check = (to_check == 0) || (it >= A.max_iter);
      to_check = (to_check == 0) ? K - 1 : to_check - 1;
      const V4* Hc = cur ? H1 : H0;
      V4* Hn = cur ? H0 : H1;
      // forces on the owned nodes from their incidence slots, two slots in flight
      T fx[NPT], fy[NPT], fz[NPT], fw[NPT];
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        T ax = T(0), ay = T(0), az = T(0), aw = T(0);
        V4 hs;
        hs.x = hx[q];
        hs.y = hy[q];
        hs.z = hz[q];
        hs.w = T(0);
        const V4* pp = PP + size_t(2 * os.off[q]) * NT + tid;
        const int dq = os.deg[q];
        int k = 0;
        for (; k + 1 < dq; k += 2) {
          const V4 p0a = pp[0], p1a = pp[NT], p0b = pp[2 * NT], p1b = pp[3 * NT];
          const V4 ha = Hc[k_unpack_ij(p1a.w)], hb = Hc[k_unpack_ij(p1b.w)];
          T Dx, Dy, Dz, s, sbar;
          fiber_force<T>(p0a, p1a, hs, ha, Dx, Dy, Dz, s, sbar);
          ax += s * Dx;
          ay += s * Dy;
          az += s * Dz;
          aw += sbar;
          fiber_force<T>(p0b, p1b, hs, hb, Dx, Dy, Dz, s, sbar);
          ax += s * Dx;
          ay += s * Dy;
          az += s * Dz;
          aw += sbar;
          pp += 4 * NT;
        }
        if (k < dq) {
          const V4 p0a = pp[0], p1a = pp[NT];
          const V4 ha = Hc[k_unpack_ij(p1a.w)];
          T Dx, Dy, Dz, s, sbar;
          fiber_force<T>(p0a, p1a, hs, ha, Dx, Dy, Dz, s, sbar);
          ax += s * Dx;
          ay += s * Dy;
          az += s * Dz;
          aw += sbar;
        }
        fx[q] = ax;
        fy[q] = ay;
        fz[q] = az;
        fw[q] = aw;
      }
      bool do_rebase = false;
      if (check) {
        // ||f||^2, v.(f_new - f_old) and v.M v: node terms in T, sums in FP64
        double t3[3] = {0.0, 0.0, pm};
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          if (os.own[q] >= 0) {
            t3[0] += double(fx[q] * fx[q] + fy[q] * fy[q] + fz[q] * fz[q]);
            t3[1] += double(vx[q] * fx[q] + vy[q] * fy[q] + vz[q] * fz[q]);
          }
        }
        t3[1] -= pre;
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int k = 0; k < 3; ++k) t3[k] = warp_sum(t3[k]);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) red[warp * 9 + k] = t3[k];
        }
        if (sig_test) node_stress_partials<T, V4, NT, NPT, false>(PP, Hc, os, nf, red);
        __syncthreads();
        if (warp == 0)
          check_decide<T, NT / 32>(red, sig_test, n_checks, it, it0, have_pre, adaptive, A.max_iter, A.damping_scale,
                                   A.sigma_tol, A.resume ? A.wave_iters : 0, sThr, sSig, sBB, sAB, &sC, &sFlag);
        __syncthreads();
        const int flag = sFlag;
        if (flag == RVE_STATUS_NONFINITE || flag == RVE_STATUS_CONVERGED || flag == RVE_STATUS_PARKED_INTERNAL) {
          status = flag;
          break;
        }
        if (flag == RVE_STATUS_MAX_ITER) break;
        alpha = sAB[0];
        beta = sAB[1];
        pre = 0.0;
        pm = 0.0;
        have_pre = false;
        ++n_checks;
        do_rebase = std::is_same<T, float>::value && (n_checks % REBASE_EVERY == 0);
      }
      const bool pre_it = adaptive && (to_check == 0);
      // update owned nodes, publish their corrections in the other buffer
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        const int a = os.own[q];
        if (a >= 0) {
          const T m = T(MASS_COEF) * fw[q];
          const T bm = k_div(beta, m);
          T nvx = alpha * vx[q] + bm * fx[q];
          T nvy = alpha * vy[q] + bm * fy[q];
          T nvz = alpha * vz[q] + bm * fz[q];
          const T sp2 = nvx * nvx + nvy * nvy + nvz * nvz;
          const T cp = T(cap[q]);
          if (sp2 > cp * cp) {
            const T sc = cp * k_rsqrt(sp2);
            nvx *= sc;
            nvy *= sc;
            nvz *= sc;
          }
          hx[q] += nvx;
          hy[q] += nvy;
          hz[q] += nvz;
          vx[q] = nvx;
          vy[q] = nvy;
          vz[q] = nvz;
          V4 h4;
          h4.x = hx[q];
          h4.y = hy[q];
          h4.z = hz[q];
          h4.w = T(0);
          Hn[node_rank(q, tid, NT)] = h4;
          if (pre_it) {
            pre += double(nvx * fx[q] + nvy * fy[q] + nvz * fz[q]);
            pm += double(m * (nvx * nvx + nvy * nvy + nvz * nvz));
          }
        }
      }
      if (pre_it) have_pre = true;
      if (do_rebase) {
        node_rebase<T, NT, NPT>(A, wk, M, sF, os, Hn, PP, false, true, hx, hy, hz);
      } else {
        __syncthreads();
      }
      cur ^= 1;
    }
  }
  const V4* Hf = cur ? H1 : H0;  // the state the loop stopped at

  if (status == RVE_STATUS_PARKED_INTERNAL) {
    double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int a = os.own[q];
      if (a >= 0) {
        st[4 * a + 0] += double(hx[q]);
        st[4 * a + 1] += double(hy[q]);
        st[4 * a + 2] += double(hz[q]);
        T* vv = A.vel + 4 * size_t(wk.state_off + a);
        vv[0] = vx[q];
        vv[1] = vy[q];
        vv[2] = vz[q];
        vv[3] = T(0);
      }
    }
    if (tid == 0) {
      ResumeRec r;
      r.it = it;
      r.n_checks = n_checks;
      r.c = sC;
      r.ke_prev = 0.f;
      r.kin_half = 0;
      r.active = 1;
      r.pad = 0;
      A.resume[wk.rve] = r;
      if (A.iters) A.iters[wk.out] = it;
      if (A.status) A.status[wk.out] = status;
    }
    pdl_epilogue(A);
    return;
  }

  // ---- stress at the final state
  __syncthreads();
  node_stress_partials<T, V4, NT, NPT, true>(PP, Hf, os, nf, red);
  __syncthreads();
  if (tid < 6) {
    double s = sBB[2 * tid], cc = sBB[2 * tid + 1];
    for (int w = 0; w < NT / 32; ++w) {
      double t, e;
      two_sum(s, red[(w * 6 + tid) * 2 + 0], t, e);
      s = t;
      cc += e + red[(w * 6 + tid) * 2 + 1];
    }
    sRes[tid] = s + cc;
  }
  {
    double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int a = os.own[q];
      if (a >= 0) {
        st[4 * a + 0] += double(hx[q]);
        st[4 * a + 1] += double(hy[q]);
        st[4 * a + 2] += double(hz[q]);
      }
    }
  }
  __syncthreads();
  if (tid < 9) {
    const int i = tid / 3, j = tid % 3;
    const int idx = (i == j) ? i : 6 - i - j;
    A.sigma[9 * size_t(wk.out) + tid] = badF ? __longlong_as_double(0x7ff8000000000000ll)
                                              : sRes[idx] / (detF * M.V0);
  }
  if (tid == 0) {
    int st = status;
    if (badF) st = RVE_STATUS_NONFINITE;
    if (wk.kind == 0) {
      A.valid[wk.rve] = (st == RVE_STATUS_NONFINITE) ? 0 : 1;
      A.last_iters[wk.rve] = it;
    }
    if (A.resume) A.resume[wk.rve].active = 0;
    if (A.iters) A.iters[wk.out] = it;
    if (A.status) A.status[wk.out] = st;
  }
  pdl_epilogue(A);
}

}  // namespace rvegpu
