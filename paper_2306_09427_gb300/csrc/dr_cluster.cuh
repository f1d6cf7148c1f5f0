// Node-centric DR kernel split over a thread-block cluster: CL CTAs (one
// cluster) solve one RVE that is too large for one CTA's shared memory, with
// the whole state in the cluster's distributed shared memory.
//
// The arithmetic per DR iteration is that of dr_node_kernel (Algorithm 2,
// Sec. 3.2; FP32 loop on the FP64 reference state with rebases): every
// thread owns NPT free nodes and evaluates their incident fibers itself.
// The free nodes, in decreasing-degree order, are dealt to the CL * NT
// threads of the cluster in snake order (node_rank over the cluster), so
// each CTA owns a share of the network:
//   H0, H1  (every CTA) a full replica of the corrections of all free nodes
//           at their ranks, and the zero slot nf of boundary ends; an owner
//           writes its node's new correction into every CTA's replica of the
//           next buffer (remote stores through distributed shared memory,
//           which the thread does not wait for), so every slot read is a
//           local shared-memory load;
//   PP      (per CTA) the incidence slots of the CTA's threads, laid out as
//           in dr_node_kernel;
//   gat     (CTA 0) per-CTA partials of the checks and of the stress.
// One cluster barrier per iteration (release/acquire: every CTA's stores
// into every replica of the next buffer land before any read of it).  The
// checks: each CTA reduces its warps, writes its partials to CTA 0, cluster
// barrier, CTA 0 takes the decisions (check_decide over the CTA partials in
// rank order: deterministic), writes them to every CTA, cluster barrier.
// Every CTA follows the same control flow (the decisions are the
// cluster's), so every CTA reaches every cluster barrier; before it exits,
// each CTA waits at a last cluster barrier, after which no CTA touches
// another's shared memory.
// Boundary-fiber stress, R_aff and the thresholds are computed by every CTA
// (the same sums in the same order, so the same values); only CTA 0 uses
// the stress terms.
#pragma once

#include <cooperative_groups.h>

#include "dr_node.cuh"

namespace rvegpu {

// Store v at position k of the buffer `buf` in every CTA of the cluster.
template <typename V4>
__device__ __forceinline__ void store_replicas(V4* buf, int k, const V4& v, int CL) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  for (int r = 0; r < CL; ++r) cl.map_shared_rank(buf, r)[k] = v;
}

template <typename T, int NT, int NPT>
__global__ void __launch_bounds__(NT, 1) dr_cluster_kernel(const DrArgs<T> A) {
  namespace cg = cooperative_groups;
  using V4 = typename Vec4<T>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sF[9], sE[9];
  __shared__ double sRes[8], sBB[12];
  __shared__ double sThr[2], sSig[SIG_WINDOW + 1][8];
  __shared__ int sFlag;
  __shared__ T sAB[2];
  __shared__ double sC;

  cg::cluster_group cl = cg::this_cluster();
  const int CL = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const Work wk = A.work[blockIdx.x / CL];
  const RveMeta M = A.meta[wk.rve];
  const int tid = threadIdx.x;
  const int nf = M.nf, na = M.na, nb = M.nb;
  const int ntc = CL * NT;       // threads sharing the RVE
  const int g = rank * NT + tid;  // this thread among them

  // ---- shared-memory carve-up (layout mirrored by smem_cluster)
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = smem + off;
    off += align_up(bytes, 16);
    return p;
  };
  V4* H0 = reinterpret_cast<V4*>(carve(size_t(nf + 1) * sizeof(V4)));
  V4* H1 = reinterpret_cast<V4*>(carve(size_t(nf + 1) * sizeof(V4)));
  double* red = reinterpret_cast<double*>(carve(size_t(NT / 32) * 12 * sizeof(double) + 256));
  double* gat = reinterpret_cast<double*>(carve(size_t(CLUSTER_MAX) * 12 * sizeof(double)));
  V4* PP = reinterpret_cast<V4*>(smem + off);
  double* gat0 = cl.map_shared_rank(gat, 0);  // CTA 0's gather rows

  if (tid < 9) sF[tid] = A.F[9 * size_t(wk.out) + tid];
  __syncthreads();
  if (tid < 9) {
    const int k = tid / 3, l = tid % 3;
    sE[tid] = 0.5 * (sF[k] * sF[l] + sF[3 + k] * sF[3 + l] + sF[6 + k] * sF[6 + l] - (k == l ? 1.0 : 0.0));
  }
  for (int k = tid; k < CLUSTER_MAX * 12; k += NT) gat[k] = 0.0;  // rows of absent ranks stay zero
  __syncthreads();
  const double detF = sF[0] * (sF[4] * sF[8] - sF[5] * sF[7]) - sF[1] * (sF[3] * sF[8] - sF[5] * sF[6]) +
                      sF[2] * (sF[3] * sF[7] - sF[4] * sF[6]);
  const bool badF = !(detF > 0.0) || !(detF < 1e300);

  // ---- set-up (every CTA: the same sums, so the same thresholds)
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
  uint16_t* rank_of = reinterpret_cast<uint16_t*>(H1);  // holds nothing before the first update
  for (int k = tid; k < nf; k += NT) rank_of[A.nord[M.node_off + k]] = uint16_t(k);
  __syncthreads();
  const OwnSet<NPT> os = node_setup_slots<T, V4, NT, NPT>(A, M, rank_of, PP, g, ntc);
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
  __syncthreads();  // rank_of and red read before they are reused
  {
    double v1[1] = {raff2};
    block_allreduce<NT, 1>(v1, red);
    raff2 = v1[0];
  }
  const double thr = fmax(A.tol * sqrt(raff2), ABS_FLOOR * M.sum_EA);
  const double thr2 = thr * thr;
  {
    V4 z;
    z.x = z.y = z.z = z.w = T(0);
    for (int k = tid; k <= nf; k += NT) {
      H0[k] = z;  // every correction starts at zero after the first rebase
      H1[k] = z;
    }
  }
  ResumeRec rr{};
  if (A.resume) rr = A.resume[wk.rve];
  const bool resumed = A.resume != nullptr && rr.active != 0;
  const bool warm = resumed || wk.kind == 1 || (A.warm_start && A.valid[wk.rve]);
  T hx[NPT], hy[NPT], hz[NPT], vx[NPT], vy[NPT], vz[NPT];
  float cap[NPT];
  double* st = A.state + 4 * size_t(wk.state_off);
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
      // initial reference state: the warm state, or h = 0
      double rx = 0.0, ry = 0.0, rz = 0.0;
      if (warm) {
        rx = st[4 * a + 0];
        ry = st[4 * a + 1];
        rz = st[4 * a + 2];
      }
      st[4 * a + 0] = rx;
      st[4 * a + 1] = ry;
      st[4 * a + 2] = rz;
      st[4 * a + 3] = 0.0;
    }
  }
  // every CTA's state writes (and zeroed replicas) before any slot reads them
  __threadfence();
  cl.sync();
  node_rebase_slots<T, V4, NT, NPT>(A, M, os, sF, st, PP);

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
  int cur = 0;
  int status = RVE_STATUS_EMPTY;
  if (nf > 0 && !badF) {
    status = RVE_STATUS_MAX_ITER;
    int to_check = 0;
    for (;; ++it) {
      const bool check = (to_check == 0) || (it >= A.max_iter);
      to_check = (to_check == 0) ? K - 1 : to_check - 1;
      const V4* Hc = cur ? H1 : H0;
      V4* Hn = cur ? H0 : H1;
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
        if (sig_test) node_stress_partials<T, V4, NT, NPT, false>(PP, Hc, os, nf, red, g, ntc);
        __syncthreads();
        // this CTA's totals (warps in order) to CTA 0's row `rank`
        if (tid < 9) {
          double v = 0.0;
          if (tid < 3 || sig_test)
            for (int w = 0; w < NT / 32; ++w) v += red[w * 9 + tid];
          gat0[rank * 9 + tid] = v;
        }
        cl.sync();
        if (rank == 0 && warp == 0)
          check_decide<T, CLUSTER_MAX>(gat, sig_test, n_checks, it, it0, have_pre, adaptive, A.max_iter,
                                       A.damping_scale, A.sigma_tol, A.resume ? A.wave_iters : 0, sThr, sSig, sBB, sAB,
                                       &sC, &sFlag);
        if (rank == 0 && tid == 0) {
          // publish the decisions in every other CTA (this thread wrote them)
          for (int r = 1; r < CL; ++r) {
            *cl.map_shared_rank(&sFlag, r) = sFlag;
            *cl.map_shared_rank(&sC, r) = sC;
            T* ab = cl.map_shared_rank(sAB, r);
            ab[0] = sAB[0];
            ab[1] = sAB[1];
          }
        }
        cl.sync();
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
          if (do_rebase) {
            // fold the correction into the FP64 state; the new one is zero
            st[4 * a + 0] += double(hx[q]);
            st[4 * a + 1] += double(hy[q]);
            st[4 * a + 2] += double(hz[q]);
            hx[q] = hy[q] = hz[q] = T(0);
          }
          V4 h4;
          h4.x = hx[q];
          h4.y = hy[q];
          h4.z = hz[q];
          h4.w = T(0);
          store_replicas(Hn, node_rank(q, g, ntc), h4, CL);
          if (pre_it) {
            pre += double(nvx * fx[q] + nvy * fy[q] + nvz * fz[q]);
            pm += double(m * (nvx * nvx + nvy * nvy + nvz * nvz));
          }
        }
      }
      if (pre_it) have_pre = true;
      if (do_rebase) {
        // the slots read other nodes' FP64 state: cluster-wide barrier first
        __threadfence();
        cl.sync();
        node_rebase_slots<T, V4, NT, NPT>(A, M, os, sF, st, PP);
      } else {
        cl.sync();
      }
      cur ^= 1;
    }
  }
  const V4* Hf = cur ? H1 : H0;

  if (status == RVE_STATUS_PARKED_INTERNAL) {
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
    if (rank == 0 && tid == 0) {
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
    cl.sync();  // no CTA leaves while another may still touch its shared memory
    return;
  }

  // ---- stress at the final state: CTA partials to CTA 0, combined in rank order
  __syncthreads();
  node_stress_partials<T, V4, NT, NPT, true>(PP, Hf, os, nf, red, g, ntc);
  __syncthreads();
  if (tid < 6) {
    double s = 0.0, cc = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      double t, e;
      two_sum(s, red[(w * 6 + tid) * 2 + 0], t, e);
      s = t;
      cc += e + red[(w * 6 + tid) * 2 + 1];
    }
    gat0[rank * 12 + 2 * tid] = s;
    gat0[rank * 12 + 2 * tid + 1] = cc;
  }
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = os.own[q];
    if (a >= 0) {
      st[4 * a + 0] += double(hx[q]);
      st[4 * a + 1] += double(hy[q]);
      st[4 * a + 2] += double(hz[q]);
    }
  }
  cl.sync();
  if (rank == 0) {
    if (tid < 6) {
      double s = sBB[2 * tid], cc = sBB[2 * tid + 1];
      for (int r = 0; r < CL; ++r) {
        double t, e;
        two_sum(s, gat[r * 12 + 2 * tid], t, e);
        s = t;
        cc += e + gat[r * 12 + 2 * tid + 1];
      }
      sRes[tid] = s + cc;
    }
    __syncthreads();
    if (tid < 9) {
      const int i = tid / 3, j = tid % 3;
      const int idx = (i == j) ? i : 6 - i - j;
      A.sigma[9 * size_t(wk.out) + tid] = badF ? __longlong_as_double(0x7ff8000000000000ll)
                                                : sRes[idx] / (detF * M.V0);
    }
    if (tid == 0) {
      int stt = status;
      if (badF) stt = RVE_STATUS_NONFINITE;
      if (wk.kind == 0) {
        A.valid[wk.rve] = (stt == RVE_STATUS_NONFINITE) ? 0 : 1;
        A.last_iters[wk.rve] = it;
      }
      if (A.resume) A.resume[wk.rve].active = 0;
      if (A.iters) A.iters[wk.out] = it;
      if (A.status) A.status[wk.out] = stt;
    }
  }
  cl.sync();  // no CTA leaves while another may still touch its shared memory
}

}  // namespace rvegpu
