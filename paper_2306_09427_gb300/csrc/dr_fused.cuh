// Fused batched dynamic-relaxation kernel: one CTA solves one RVE.
//
// Per work item (RVE r, deformation gradient F):
//   set-up   per active fiber e = (i, j): the affine chord g_e = F dX_e and
//            the affine Green strain a_e = (dX.E.dX + (|dX|^2 - L0^2)/2)/L0^2,
//            E = (F^T F - I)/2, both in FP64; boundary-to-boundary fibers
//            have a fixed length, so their stress share and the affine force
//            norm R_aff are summed here once, in FP64.
//   loop     (Algorithm 2, Sec. 3.2)
//     fiber  with the fluctuation difference u = h_j - h_i (boundary ends
//            read the zero slot, h = 0 under the affine BC, Eq. affine-bc):
//              eps = a_e + u.(2 g_e + u) / (2 L0^2)      (no cancellation)
//              d = g_e + u,  l = |d|,  N = (EA/B) expm1(B eps)
//              s = N / l,  sbar = max(dN/dl, |N|/l)
//            and stores (s d, sbar) in the fiber scratch SCR;
//     gather each free node sums +-(s d) and sbar of its incident fibers in
//            a fixed CSR order, four entries per 8-byte load (runs padded
//            with a zero slot); deterministic, no atomics (the paper's
//            getInternalForces scatters with atomics, Sec. 4.3);
//     check  every check_every iterations: ||f_free||_2 (per-node terms in T,
//            per-thread, per-warp and cross-warp sums in FP64)
//            against max(tol R_aff, 1e-16 sum EA) and, with sigma_tol > 0,
//            the estimated remaining stress error; damping re-estimated,
//            c = s 2 sqrt(lambda) from the Rayleigh quotient lambda (the
//            stress-error estimate and c in T, from the FP64 sums); thread 0
//            takes these block-uniform decisions and publishes them;
//     update m = MASS_COEF sbar_sum, v <- ((2-c) v + 2 f/m)/(2+c),
//            |v| capped, h <- h + v (dt = 1); with VAR_KINETIC (kinetic damping)
//            c = 0 and a step past a kinetic-energy peak is taken back and
//            the motion restarts from rest.
//   finish   sigma = (sigma_bb + sum_e s_e d_e (x) d_e) / (det F V0) with
//            FP64 compensated (TwoSum) accumulation; h saved for warm starts.
//
// Threads own fixed free nodes (a = tid + q*NT, q < NPT) whose h, v, cap
// and CSR range live in registers; the shared array H publishes h to the
// fiber phase.  MODE 0 keeps all per-fiber data of the RVE in shared
// memory; MODE 1 reads fiber parameters and CSR from global memory (L2)
// and keeps H and SCR in shared memory; MODE 2 also moves SCR to global.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "rve_internal.h"

namespace rvegpu {

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using t = float4;
};
struct __align__(16) dvec4 {
  double x, y, z, w;
};
template <>
struct Vec4<double> {
  using t = dvec4;
};

// Minimum resident CTAs per SM requested from the register allocator:
// two 256-thread CTAs per SM (up to 128 registers per thread, no spills in
// the loop); measured faster than three CTAs at 80 registers with spills.
#ifndef RVE_MIN_BLOCKS_256
#define RVE_MIN_BLOCKS_256 2
#endif
#ifndef RVE_FIBER_UNROLL
#define RVE_FIBER_UNROLL 2
#endif
template <int NT>
constexpr int min_blocks() {
  return NT >= 1024 ? 1 : (NT >= 512 ? 1 : (RVE_MIN_BLOCKS_256 * 256 / NT));
}

// expm1 in FP32 for the hot loop: for |x| <= 1/2 the Taylor series of
// e^x - 1 through x^8 (Horner; truncation below x^9/9! < 6e-9 |x|, under the
// FP32 rounding of the result); otherwise e^x - 1 with the hardware
// exponential (__expf), where e^x - 1 is at least 0.39 |e^x| in magnitude so
// no cancellation amplifies its error.  Both are evaluated and one selected.
__device__ __forceinline__ float k_expm1(float x) {
  const float p =
      x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f +
           x * (1.0f / 720.0f + x * (1.0f / 5040.0f + x * (1.0f / 40320.0f))))))));
  const float q = __expf(x) - 1.0f;
  return fabsf(x) <= 0.5f ? p : q;
}
__device__ __forceinline__ double k_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float k_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float k_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double k_max(double a, double b) { return ::fmax(a, b); }
__device__ __forceinline__ float k_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double k_abs(double a) { return ::fabs(a); }
__device__ __forceinline__ double k_div(double a, double b) { return a / b; }
__device__ __forceinline__ float k_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double k_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ uint32_t k_unpack_ij(float w) { return __float_as_uint(w); }
__device__ __forceinline__ uint32_t k_unpack_ij(double w) { return static_cast<uint32_t>(w); }
__device__ __forceinline__ float k_pack_ij(uint32_t ij, float) { return __uint_as_float(ij); }
__device__ __forceinline__ double k_pack_ij(uint32_t ij, double) { return static_cast<double>(ij); }

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Neumaier accumulator
struct CSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    double t, e;
    two_sum(s, x, t, e);
    s = t;
    c += e;
  }
};

__device__ __forceinline__ float warp_sum_t(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_t(double v) { return warp_sum(v); }

__device__ __forceinline__ void warp_csum(double& s, double& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
    double t, e;
    two_sum(s, s2, t, e);
    s = t;
    c = c + c2 + e;
  }
}

// Sum K doubles over the block; every thread gets the totals.  One
// barrier; the caller separates successive uses of `red` by a barrier.
template <int NT, int K>
__device__ __forceinline__ void block_allreduce(double (&v)[K], double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
#pragma unroll 4
    for (int w = 0; w < NT / 32; ++w) s += red[w * K + k];
    v[k] = s;
  }
}

// Fiber force from the fluctuation formulation (see header comment).
template <typename T, typename V4>
__device__ __forceinline__ void fiber_force(const V4& p0, const V4& p1, const V4& hi, const V4& hj,
                                            T& Dx, T& Dy, T& Dz, T& s, T& sbar) {
  const T ux = hj.x - hi.x, uy = hj.y - hi.y, uz = hj.z - hi.z;
  const T t = ux * (T(2) * p0.x + ux) + uy * (T(2) * p0.y + uy) + uz * (T(2) * p0.z + uz);
  const T eps = t * p1.x + p0.w;
  Dx = p0.x + ux;
  Dy = p0.y + uy;
  Dz = p0.z + uz;
  const T l2 = Dx * Dx + Dy * Dy + Dz * Dz;
  const T rl = k_rsqrt(l2);
  const T l = l2 * rl;
  T phi, ex, ea;
  if (p1.z > T(0)) {
    phi = k_expm1(p1.z * eps);
    ex = phi + T(1);
    ea = p1.y * p1.z;
  } else {
    phi = eps;
    ex = T(1);
    ea = p1.y;
  }
  const T N = p1.y * phi;
  s = N * rl;
  const T kax = ea * ex * l * (T(2) * p1.x);
  sbar = k_max(kax, k_abs(s));
}

// Fiber law in FP64 for set-up terms: N(eps) with the B = 0 limit.
__device__ __forceinline__ double law_f64(double eps, double EA, double B) {
  return B > 0.0 ? (EA / B) * expm1(B * eps) : EA * eps;
}

// Stored energy of one fiber, w(l) = integral of N from L0 to l, by 8-point
// Gauss-Legendre quadrature on [L0, l] (nodes and weights of Abramowitz and
// Stegun, Table 25.4); N is smooth (the exponential of a quadratic in l), so
// the rule is exact to the loop type's rounding over the strains of a
// solve.  inv2L02 = 1/(2 L0^2), eab = EA/B (EA when B = 0).
template <typename T>
__device__ __forceinline__ T fiber_energy_gl8(T l, T inv2L02, T eab, T B) {
  const T t[4] = {T(0.1834346424956498), T(0.5255324099163290), T(0.7966664774136267), T(0.9602898564975363)};
  const T w[4] = {T(0.3626837833783620), T(0.3137066458778873), T(0.2223810344533745), T(0.1012285362903763)};
  const T L0 = sqrt(T(0.5) / inv2L02);
  const T mid = T(0.5) * (l + L0), half = T(0.5) * (l - L0);
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const T lk = mid + T(sgn) * half * t[k];
      const T eps = (lk * lk) * inv2L02 - T(0.5);
      const T N = B > T(0) ? eab * k_expm1(B * eps) : eab * eps;
      acc += w[k] * N;
    }
  }
  return half * acc;
}

// Accumulate a fiber's stress terms s d (x) d (o = s d) into the thread's
// partials (xx yy zz yz xz xy) in the loop type, for the stress-convergence
// test at checks; the sums over threads are FP64.  A thread holds a few
// fibers, so the FP32 rounding of its partial (~1e-7 of it) sits far below
// the relative stress change the test resolves (sigma_tol ~1e-5).
template <typename T, typename V4>
__device__ __forceinline__ void add_virial(T (&ps)[6], const V4& o, T Dx, T Dy, T Dz) {
  ps[0] += o.x * Dx;
  ps[1] += o.y * Dy;
  ps[2] += o.z * Dz;
  ps[3] += o.y * Dz;
  ps[4] += o.x * Dz;
  ps[5] += o.x * Dy;
}

// Fiber law in the loop type, N(eps) with the B = 0 limit: the affine force
// scale R_aff only sets the convergence threshold, so the loop type's
// precision is enough there.
template <typename T>
__device__ __forceinline__ T law_t(double eps, double EA, double B) {
  return B > 0.0 ? T(EA / B) * k_expm1(T(B) * T(eps)) : T(EA) * T(eps);
}

// Fiber part of a rebase: FP64 chord g_e = F dX_e + h_ref,j - h_ref,i and
// Green strain of every active fiber at the new reference state.  Out of
// line: it runs once per REBASE_EVERY checks, and its FP64 temporaries then
// do not add to the register pressure of the relaxation loop.
template <typename T, typename V4>
__device__ __noinline__ void rebase_fibers(const FibD* __restrict__ fa, int na, int tid, int nt, const double* sF,
                                           const double* HR, V4* P0, const V4* P1) {
  for (int e = tid; e < na; e += nt) {
    const FibD q = fa[e];
    const uint32_t ij = k_unpack_ij(P1[e].w);
    const uint32_t i = ij & 0xffffu, j = ij >> 16;
    const double gx = sF[0] * q.dx + sF[1] * q.dy + sF[2] * q.dz + (HR[3 * j + 0] - HR[3 * i + 0]);
    const double gy = sF[3] * q.dx + sF[4] * q.dy + sF[5] * q.dz + (HR[3 * j + 1] - HR[3 * i + 1]);
    const double gz = sF[6] * q.dx + sF[7] * q.dy + sF[8] * q.dz + (HR[3 * j + 2] - HR[3 * i + 2]);
    V4 p0;
    p0.x = T(gx);
    p0.y = T(gy);
    p0.z = T(gz);
    p0.w = T((gx * gx + gy * gy + gz * gz - q.L0 * q.L0) * q.half_inv_L02);
    P0[e] = p0;
  }
}

// Block-uniform decisions of a convergence check, taken by warp 0 (lane 0
// decides) from the per-warp FP64 partials in red (9 per warp: ||f||^2,
// v.(f_new - f_old), v.M v, then the 6 stress components when the stress
// test is on).  Publishes the outcome in *flag (-1: keep iterating, or the
// final status) and, with adaptive damping, the new damping c in *c_sh and
// its update factors in ab[0..1].  Out of line: it runs once per check
// interval.
template <typename T, int NW>
__device__ __noinline__ void check_decide(const double* red, bool sig_test, int n_checks, int it, int it0,
                                          bool have_pre, bool adaptive, int max_iter, double damping_scale,
                                          double sigma_tol, int park_after, const double* thr,
                                          double (*sig)[8], const double* bb, T* ab, double* c_sh, int* flag_out) {
  const int lane = threadIdx.x & 31;
  // cross-warp sums, one value per lane (warps in order), then lane 0
  // collects them
  const int nv = sig_test ? 9 : 3;
  double s = 0.0;
  if (lane < nv) {
#pragma unroll 4
    for (int w = 0; w < NW; ++w) s += red[w * 9 + lane];
  }
  double v3[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v3[k] = __shfl_sync(0xffffffffu, s, k);
  if (lane != 0) return;
  // The residual test and the stress differences stay in FP64; the ratios
  // derived from them (the stress-convergence estimate, the damping
  // estimate) are taken in the loop type T.
  using R = T;
  int flag = -1;  // keep iterating; otherwise the final status
  if (!(v3[0] < 1e300)) {  // NaN or Inf
    flag = RVE_STATUS_NONFINITE;
  } else {
    bool sig_ok = true;
    if (sig_test && v3[0] > thr[1]) {
      // remaining stress error of a geometrically converging sequence, from
      // the stress and residual SIG_WINDOW checks back (ring of records)
      const double* prev = sig[(n_checks + 1) % (SIG_WINDOW + 1)];
      double* next = sig[n_checks % (SIG_WINDOW + 1)];
      const R r = sqrt(R(v3[0]));
      double dn = 0.0, nn = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double sg = v3[3 + k] + bb[2 * k] + bb[2 * k + 1];
        const double d = sg - prev[k];
        const double wk2 = k < 3 ? 1.0 : 2.0;  // off-diagonal entries appear twice
        dn += wk2 * d * d;
        nn += wk2 * sg * sg;
        next[k] = sg;
      }
      sig_ok = false;
      const R dnr = R(dn), nnr = R(nn);
      if (prev[7] != 0.0 && nnr > R(0)) {
        const R rho = fmin(r / R(prev[6]), R(SIG_RHO_CAP));
        sig_ok = sqrt(dnr / nnr) * rho / (R(1) - rho) <= R(sigma_tol);
      }
      next[6] = double(r);
      next[7] = 1.0;
    } else if (sig_test) {
      sig[n_checks % (SIG_WINDOW + 1)][7] = 0.0;
    }
    if (v3[0] <= thr[0] && sig_ok) {
      flag = RVE_STATUS_CONVERGED;
    } else if (it >= max_iter) {
      flag = RVE_STATUS_MAX_ITER;
    } else {
      if (adaptive && have_pre && v3[2] > 0.0) {
        const R lam = -R(v3[1]) / R(v3[2]);
        if (lam > R(0)) {
          const R c = fmin(R(damping_scale) * R(2) * sqrt(lam), R(DAMP_C_MAX));
          *c_sh = double(c);
          ab[0] = T((R(2) - c) / (R(2) + c));
          ab[1] = T(R(2) / (R(2) + c));
        }
      }
      // end of a serving wave: park before the update of this iteration
      if (park_after > 0 && it - it0 >= park_after) flag = RVE_STATUS_PARKED_INTERNAL;
    }
  }
  *flag_out = flag;
}

// Compensated (Neumaier) FP64 sums of s d (x) d over this thread's active
// fibers at the current state (P0 at h_ref, H holding the correction),
// reduced over the warp; lane 0 writes the 6 (sum, compensation) pairs of
// its warp to red[(warp * 6 + k) * 2 + {0, 1}].  Out of line: once per solve.
template <typename T, typename V4>
__device__ __noinline__ void fiber_stress_partials(const V4* P0, const V4* P1, const V4* H, int na, int tid, int nt,
                                                   double* red) {
  CSum s6[6];
  for (int e = tid; e < na; e += nt) {
    const V4 p0 = P0[e];
    const V4 p1 = P1[e];
    const uint32_t ij = k_unpack_ij(p1.w);
    const V4 hi = H[ij & 0xffffu];
    const V4 hj = H[ij >> 16];
    T Dx, Dy, Dz, s, sbar;
    fiber_force<T>(p0, p1, hi, hj, Dx, Dy, Dz, s, sbar);
    const double sd = double(s), dx = double(Dx), dy = double(Dy), dz = double(Dz);
    s6[0].add(sd * dx * dx);
    s6[1].add(sd * dy * dy);
    s6[2].add(sd * dz * dz);
    s6[3].add(sd * dy * dz);
    s6[4].add(sd * dx * dz);
    s6[5].add(sd * dx * dy);
  }
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double s = s6[k].s, cc = s6[k].c;
    warp_csum(s, cc);
    if (lane == 0) {
      red[(warp * 6 + k) * 2 + 0] = s;
      red[(warp * 6 + k) * 2 + 1] = cc;
    }
  }
}

// Boundary-to-boundary fibers (fixed length under the affine BC): their
// stress share as compensated per-warp partials in red (layout as
// fiber_stress_partials) and their share of the affine force scale
// sum N^2 (returned, this thread's fibers).  Out of line: once per solve.
static __device__ __noinline__ double boundary_stress_partials(const FibD* __restrict__ fb, int nb, int tid, int nt,
                                                        const double* sF, const double* sE, double* red) {
  CSum sb6[6];
  double raff2 = 0.0;
  for (int e = tid; e < nb; e += nt) {
    const FibD q = fb[e];
    const double gx = sF[0] * q.dx + sF[1] * q.dy + sF[2] * q.dz;
    const double gy = sF[3] * q.dx + sF[4] * q.dy + sF[5] * q.dz;
    const double gz = sF[6] * q.dx + sF[7] * q.dy + sF[8] * q.dz;
    const double ex = sE[0] * q.dx + sE[1] * q.dy + sE[2] * q.dz;
    const double ey = sE[3] * q.dx + sE[4] * q.dy + sE[5] * q.dz;
    const double ez = sE[6] * q.dx + sE[7] * q.dy + sE[8] * q.dz;
    const double L02 = q.L0 * q.L0;
    const double a = (q.dx * ex + q.dy * ey + q.dz * ez + 0.5 * (q.dx * q.dx + q.dy * q.dy + q.dz * q.dz - L02)) / L02;
    const double N = law_f64(a, q.EA, q.B);
    raff2 += N * N;
    const double s = N / sqrt(gx * gx + gy * gy + gz * gz);
    sb6[0].add(s * gx * gx);
    sb6[1].add(s * gy * gy);
    sb6[2].add(s * gz * gz);
    sb6[3].add(s * gy * gz);
    sb6[4].add(s * gx * gz);
    sb6[5].add(s * gx * gy);
  }
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double s = sb6[k].s, cc = sb6[k].c;
    warp_csum(s, cc);
    if (lane == 0) {
      red[(warp * 6 + k) * 2 + 0] = s;
      red[(warp * 6 + k) * 2 + 1] = cc;
    }
  }
  return raff2;
}

// Rebase (mixed-precision iterative refinement of the reference state).
// The FP64 reference fluctuation h_ref of every free node lives in the
// state slot; the FP32 loop works on the correction d = h - h_ref.  A
// rebase folds d into h_ref, then recomputes each active fiber's chord
// g_e = F dX_e + h_ref,j - h_ref,i and Green strain a_e in FP64 and rounds
// them to the loop type.  Near equilibrium the relaxed strain is small, so
// its FP32 rounding is tiny in absolute terms, and the correction u is
// small, so u.(2g + u) keeps full relative precision: the force residual
// no longer floors at the rounding of |h| ~ one grid spacing.
// Node part (owned nodes), then a barrier, then the fiber part, then a
// barrier.  HR is an FP64 scratch copy of h_ref ((nf+1) x 3 doubles).
template <typename T, int NT, int NPT, typename V4>
__device__ __forceinline__ void rebase(const DrArgs<T>& A, const Work& wk, const RveMeta& M, const double* sF,
                                       V4* H, V4* P0, const V4* P1, double* HR, bool init, bool warm,
                                       T (&hx)[NPT], T (&hy)[NPT], T (&hz)[NPT]) {
  const int tid = threadIdx.x;
  const int nf = M.nf, na = M.na;
  double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = tid + q * NT;
    if (a < nf) {
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
      HR[3 * a + 0] = rx;
      HR[3 * a + 1] = ry;
      HR[3 * a + 2] = rz;
      hx[q] = hy[q] = hz[q] = T(0);
      V4 z;
      z.x = z.y = z.z = z.w = T(0);
      H[a] = z;
    }
  }
  if (tid == 0) {
    HR[3 * nf + 0] = HR[3 * nf + 1] = HR[3 * nf + 2] = 0.0;
    V4 z;
    z.x = z.y = z.z = z.w = T(0);
    H[nf] = z;
  }
  __syncthreads();
  rebase_fibers<T, V4>(A.fa + M.fa_off, na, tid, NT, sF, HR, P0, P1);
  __syncthreads();
}

// End of a CTA of a programmatic dependent launch (A.pdl_done set): the last
// CTA to finish waits until the launch it depends on has completed and its
// writes are visible, so that this launch's completion implies that one's
// for whatever follows on the stream.  It then resets the counter for the
// next launch (graph replays included).
template <typename T>
__device__ __forceinline__ void pdl_epilogue(const DrArgs<T>& A) {
  if (A.pdl_done == nullptr) return;
  __shared__ int sLast;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sLast = atomicAdd(A.pdl_done, 1) == A.n_work - 1;
  }
  __syncthreads();
  if (sLast) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) *A.pdl_done = 0;
  }
}

// VAR selects the loop variant, each its own instantiation so that the
// viscous default carries none of the others' code or registers:
// VAR_VISCOUS (adaptive or fixed viscous damping), VAR_KINETIC (kinetic
// damping), VAR_ENERGY (viscous damping with Algorithm 2's optional energy
// balance bookkeeping).
template <typename T, int NT, int NPT, int MODE, int VAR>
__global__ void __launch_bounds__(NT, min_blocks<NT>()) dr_fused_kernel(const DrArgs<T> A) {
  using V4 = typename Vec4<T>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sF[9], sE[9];
  __shared__ double sRes[8], sBB[12];
  // loop-carried block-uniform scalars kept in shared memory, not registers
  // (thresholds; previous stress and residual, double-buffered by check parity)
  __shared__ double sThr[2], sSig[SIG_WINDOW + 1][8];
  // decisions of a check, published by thread 0: outcome and damping factors
  __shared__ int sFlag;
  __shared__ T sAB[2];
  __shared__ double sC;  // damping coefficient in use (thread 0 decides it)
  // kinetic damping: per-warp kinetic-energy partials, double-buffered by iteration parity
  __shared__ T sKE[2][32];
  // energy balance (VAR_ENERGY, thread 0): stored energy at the start, running
  // FP64 totals of the damping and cap dissipation and the mass-change work,
  // the last check's stored-energy change and kinetic energy, and the largest
  // relative balance error seen
  __shared__ double sEn[8];

  // a launch that follows this one as a programmatic dependent (the rest of a
  // bin whose costliest RVEs run here, one per SM) may start once every CTA
  // of this launch is resident; it reads nothing written here
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const Work wk = A.work[blockIdx.x];
  const RveMeta M = A.meta[wk.rve];
  const int tid = threadIdx.x;
  const int nf = M.nf, na = M.na, nb = M.nb;

  // ---- shared-memory carve-up (layout mirrored by smem_resident/smem_streamed)
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = smem + off;
    off += align_up(bytes, 16);
    return p;
  };
  const size_t scr_bytes = scr_region_bytes<T>(nf, na);
  V4* H = reinterpret_cast<V4*>(carve(size_t(nf + 1) * sizeof(V4)));
  V4* P0;
  V4* P1;
  V4* SCR;
  double* HR;
  const uint16_t* CSR;
  if constexpr (MODE == 0) {
    P0 = reinterpret_cast<V4*>(carve(size_t(na) * sizeof(V4)));
    P1 = reinterpret_cast<V4*>(carve(size_t(na) * sizeof(V4)));
    SCR = reinterpret_cast<V4*>(carve(scr_bytes));
    HR = reinterpret_cast<double*>(SCR);
    CSR = reinterpret_cast<const uint16_t*>(carve(size_t(M.csr_len) * sizeof(uint16_t)));
  } else {
    P0 = reinterpret_cast<V4*>(A.gP0) + wk.scr_off;
    P1 = reinterpret_cast<V4*>(A.gP1) + wk.scr_off;
    if constexpr (MODE == 1) {
      SCR = reinterpret_cast<V4*>(carve(scr_bytes));
      HR = reinterpret_cast<double*>(SCR);
    } else {
      SCR = reinterpret_cast<V4*>(A.gSCR) + wk.scr_off;
      HR = reinterpret_cast<double*>(carve(size_t(nf + 1) * 3 * sizeof(double)));
    }
    CSR = A.csr + M.csr_off;
  }
  double* red = reinterpret_cast<double*>(carve(size_t(NT / 32) * 12 * sizeof(double) + 256));

  if (tid < 9) sF[tid] = A.F[9 * size_t(wk.out) + tid];
  __syncthreads();
  if (tid < 9) {
    const int k = tid / 3, l = tid % 3;
    sE[tid] = 0.5 * (sF[k] * sF[l] + sF[3 + k] * sF[3 + l] + sF[6 + k] * sF[6 + l] - (k == l ? 1.0 : 0.0));
  }
  __syncthreads();
  const double detF = sF[0] * (sF[4] * sF[8] - sF[5] * sF[7]) - sF[1] * (sF[3] * sF[8] - sF[5] * sF[6]) +
                      sF[2] * (sF[3] * sF[7] - sF[4] * sF[6]);
  const bool badF = !(detF > 0.0) || !(detF < 1e300);  // inverted, degenerate or non-finite F

  // ---- set-up: static loop parameters and the affine force scale (FP64)
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
    V4 p1;
    p1.x = T(0.5 / L02);
    p1.y = T(q.B > 0.0 ? q.EA / q.B : q.EA);
    p1.z = T(q.B);
    p1.w = k_pack_ij(A.fij[M.fa_off + e], T(0));
    P1[e] = p1;
  }
  // boundary-to-boundary fibers: fixed length, stress share summed once
  // (per-warp compensated partials into red, combined below)
  raff2 += boundary_stress_partials(A.fb + M.fb_off, nb, tid, NT, sF, sE, red);
  if constexpr (MODE == 0) {
    // runs are padded to 4 entries and start 8-byte aligned: copy 4 at a time
    uint2* csr_s = reinterpret_cast<uint2*>(const_cast<uint16_t*>(CSR));
    const uint2* csr_g = reinterpret_cast<const uint2*>(A.csr + M.csr_off);
    for (int k = tid; k < M.csr_len / 4; k += NT) csr_s[k] = csr_g[k];
  }
  const uint32_t zero_run = (uint32_t(na) << 1) | (uint32_t(na) << 17);  // two entries at the zero slot
  if (tid == 0) {  // zero slot that padded CSR entries point at
    V4 z;
    z.x = z.y = z.z = z.w = T(0);
    SCR[na] = z;
  }
  // a solve parked by the previous wave resumes from its record
  ResumeRec rr{};
  if (A.resume) rr = A.resume[wk.rve];
  const bool resumed = A.resume != nullptr && rr.active != 0;
  // owned free nodes: correction d (= h - h_ref), velocity, step cap, CSR range
  const bool warm = resumed || wk.kind == 1 || (A.warm_start && A.valid[wk.rve]);
  T hx[NPT], hy[NPT], hz[NPT], vx[NPT], vy[NPT], vz[NPT];
  float cap[NPT];
  uint32_t cs[NPT];
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int a = tid + q * NT;
    hx[q] = hy[q] = hz[q] = T(0);
    vx[q] = vy[q] = vz[q] = T(0);
    cap[q] = 0.f;
    cs[q] = 0u;
    if (a < nf) {
      cap[q] = A.ncap[M.node_off + a];
      cs[q] = A.ncsr[M.node_off + a];
      if (resumed) {
        const T* vv = A.vel + 4 * size_t(wk.state_off + a);
        vx[q] = vv[0];
        vy[q] = vv[1];
        vz[q] = vv[2];
      }
    }
  }
  // boundary-fiber stress share (compensated) -> sBB, then R_aff
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
  // initial reference state: h_ref = warm state or 0 (P1 and CSR written above)
  __syncthreads();
  rebase<T, NT, NPT>(A, wk, M, sF, H, P0, P1, HR, true, warm, hx, hy, hz);

  // ---- dynamic relaxation loop
  const int K = A.check_every;
  // kinetic damping: no viscous term (c = 0, so alpha = beta = 1); when the
  // kinetic energy of a step is below the previous step's, that step went
  // past a peak: it is taken back and the motion restarts from rest.
  // Otherwise viscous damping, fixed or adaptive.
  constexpr bool kinetic = VAR == VAR_KINETIC;
  constexpr bool energy = VAR == VAR_ENERGY;
  const bool adaptive = !kinetic && !(A.damping > 0.0);
  double c = kinetic ? 0.0 : (adaptive ? DAMP_C0 : A.damping);  // start value; then sC
  T ke_prev = T(0);      // kinetic energy (sum m |v|^2) of the previous iteration's step
  bool kin_half = true;  // kinetic damping: the next step starts from rest (half step)
  if (resumed) {
    c = rr.c;
    ke_prev = T(rr.ke_prev);
    kin_half = rr.kin_half != 0;
  }
  T alpha = T((2.0 - c) / (2.0 + c)), beta = T(2.0 / (2.0 + c));
  if (tid == 0) {
    sAB[0] = alpha;
    sAB[1] = beta;
    sC = c;
  }
  double pre = 0.0, pm = 0.0;  // thread partials (FP64) from the iteration before a check
  bool have_pre = false;
  // energy balance, per thread in T over a check interval (VAR_ENERGY), per
  // step with the mean velocity vb = (v_old + v_new)/2 of the step taken:
  // e_loss = f.vb - m (|v_new|^2 - |v_old|^2)/2, the kinetic energy the step
  // lost to damping and the step cap; e_damp = c m |vb|^2, its viscous part;
  // e_mass = (m - m_prev) |v_old|^2 / 2, the work of the mass change (the
  // mass is re-evaluated every iteration)
  T e_loss = T(0), e_damp = T(0), e_mass = T(0);
  T m_prev[NPT];
#pragma unroll
  for (int q = 0; q < NPT; ++q) m_prev[q] = T(0);
  if (energy && tid < 8) sEn[tid] = 0.0;
  int it = resumed ? rr.it : 0, n_checks = resumed ? rr.n_checks : 0;
  const int it0 = it;  // where this launch took the solve up (wave length)
  // stress-convergence test: below thr_tight the residual alone decides
  const bool sig_test = A.sigma_tol > 0.0;
  if (tid == 0) {
    const double thr_tight = fmax(1e-3 * A.sigma_tol * sqrt(raff2), ABS_FLOOR * M.sum_EA);
    sThr[0] = thr2;
    sThr[1] = thr_tight * thr_tight;
    for (int k = 0; k <= SIG_WINDOW; ++k) sSig[k][7] = 0.0;  // "record present" flags
  }
  __syncthreads();
  int status = RVE_STATUS_EMPTY;
  if (nf > 0 && !badF) {
    status = RVE_STATUS_MAX_ITER;
    int to_check = 0;  // iterations until the next check (it % K without a division)
    for (;; ++it) {
      const bool check = (to_check == 0) || (it >= A.max_iter);
      to_check = (to_check == 0) ? K - 1 : to_check - 1;
      const bool want_sig = check && sig_test;
      // fiber phase (RVE_FIBER_UNROLL fibers per step: independent shared-memory loads overlap)
      for (int e = tid; e < na; e += RVE_FIBER_UNROLL * NT) {
        V4 p0[RVE_FIBER_UNROLL], p1[RVE_FIBER_UNROLL], hi[RVE_FIBER_UNROLL], hj[RVE_FIBER_UNROLL];
#pragma unroll
        for (int u = 0; u < RVE_FIBER_UNROLL; ++u) {
          const int eu = (e + u * NT < na) ? e + u * NT : e;
          p0[u] = P0[eu];
          p1[u] = P1[eu];
        }
#pragma unroll
        for (int u = 0; u < RVE_FIBER_UNROLL; ++u) {
          const uint32_t ij = k_unpack_ij(p1[u].w);
          hi[u] = H[ij & 0xffffu];
          hj[u] = H[ij >> 16];
        }
#pragma unroll
        for (int u = 0; u < RVE_FIBER_UNROLL; ++u) {
          if (u == 0 || e + u * NT < na) {
            T Dx, Dy, Dz, s, sbar;
            fiber_force<T>(p0[u], p1[u], hi[u], hj[u], Dx, Dy, Dz, s, sbar);
            V4 o;
            o.x = s * Dx;
            o.y = s * Dy;
            o.z = s * Dz;
            o.w = sbar;
            SCR[e + u * NT] = o;
          }
        }
      }
      __syncthreads();
      // gather: the first run of 4 CSR entries of every owned node is loaded
      // unconditionally (a free node keeps >= 2 fibers, its run is padded to 4
      // with the zero slot), so all owned nodes' loads are in flight together;
      // nodes with more than 4 fibers continue in a loop.
      T fx[NPT], fy[NPT], fz[NPT], fw[NPT];
      {
        uint2 pk[NPT];
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          const int a = tid + q * NT;
          pk[q] = (a < nf) ? *reinterpret_cast<const uint2*>(CSR + (cs[q] >> 8)) : make_uint2(zero_run, zero_run);
        }
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          const uint32_t e0 = pk[q].x & 0xffffu, e1 = pk[q].x >> 16, e2 = pk[q].y & 0xffffu, e3 = pk[q].y >> 16;
          const V4 s0 = SCR[e0 >> 1], s1 = SCR[e1 >> 1], s2 = SCR[e2 >> 1], s3 = SCR[e3 >> 1];
          const T g0 = (e0 & 1u) ? T(-1) : T(1), g1 = (e1 & 1u) ? T(-1) : T(1);
          const T g2 = (e2 & 1u) ? T(-1) : T(1), g3 = (e3 & 1u) ? T(-1) : T(1);
          fx[q] = g0 * s0.x + g1 * s1.x + g2 * s2.x + g3 * s3.x;
          fy[q] = g0 * s0.y + g1 * s1.y + g2 * s2.y + g3 * s3.y;
          fz[q] = g0 * s0.z + g1 * s1.z + g2 * s2.z + g3 * s3.z;
          fw[q] = (s0.w + s1.w) + (s2.w + s3.w);
        }
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          const int a = tid + q * NT;
          if (a < nf) {
            const uint32_t b = cs[q] >> 8, n = cs[q] & 0xffu;  // n is a multiple of 4
            for (uint32_t k = 4; k < n; k += 4) {
              const uint2 p2 = *reinterpret_cast<const uint2*>(CSR + b + k);
              const uint32_t e0 = p2.x & 0xffffu, e1 = p2.x >> 16, e2 = p2.y & 0xffffu, e3 = p2.y >> 16;
              const V4 s0 = SCR[e0 >> 1], s1 = SCR[e1 >> 1], s2 = SCR[e2 >> 1], s3 = SCR[e3 >> 1];
              const T g0 = (e0 & 1u) ? T(-1) : T(1), g1 = (e1 & 1u) ? T(-1) : T(1);
              const T g2 = (e2 & 1u) ? T(-1) : T(1), g3 = (e3 & 1u) ? T(-1) : T(1);
              fx[q] += g0 * s0.x + g1 * s1.x + g2 * s2.x + g3 * s3.x;
              fy[q] += g0 * s0.y + g1 * s1.y + g2 * s2.y + g3 * s3.y;
              fz[q] += g0 * s0.z + g1 * s1.z + g2 * s2.z + g3 * s3.z;
              fw[q] += (s0.w + s1.w) + (s2.w + s3.w);
            }
          }
        }
      }
      bool do_rebase = false;
      if (check) {
        // ||f||^2, v.(f_new - f_old) and v.M v: each node's term in the loop
        // type, every sum over nodes in FP64 (per thread, per warp, across
        // warps); warp 0 finishes the cross-warp sum and its lane 0 takes every
        // block-uniform decision once (convergence, damping) and publishes it
        // in shared memory.  (GB300 runs FP64 at 1/64 of the FP32 rate: the
        // per-node products in FP64 cost 8 % of the loop at checks every 50
        // iterations.)
        double t3[3] = {0.0, 0.0, pm};
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          if (tid + q * NT < nf) {
            t3[0] += double(fx[q] * fx[q] + fy[q] * fy[q] + fz[q] * fz[q]);
            t3[1] += double(vx[q] * fx[q] + vy[q] * fy[q] + vz[q] * fz[q]);
          }
        }
        t3[1] -= pre;
        // stress-convergence test: the fiber stress sum at this iterate, in a
        // pass of its own (the fiber loop keeps no FP64 partials live)
        T ps_t[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (want_sig) {
          for (int e = tid; e < na; e += NT) {
            T Dx, Dy, Dz, sv, sbar;
            const V4 p1 = P1[e];
            const uint32_t ij = k_unpack_ij(p1.w);
            fiber_force<T>(P0[e], p1, H[ij & 0xffffu], H[ij >> 16], Dx, Dy, Dz, sv, sbar);
            V4 o;
            o.x = sv * Dx;
            o.y = sv * Dy;
            o.z = sv * Dz;
            o.w = sbar;
            add_virial(ps_t, o, Dx, Dy, Dz);
          }
        }
        double ps[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) ps[k] = double(ps_t[k]);
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int k = 0; k < 3; ++k) t3[k] = warp_sum(t3[k]);
        if (sig_test) {
#pragma unroll
          for (int k = 0; k < 6; ++k) ps[k] = warp_sum(ps[k]);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) red[warp * 9 + k] = t3[k];
          if (sig_test) {
#pragma unroll
            for (int k = 0; k < 6; ++k) red[warp * 9 + 3 + k] = ps[k];
          }
        }
        __syncthreads();
        if (warp == 0)
          check_decide<T, NT / 32>(red, sig_test, n_checks, it, it0, have_pre, adaptive, A.max_iter, A.damping_scale,
                                   A.sigma_tol, A.resume ? A.wave_iters : 0, sThr, sSig, sBB, sAB, &sC, &sFlag);
        __syncthreads();
        const int flag = sFlag;
        if constexpr (energy) {
          // Energy balance at this iterate x^n (Belytschko's check; three
          // further sums of the state, as Algorithm 2 notes): the exact stored
          // energy W of the active fibers (boundary-to-boundary fibers keep
          // their length), the kinetic energy K of the last half step, the
          // losses and mass work summed over the steps.  Along the trajectory
          // -sum f.vb - v_old.f^n / 2 is the trapezoidal rule of the force
          // work, and K + L - M equals it exactly (L = sum e_loss, M = sum
          // e_mass), so the residual dW + K + L - M + v_old.f^n / 2 is the
          // quadrature error of the central difference's steps against the
          // exact energy change dW: the time-integration error the check
          // exists to expose.
          double ev[6] = {double(e_loss), double(e_damp), double(e_mass), 0.0, 0.0, 0.0};
#pragma unroll
          for (int q = 0; q < NPT; ++q) {
            if (tid + q * NT < nf) {
              ev[3] += 0.5 * double(m_prev[q]) * double(vx[q] * vx[q] + vy[q] * vy[q] + vz[q] * vz[q]);
              ev[4] += 0.5 * double(vx[q] * fx[q] + vy[q] * fy[q] + vz[q] * fz[q]);
            }
          }
          for (int e = tid; e < na; e += NT) {
            const V4 p0 = P0[e], p1 = P1[e];
            const uint32_t ij = k_unpack_ij(p1.w);
            const V4 hi = H[ij & 0xffffu], hj = H[ij >> 16];
            const T dx = p0.x + (hj.x - hi.x), dy = p0.y + (hj.y - hi.y), dz = p0.z + (hj.z - hi.z);
            ev[5] += double(fiber_energy_gl8<T>(sqrt(dx * dx + dy * dy + dz * dz), p1.x, p1.y, p1.z));
          }
          block_allreduce<NT, 6>(ev, red);
          if (tid == 0) {
            sEn[1] += ev[0];  // L
            sEn[2] += ev[1];  // D
            sEn[3] += ev[2];  // M
            if (n_checks == 0) sEn[0] = ev[5];  // stored energy at the start state
            const double dW = ev[5] - sEn[0], K = ev[3];
            sEn[4] = dW;
            sEn[5] = K;
            const double scale = fmax(fmax(fabs(dW), K), sEn[1]);
            if (scale > 1e-300) sEn[6] = fmax(sEn[6], fabs(dW + K + sEn[1] - sEn[3] + ev[4]) / scale);
          }
          e_loss = e_damp = e_mass = T(0);
          __syncthreads();  // red is free again
        }
        if (flag == RVE_STATUS_NONFINITE || flag == RVE_STATUS_CONVERGED) {
          status = flag;
          break;
        }
        if (flag == RVE_STATUS_MAX_ITER) break;  // status is already RVE_STATUS_MAX_ITER
        if (flag == RVE_STATUS_PARKED_INTERNAL) {
          status = flag;
          break;
        }
        alpha = sAB[0];
        beta = sAB[1];
        pre = 0.0;
        pm = 0.0;
        have_pre = false;
        ++n_checks;
        do_rebase = std::is_same<T, float>::value && (n_checks % REBASE_EVERY == 0);
      }
      const bool pre_it = adaptive && (to_check == 0);  // the iteration before a check
      T b_step = beta;    // beta, or beta / 2 on the first step from rest
      bool undo = false;  // kinetic damping: take back the step that went past a peak
      if (kinetic) {
        if (it > 0) {
          // the kinetic energy of the step taken last iteration (partials
          // published before the barrier that ended it)
          const T* kp = sKE[(it - 1) & 1];
          T ke = T(0);
          for (int w = 0; w < NT / 32; ++w) ke += kp[w];
          if (ke < ke_prev) {
            undo = true;
            ke_prev = T(0);
          } else {
            ke_prev = ke;
          }
        }
        if (kin_half) b_step = T(0.5) * beta;  // central difference's starting half step v = (dt/2) f/m
      }
      T ke_t = T(0);
      // update owned nodes
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        const int a = tid + q * NT;
        if (a < nf) {
          const T m = T(MASS_COEF) * fw[q];
          T nvx, nvy, nvz;
          if (undo) {
            // past the kinetic-energy peak: back to the position before the
            // last step, at rest; no step this iteration (the forces just
            // gathered belong to the position being left)
            hx[q] -= vx[q];
            hy[q] -= vy[q];
            hz[q] -= vz[q];
            nvx = nvy = nvz = T(0);
          } else {
            const T bm = k_div(b_step, m);  // fictitious mass: an approximate quotient is enough
            nvx = alpha * vx[q] + bm * fx[q];
            nvy = alpha * vy[q] + bm * fy[q];
            nvz = alpha * vz[q] + bm * fz[q];
            const T sp2 = nvx * nvx + nvy * nvy + nvz * nvz;
            const T cp = T(cap[q]);
            if (sp2 > cp * cp) {
              const T sc = cp * k_rsqrt(sp2);
              nvx *= sc;
              nvy *= sc;
              nvz *= sc;
            }
            if constexpr (energy) {
              const T cc = T(2) * (T(1) - alpha) / (T(1) + alpha);
              const T bx = T(0.5) * (vx[q] + nvx), by = T(0.5) * (vy[q] + nvy), bz = T(0.5) * (vz[q] + nvz);
              const T v2 = vx[q] * vx[q] + vy[q] * vy[q] + vz[q] * vz[q];
              e_loss += (bx * fx[q] + by * fy[q] + bz * fz[q]) - T(0.5) * m * (nvx * nvx + nvy * nvy + nvz * nvz - v2);
              e_damp += cc * m * (bx * bx + by * by + bz * bz);
              e_mass += T(0.5) * (m - m_prev[q]) * v2;
              m_prev[q] = m;
            }
            hx[q] += nvx;
            hy[q] += nvy;
            hz[q] += nvz;
          }
          vx[q] = nvx;
          vy[q] = nvy;
          vz[q] = nvz;
          V4 h4;
          h4.x = hx[q];
          h4.y = hy[q];
          h4.z = hz[q];
          h4.w = T(0);
          H[a] = h4;
          if (pre_it) {
            pre += double(nvx * fx[q] + nvy * fy[q] + nvz * fz[q]);
            pm += double(m * (nvx * nvx + nvy * nvy + nvz * nvz));
          }
          if (kinetic) ke_t += m * (nvx * nvx + nvy * nvy + nvz * nvz);
        }
      }
      kin_half = undo;  // after a take-back the next step starts from rest
      if (pre_it) have_pre = true;
      if (kinetic) {
        ke_t = warp_sum_t(ke_t);
        if ((tid & 31) == 0) sKE[it & 1][tid >> 5] = ke_t;
      }
      if (do_rebase) {
        rebase<T, NT, NPT>(A, wk, M, sF, H, P0, P1, HR, false, true, hx, hy, hz);
      } else {
        __syncthreads();
      }
    }
  }

  if (status == RVE_STATUS_PARKED_INTERNAL) {
    // park: h = h_ref + d into the state, the velocity and the loop scalars
    // beside it; the next wave resumes from here (no stress yet)
    double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int a = tid + q * NT;
      if (a < nf) {
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
      r.ke_prev = float(ke_prev);
      r.kin_half = kin_half ? 1 : 0;
      r.active = 1;
      r.pad = 0;
      A.resume[wk.rve] = r;
      if (A.iters) A.iters[wk.out] = it;
      if (A.status) A.status[wk.out] = status;
    }
    pdl_epilogue(A);
    return;
  }

  // ---- stress: active fibers at the final state (P0 at h_ref, H holds d)
  __syncthreads();  // red free (last allreduce read before the previous barrier)
  fiber_stress_partials<T, V4>(P0, P1, H, na, tid, NT, red);
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
  // save state: h = h_ref + d (FP64)
  {
    double* st = A.state + 4 * size_t(wk.state_off);
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int a = tid + q * NT;
      if (a < nf) {
        st[4 * a + 0] += double(hx[q]);
        st[4 * a + 1] += double(hy[q]);
        st[4 * a + 2] += double(hz[q]);
      }
    }
  }
  __syncthreads();
  if (tid < 9) {
    // sigma components in order xx yy zz yz xz xy
    const int i = tid / 3, j = tid % 3;
    const int idx = (i == j) ? i : 6 - i - j;
    A.sigma[9 * size_t(wk.out) + tid] = badF ? __longlong_as_double(0x7ff8000000000000ll)
                                              : sRes[idx] / (detF * M.V0);
  }
  if (tid == 0) {
    int st = status;
    if (badF) st = RVE_STATUS_NONFINITE;
    if (wk.kind == 0) {
      A.valid[wk.rve] = (st == RVE_STATUS_NONFINITE) ? 0 : 1;  // never warm-start from NaN
      A.last_iters[wk.rve] = it;
    }
    if (A.resume) A.resume[wk.rve].active = 0;  // the next request starts afresh
    if (energy && A.energy) {
      double* E = A.energy + 6 * size_t(wk.out);
      E[0] = sEn[4];           // stored-energy change from the start state
      E[1] = sEn[5];           // kinetic energy at the last check
      E[2] = sEn[2];           // viscous damping dissipation
      E[3] = sEn[1] - sEn[2];  // further loss (step cap)
      E[4] = sEn[3];           // work of the mass changes
      E[5] = sEn[6];           // largest relative balance error over the checks
    }
    if (A.iters) A.iters[wk.out] = it;
    if (A.status) A.status[wk.out] = st;
  }
  pdl_epilogue(A);
}

}  // namespace rvegpu
