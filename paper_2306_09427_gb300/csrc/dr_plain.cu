// Plain FP64 per-RVE path: the reference the batched kernel is measured
// against.  Like the paper's naive GPU approach (Sec. 4.3) it solves one
// RVE at a time with several kernel launches per dynamic-relaxation
// iteration and lets the host test convergence:
//   fiber kernel   per active fiber: (s d, sbar) into a global scratch;
//   node kernel    per free node: CSR gather of the fiber scratch, then the
//                  damped update (gather and update fused: same loop shape);
//   check          every check_every iterations the node kernel only
//                  gathers and writes per-block partial sums, a one-block
//                  kernel reduces them, the host reads the result back
//                  (synchronising the stream), decides, and a third node
//                  kernel applies the update.
// The arithmetic (fiber law, lumped mass, damping rule, step cap,
// convergence test) is the batched kernel's, in FP64.
#include <cmath>

#include "batch.h"
#include "dr_fused.cuh"

namespace rvegpu {

namespace {

constexpr int PT = 256;  // threads per block of the plain kernels

struct PlainBufs {
  dvec4 *P0, *P1, *SCR, *H, *V, *Fn;
  double* part;  // per block: pre, pm, r2, post
  double* res;   // [0] R_aff^2, [1..12] sigma_bb (s, c) pairs, [16..19] reduced partials
  double* sig;   // per block 12 doubles of stress partials
};

__global__ void pl_setup(const RveMeta* meta, int r, const FibD* fa, const uint32_t* fij, const FibD* fb,
                         const double* F, int out, const double* state, const uint8_t* valid, int warm_start,
                         PlainBufs B) {
  const RveMeta M = meta[r];
  __shared__ double sF[9], sE[9];
  __shared__ double red[(PT / 32) * 12 + 32];
  const int tid = threadIdx.x;
  if (tid < 9) sF[tid] = F[9 * size_t(out) + tid];
  __syncthreads();
  if (tid < 9) {
    const int k = tid / 3, l = tid % 3;
    sE[tid] = 0.5 * (sF[k] * sF[l] + sF[3 + k] * sF[3 + l] + sF[6 + k] * sF[6 + l] - (k == l ? 1.0 : 0.0));
  }
  __syncthreads();
  double raff2 = 0.0;
  for (int e = tid; e < M.na; e += PT) {
    const FibD q = fa[M.fa_off + e];
    const double gx = sF[0] * q.dx + sF[1] * q.dy + sF[2] * q.dz;
    const double gy = sF[3] * q.dx + sF[4] * q.dy + sF[5] * q.dz;
    const double gz = sF[6] * q.dx + sF[7] * q.dy + sF[8] * q.dz;
    const double ex = sE[0] * q.dx + sE[1] * q.dy + sE[2] * q.dz;
    const double ey = sE[3] * q.dx + sE[4] * q.dy + sE[5] * q.dz;
    const double ez = sE[6] * q.dx + sE[7] * q.dy + sE[8] * q.dz;
    const double L02 = q.L0 * q.L0;
    const double a = (q.dx * ex + q.dy * ey + q.dz * ez + 0.5 * (q.dx * q.dx + q.dy * q.dy + q.dz * q.dz - L02)) / L02;
    const double Na = law_f64(a, q.EA, q.B);
    raff2 += Na * Na;
    B.P0[e] = dvec4{gx, gy, gz, a};
    B.P1[e] = dvec4{0.5 / L02, q.B > 0.0 ? q.EA / q.B : q.EA, q.B, double(fij[M.fa_off + e])};
  }
  CSum sb[6];
  for (int e = tid; e < M.nb; e += PT) {
    const FibD q = fb[M.fb_off + e];
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
    sb[0].add(s * gx * gx);
    sb[1].add(s * gy * gy);
    sb[2].add(s * gz * gz);
    sb[3].add(s * gy * gz);
    sb[4].add(s * gx * gz);
    sb[5].add(s * gx * gy);
  }
  const bool warm = warm_start && valid[r];
  for (int a = tid; a < M.nf; a += PT) {
    dvec4 h{0.0, 0.0, 0.0, 0.0};
    if (warm) {
      const dvec4 s4 = reinterpret_cast<const dvec4*>(state)[M.node_off + a];
      h = dvec4{s4.x, s4.y, s4.z, 0.0};
    }
    B.H[a] = h;
    B.V[a] = dvec4{0.0, 0.0, 0.0, 0.0};
  }
  if (tid == 0) {
    B.H[M.nf] = dvec4{0.0, 0.0, 0.0, 0.0};
    B.SCR[M.na] = dvec4{0.0, 0.0, 0.0, 0.0};  // zero slot of the padded CSR runs
  }
  const int warp = tid >> 5, lane = tid & 31;
  const double r2 = warp_sum(raff2);
  for (int k = 0; k < 6; ++k) {
    double s = sb[k].s, c = sb[k].c;
    warp_csum(s, c);
    if (lane == 0) {
      red[(warp * 6 + k) * 2] = s;
      red[(warp * 6 + k) * 2 + 1] = c;
    }
  }
  if (lane == 0) red[(PT / 32) * 12 + warp] = r2;
  __syncthreads();
  if (tid < 6) {
    double s = 0.0, c = 0.0;
    for (int w = 0; w < PT / 32; ++w) {
      double t, e;
      two_sum(s, red[(w * 6 + tid) * 2], t, e);
      s = t;
      c += e + red[(w * 6 + tid) * 2 + 1];
    }
    B.res[1 + 2 * tid] = s;
    B.res[2 + 2 * tid] = c;
  }
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < PT / 32; ++w) s += red[(PT / 32) * 12 + w];
    B.res[0] = s;
    B.res[13] = sF[0] * (sF[4] * sF[8] - sF[5] * sF[7]) - sF[1] * (sF[3] * sF[8] - sF[5] * sF[6]) +
                sF[2] * (sF[3] * sF[7] - sF[4] * sF[6]);
  }
}

// per active fiber: (s d, sbar); with want_sig also per-block stress partials
__global__ void pl_fiber(int na, int want_sig, PlainBufs B) {
  const int e = blockIdx.x * PT + threadIdx.x;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (e < na) {
    const dvec4 p0 = B.P0[e], p1 = B.P1[e];
    const uint32_t ij = static_cast<uint32_t>(p1.w);
    const dvec4 hi = B.H[ij & 0xffffu], hj = B.H[ij >> 16];
    double Dx, Dy, Dz, s, sbar;
    fiber_force<double>(p0, p1, hi, hj, Dx, Dy, Dz, s, sbar);
    const dvec4 o{s * Dx, s * Dy, s * Dz, sbar};
    B.SCR[e] = o;
    t[0] = o.x * Dx;
    t[1] = o.y * Dy;
    t[2] = o.z * Dz;
    t[3] = o.y * Dz;
    t[4] = o.x * Dz;
    t[5] = o.x * Dy;
  }
  if (!want_sig) return;
  __shared__ double red[6 * (PT / 32)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum(t[k]);
    if (lane == 0) red[6 * warp + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < PT / 32; ++w) v += red[6 * w + threadIdx.x];
    B.sig[12 * blockIdx.x + threadIdx.x] = v;
  }
}

__device__ __forceinline__ void pl_gather(int a, const RveMeta& M, const uint16_t* csr, const uint32_t* ncsr,
                                          const dvec4* SCR, double& fx, double& fy, double& fz, double& fw) {
  const uint32_t cs = ncsr[M.node_off + a];
  const uint16_t* C = csr + M.csr_off;
  fx = fy = fz = fw = 0.0;
  for (uint32_t k = 0; k < (cs & 0xffu); ++k) {
    const uint32_t ent = C[(cs >> 8) + k];
    const dvec4 s4 = SCR[ent >> 1];
    if (ent & 1u) {
      fx -= s4.x;
      fy -= s4.y;
      fz -= s4.z;
    } else {
      fx += s4.x;
      fy += s4.y;
      fz += s4.z;
    }
    fw += s4.w;
  }
}

__device__ __forceinline__ void pl_update(int a, const RveMeta& M, const float* ncap, double fx, double fy, double fz,
                                          double fw, double alpha, double beta, PlainBufs& B, double& pre,
                                          double& pm) {
  const double m = MASS_COEF * fw;
  const double bm = beta / m;
  const dvec4 v = B.V[a];
  double nvx = alpha * v.x + bm * fx, nvy = alpha * v.y + bm * fy, nvz = alpha * v.z + bm * fz;
  const double sp2 = nvx * nvx + nvy * nvy + nvz * nvz;
  const double cp = double(ncap[M.node_off + a]);
  if (sp2 > cp * cp) {
    const double sc = cp / sqrt(sp2);
    nvx *= sc;
    nvy *= sc;
    nvz *= sc;
  }
  B.V[a] = dvec4{nvx, nvy, nvz, 0.0};
  const dvec4 h = B.H[a];
  B.H[a] = dvec4{h.x + nvx, h.y + nvy, h.z + nvz, 0.0};
  pre += nvx * fx + nvy * fy + nvz * fz;
  pm += m * (nvx * nvx + nvy * nvy + nvz * nvz);
}

// block sum of two doubles into part[blk*4 + slot .. slot+1]
__device__ __forceinline__ void block_pair(double a, double b, double* part, int slot) {
  __shared__ double red[2 * (PT / 32)];
  a = warp_sum(a);
  b = warp_sum(b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[2 * warp] = a;
    red[2 * warp + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < PT / 32; ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    part[blockIdx.x * 4 + slot] = s0;
    part[blockIdx.x * 4 + slot + 1] = s1;
  }
}

// gather + update (non-check iterations); pre_it: record the Rayleigh partials
__global__ void pl_node(const RveMeta* meta, int r, const uint16_t* csr, const uint32_t* ncsr, const float* ncap,
                        double alpha, double beta, int pre_it, PlainBufs B) {
  const RveMeta M = meta[r];
  const int a = blockIdx.x * PT + threadIdx.x;
  double pre = 0.0, pm = 0.0;
  if (a < M.nf) {
    double fx, fy, fz, fw;
    pl_gather(a, M, csr, ncsr, B.SCR, fx, fy, fz, fw);
    pl_update(a, M, ncap, fx, fy, fz, fw, alpha, beta, B, pre, pm);
  }
  if (pre_it) block_pair(pre, pm, B.part, 0);
}

// gather only (check iterations): forces kept, residual partials written
__global__ void pl_node_check(const RveMeta* meta, int r, const uint16_t* csr, const uint32_t* ncsr, PlainBufs B) {
  const RveMeta M = meta[r];
  const int a = blockIdx.x * PT + threadIdx.x;
  double r2 = 0.0, post = 0.0;
  if (a < M.nf) {
    double fx, fy, fz, fw;
    pl_gather(a, M, csr, ncsr, B.SCR, fx, fy, fz, fw);
    B.Fn[a] = dvec4{fx, fy, fz, fw};
    const dvec4 v = B.V[a];
    r2 = fx * fx + fy * fy + fz * fz;
    post = v.x * fx + v.y * fy + v.z * fz;
  }
  block_pair(r2, post, B.part, 2);
}

__global__ void pl_node_apply(const RveMeta* meta, int r, const float* ncap, double alpha, double beta, int pre_it,
                              PlainBufs B) {
  const RveMeta M = meta[r];
  const int a = blockIdx.x * PT + threadIdx.x;
  double pre = 0.0, pm = 0.0;
  if (a < M.nf) {
    const dvec4 f = B.Fn[a];
    pl_update(a, M, ncap, f.x, f.y, f.z, f.w, alpha, beta, B, pre, pm);
  }
  if (pre_it) block_pair(pre, pm, B.part, 0);
}

// res[16..19] = pre, pm, r2, post; res[20..25] = stress partial sums
__global__ void pl_reduce(int nblk, int nblk_a, int want_sig, PlainBufs B) {
  __shared__ double red[10 * (PT / 32)];
  double v[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += PT)
    for (int k = 0; k < 4; ++k) v[k] += B.part[4 * b + k];
  if (want_sig)
    for (int b = threadIdx.x; b < nblk_a; b += PT)
      for (int k = 0; k < 6; ++k) v[4 + k] += B.sig[12 * b + k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 10; ++k) {
    v[k] = warp_sum(v[k]);
    if (lane == 0) red[10 * warp + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double s = 0.0;
    for (int w = 0; w < PT / 32; ++w) s += red[10 * w + threadIdx.x];
    B.res[16 + threadIdx.x] = s;
  }
}

__global__ void pl_sigma(int na, PlainBufs B) {
  __shared__ double red[(PT / 32) * 12];
  const int e = blockIdx.x * PT + threadIdx.x;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (e < na) {
    const dvec4 p0 = B.P0[e], p1 = B.P1[e];
    const uint32_t ij = static_cast<uint32_t>(p1.w);
    double Dx, Dy, Dz, s, sbar;
    fiber_force<double>(p0, p1, B.H[ij & 0xffffu], B.H[ij >> 16], Dx, Dy, Dz, s, sbar);
    t[0] = s * Dx * Dx;
    t[1] = s * Dy * Dy;
    t[2] = s * Dz * Dz;
    t[3] = s * Dy * Dz;
    t[4] = s * Dx * Dz;
    t[5] = s * Dx * Dy;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 6; ++k) {
    double s = t[k], c = 0.0;
    warp_csum(s, c);
    if (lane == 0) {
      red[(warp * 6 + k) * 2] = s;
      red[(warp * 6 + k) * 2 + 1] = c;
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0, c = 0.0;
    for (int w = 0; w < PT / 32; ++w) {
      double tt, ee;
      two_sum(s, red[(w * 6 + threadIdx.x) * 2], tt, ee);
      s = tt;
      c += ee + red[(w * 6 + threadIdx.x) * 2 + 1];
    }
    B.sig[12 * blockIdx.x + 2 * threadIdx.x] = s;
    B.sig[12 * blockIdx.x + 2 * threadIdx.x + 1] = c;
  }
}

__global__ void pl_finish(const RveMeta* meta, int r, int nblk, const double* F, int out, int it, int status,
                          double* sigma, int32_t* iters, int32_t* st, uint8_t* valid, PlainBufs B) {
  __shared__ double comp[6];
  const RveMeta M = meta[r];
  if (threadIdx.x < 6) {
    double s = B.res[1 + 2 * threadIdx.x], c = B.res[2 + 2 * threadIdx.x];
    for (int b = 0; b < nblk; ++b) {
      double tt, ee;
      two_sum(s, B.sig[12 * b + 2 * threadIdx.x], tt, ee);
      s = tt;
      c += ee + B.sig[12 * b + 2 * threadIdx.x + 1];
    }
    comp[threadIdx.x] = s + c;
  }
  __syncthreads();
  const double* f = F + 9 * size_t(out);
  const double detF = f[0] * (f[4] * f[8] - f[5] * f[7]) - f[1] * (f[3] * f[8] - f[5] * f[6]) +
                      f[2] * (f[3] * f[7] - f[4] * f[6]);
  const bool badF = !(detF > 0.0) || !(detF < 1e300);
  if (threadIdx.x < 9) {
    const int i = threadIdx.x / 3, j = threadIdx.x % 3;
    const int idx = (i == j) ? i : 6 - i - j;  // xx yy zz | yz xz xy
    sigma[9 * size_t(out) + threadIdx.x] = badF ? __longlong_as_double(0x7ff8000000000000ll) : comp[idx] / (detF * M.V0);
  }
  if (threadIdx.x == 0) {
    const int s = badF ? RVE_STATUS_NONFINITE : status;
    if (iters) iters[out] = it;
    if (st) st[out] = s;
    valid[r] = s == RVE_STATUS_NONFINITE ? 0 : 1;
  }
}

__global__ void pl_save(const RveMeta* meta, int r, double* state, PlainBufs B) {
  const RveMeta M = meta[r];
  const int a = blockIdx.x * PT + threadIdx.x;
  if (a < M.nf) reinterpret_cast<dvec4*>(state)[M.node_off + a] = B.H[a];
}

}  // namespace

int plain_scratch_bytes(int nf_max, int na_max) {
  const int nblk_n = (nf_max + PT - 1) / PT + 1, nblk_a = (na_max + PT - 1) / PT + 1;
  return int(sizeof(dvec4)) * (3 * (na_max + 1) + 3 * (nf_max + 1)) + 8 * (4 * nblk_n + 32 + 12 * nblk_a) + 1024;
}

namespace {

// Carve the plain path's working buffers for one RVE out of `base`;
// returns the bytes used (256-byte aligned pieces).
size_t carve_plain(unsigned char* base, int nf, int na, PlainBufs& B) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align_up(bytes, 256);
    return p;
  };
  B.P0 = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(na + 1)));
  B.P1 = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(na + 1)));
  B.SCR = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(na + 1)));
  B.H = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(nf + 1)));
  B.V = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(nf + 1)));
  B.Fn = reinterpret_cast<dvec4*>(take(sizeof(dvec4) * size_t(nf + 1)));
  const int nblk_n = (nf + PT - 1) / PT, nblk_a = (na + PT - 1) / PT;
  B.part = reinterpret_cast<double*>(take(sizeof(double) * 4 * size_t(nblk_n + 1)));
  B.res = reinterpret_cast<double*>(take(sizeof(double) * 32));
  B.sig = reinterpret_cast<double*>(take(sizeof(double) * 12 * size_t(nblk_a + 1)));
  return off;
}

// Set-up and host-driven DR loop of the plain path for RVE r (F[9*out..]).
// On return it / st hold the iterations and status; B.H holds the final state.
int plain_run(rve_batch* b, int r, int out, const double* F, double tol, int max_iter, const PlainBufs& B,
              cudaStream_t s, const double* state, const uint8_t* valid, int warm_start, int& it_out, int& st_out) {
  const RveMeta& M = b->topo.meta[r];
  const int na = M.na, nf = M.nf;
  const int nblk_n = (nf + PT - 1) / PT, nblk_a = (na + PT - 1) / PT;
  RVE_CUDA_TRY(cudaMemsetAsync(B.part, 0, sizeof(double) * 4 * size_t(nblk_n + 1), s));
  RVE_CUDA_TRY(cudaMemsetAsync(B.res, 0, sizeof(double) * 32, s));
  pl_setup<<<1, PT, 0, s>>>(b->d_meta, r, b->d_fa, b->d_fij, b->d_fb, F, out, state, valid, warm_start, B);
  RVE_CUDA_TRY(cudaGetLastError());
  RVE_CUDA_TRY(cudaMemcpyAsync(b->h_pl, B.res, 14 * sizeof(double), cudaMemcpyDeviceToHost, s));
  RVE_CUDA_TRY(cudaStreamSynchronize(s));
  const double raff = std::sqrt(b->h_pl[0]);
  double sbb[6];
  for (int k = 0; k < 6; ++k) sbb[k] = b->h_pl[1 + 2 * k] + b->h_pl[2 + 2 * k];
  const double detF = b->h_pl[13];
  const bool badF = !(detF > 0.0) || !(detF < 1e300);  // reported as non-finite by the finish kernel
  const double thr = std::fmax(tol * raff, ABS_FLOOR * M.sum_EA);
  const double thr2 = thr * thr;
  const bool sig_test = b->opt.sigma_tol > 0.0;
  const double thr_tight = std::fmax(1e-3 * b->opt.sigma_tol * raff, ABS_FLOOR * M.sum_EA);
  const int K = b->opt.check_every;
  const bool adaptive = !(b->opt.damping > 0.0);
  double c = adaptive ? DAMP_C0 : b->opt.damping;
  const double scale = b->opt.damping_scale > 0.0 ? b->opt.damping_scale : DAMP_SCALE;
  double alpha = (2.0 - c) / (2.0 + c), beta = 2.0 / (2.0 + c);
  bool have_pre = false;
  double sig_hist[SIG_WINDOW + 1][8] = {};  // ring of (stress, residual, present) per check
  int n_checks = 0;
  int it = 0, st = RVE_STATUS_EMPTY;
  if (nf > 0 && !badF) {
    st = RVE_STATUS_MAX_ITER;
    for (;; ++it) {
      const bool check = (it % K == 0) || it >= max_iter;
      const int pre_it = adaptive && ((it + 1) % K == 0);
      pl_fiber<<<(na + PT - 1) / PT, PT, 0, s>>>(na, check && sig_test, B);
      if (!check) {
        pl_node<<<nblk_n, PT, 0, s>>>(b->d_meta, r, b->d_csr, b->d_ncsr, b->d_ncap, alpha, beta, pre_it, B);
      } else {
        pl_node_check<<<nblk_n, PT, 0, s>>>(b->d_meta, r, b->d_csr, b->d_ncsr, B);
        pl_reduce<<<1, PT, 0, s>>>(nblk_n, nblk_a, sig_test, B);
        RVE_CUDA_TRY(cudaGetLastError());
        RVE_CUDA_TRY(cudaMemcpyAsync(b->h_pl, B.res + 16, 10 * sizeof(double), cudaMemcpyDeviceToHost, s));
        RVE_CUDA_TRY(cudaStreamSynchronize(s));
        const double pre = b->h_pl[0], pm = b->h_pl[1], r2 = b->h_pl[2], post = b->h_pl[3];
        if (!(r2 < 1e300)) {
          st = RVE_STATUS_NONFINITE;
          break;
        }
        bool sig_ok = true;
        double* next = sig_hist[n_checks % (SIG_WINDOW + 1)];
        if (sig_test && r2 > thr_tight * thr_tight) {
          const double* prev = sig_hist[(n_checks + 1) % (SIG_WINDOW + 1)];
          const double rr = std::sqrt(r2);
          double dn = 0.0, nn = 0.0;
          for (int k = 0; k < 6; ++k) {
            const double sg = b->h_pl[4 + k] + sbb[k];
            const double wk2 = k < 3 ? 1.0 : 2.0;
            dn += wk2 * (sg - prev[k]) * (sg - prev[k]);
            nn += wk2 * sg * sg;
            next[k] = sg;
          }
          sig_ok = false;
          if (prev[7] != 0.0 && nn > 0.0) {
            const double rho = std::fmin(rr / prev[6], SIG_RHO_CAP);
            sig_ok = std::sqrt(dn / nn) * rho / (1.0 - rho) <= b->opt.sigma_tol;
          }
          next[6] = rr;
          next[7] = 1.0;
        } else {
          next[7] = 0.0;
        }
        ++n_checks;
        if (r2 <= thr2 && sig_ok) {
          st = RVE_STATUS_CONVERGED;
          break;
        }
        if (it >= max_iter) break;
        if (adaptive && have_pre && pm > 0.0) {
          const double lam = -(post - pre) / pm;
          if (lam > 0.0) {
            c = std::fmin(scale * 2.0 * std::sqrt(lam), DAMP_C_MAX);
            alpha = (2.0 - c) / (2.0 + c);
            beta = 2.0 / (2.0 + c);
          }
        }
        pl_node_apply<<<nblk_n, PT, 0, s>>>(b->d_meta, r, b->d_ncap, alpha, beta, pre_it, B);
      }
      RVE_CUDA_TRY(cudaGetLastError());
      have_pre = pre_it != 0;
    }
  }
  it_out = it;
  st_out = st;
  return RVE_OK;
}

}  // namespace

// Solve RVE `r` with F[9*out..] on `s`, outputs at index `out`.
int plain_solve_one(rve_batch* b, int r, int out, const double* F, double tol, int max_iter, double* sigma,
                    int32_t* iters, int32_t* status, cudaStream_t s) {
  const RveMeta& M = b->topo.meta[r];
  PlainBufs B;
  if (carve_plain(reinterpret_cast<unsigned char*>(b->d_pl), M.nf, M.na, B) > b->pl_bytes)
    return fail(RVE_EINVAL, "plain scratch too small");
  int it = 0, st = 0;
  const int rc = plain_run(b, r, out, F, tol, max_iter, B, s, static_cast<double*>(b->pd.d_state), b->pd.d_valid,
                           b->opt.warm_start, it, st);
  if (rc != RVE_OK) return rc;
  const int nblk_n = (M.nf + PT - 1) / PT, nblk_a = (M.na + PT - 1) / PT;
  if (M.na > 0) pl_sigma<<<nblk_a, PT, 0, s>>>(M.na, B);
  pl_finish<<<1, 32, 0, s>>>(b->d_meta, r, M.na > 0 ? nblk_a : 0, F, out, it, st, sigma, iters, status,
                             b->pd.d_valid, B);
  if (M.nf > 0) pl_save<<<nblk_n, PT, 0, s>>>(b->d_meta, r, static_cast<double*>(b->pd.d_state), B);
  RVE_CUDA_TRY(cudaGetLastError());
  return RVE_OK;
}

}  // namespace rvegpu

// ---------------------------------------------------------------------------
// Allocation-free variant of the plain FP64 solve.
//
// Some callers must not allocate device memory while they solve: programs
// whose device memory is carved up once at start-up (a caching allocator
// or a fixed budget shared with other work, where a cudaMalloc may fail or
// implicitly synchronise the device and stall every stream) and loops with
// latency limits that forbid allocator calls.  rve_solve_plain_noalloc
// serves them: it solves one RVE of an existing batch with the plain FP64
// kernels above, taking its working buffers from a fixed scratch array
// compiled into this library instead of the batch's own scratch.  The
// array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (about 2.3 MB) until the process exits.
#include <mutex>

namespace rvegpu {
namespace {

constexpr int NOALLOC_NA = RVE_NOALLOC_MAX_ACTIVE_FIBERS;
constexpr int NOALLOC_NF = RVE_NOALLOC_MAX_FREE_NODES;

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t noalloc_bytes() {
  return 3 * na_align(sizeof(dvec4) * size_t(NOALLOC_NA + 1)) + 3 * na_align(sizeof(dvec4) * size_t(NOALLOC_NF + 1)) +
         na_align(sizeof(double) * 4 * size_t(NOALLOC_NF / PT + 2)) + na_align(sizeof(double) * 32) +
         na_align(sizeof(double) * 12 * size_t(NOALLOC_NA / PT + 2));
}

__device__ __align__(256) unsigned char g_noalloc_scratch[noalloc_bytes()];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// pl_finish without touching the batch's warm-start flags
__global__ void pl_finish_noalloc(const RveMeta* meta, int r, int nblk, const double* F, int it, int status,
                                  double* sigma, int32_t* iters, int32_t* st, PlainBufs B) {
  __shared__ double comp[6];
  const RveMeta M = meta[r];
  if (threadIdx.x < 6) {
    double s = B.res[1 + 2 * threadIdx.x], c = B.res[2 + 2 * threadIdx.x];
    for (int b = 0; b < nblk; ++b) {
      double tt, ee;
      two_sum(s, B.sig[12 * b + 2 * threadIdx.x], tt, ee);
      s = tt;
      c += ee + B.sig[12 * b + 2 * threadIdx.x + 1];
    }
    comp[threadIdx.x] = s + c;
  }
  __syncthreads();
  const double detF = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                      F[2] * (F[3] * F[7] - F[4] * F[6]);
  const bool badF = !(detF > 0.0) || !(detF < 1e300);
  if (threadIdx.x < 9) {
    const int i = threadIdx.x / 3, j = threadIdx.x % 3;
    const int idx = (i == j) ? i : 6 - i - j;
    sigma[threadIdx.x] = badF ? __longlong_as_double(0x7ff8000000000000ll) : comp[idx] / (detF * M.V0);
  }
  if (threadIdx.x == 0) {
    if (iters) *iters = it;
    if (st) *st = badF ? RVE_STATUS_NONFINITE : status;
  }
}

}  // namespace
}  // namespace rvegpu

extern "C" int rve_solve_plain_noalloc(rve_batch* b, int64_t r, const double* F, double tol, int32_t max_iter,
                                       double* sigma, int32_t* iters, int32_t* status, void* stream) {
  using namespace rvegpu;
  if (!b || !F || !sigma) return fail(RVE_EINVAL, "batch, F and sigma are required");
  if (r < 0 || r >= b->n_rve) return fail(RVE_EINVAL, "RVE index out of range");
  const RveMeta& M = b->topo.meta[r];
  if (M.na > NOALLOC_NA || M.nf > NOALLOC_NF)
    return fail(RVE_EINVAL, "RVE " + std::to_string(r) + " has " + std::to_string(M.na) + " active fibers and " +
                                std::to_string(M.nf) + " free nodes; rve_solve_plain_noalloc handles at most " +
                                std::to_string(NOALLOC_NA) + " and " + std::to_string(NOALLOC_NF));
  if (!(tol > 0.0)) tol = b->opt.tol;
  if (max_iter <= 0) max_iter = b->opt.max_iter;
  RVE_CUDA_TRY(cudaSetDevice(b->device));
  if (b->device < 0 || b->device >= 64) return fail(RVE_EINVAL, "device ordinal too large");
  void* base_v = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[b->device]) {
      void* p = nullptr;
      RVE_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[b->device] = p;
    }
    base_v = g_noalloc_addr[b->device];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PlainBufs B;
  if (carve_plain(static_cast<unsigned char*>(base_v), M.nf, M.na, B) > noalloc_bytes())
    return fail(RVE_EINVAL, "internal: no-alloc scratch layout overflow");
  // the array keeps the previous call's contents; plain_run clears what accumulates
  int it = 0, st = 0;
  const int rc = plain_run(b, int(r), 0, F, tol, max_iter, B, s, nullptr, nullptr, 0, it, st);
  if (rc != RVE_OK) return rc;
  const int na = M.na, nblk_a = (na + PT - 1) / PT;
  if (na > 0) pl_sigma<<<nblk_a, PT, 0, s>>>(na, B);
  pl_finish_noalloc<<<1, 32, 0, s>>>(b->d_meta, int(r), na > 0 ? nblk_a : 0, F, it, st, sigma, iters, status, B);
  RVE_CUDA_TRY(cudaGetLastError());
  return RVE_OK;
}
