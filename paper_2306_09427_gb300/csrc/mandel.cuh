// The paper's material tangent by six forward-difference solves (Sec. 3.2):
// device-side FP64 algebra around the batched solves, one thread per RVE.
//
// F = R U (polar decomposition).  The second Piola-Kirchhoff stress
// Pi = J F^-1 sigma F^-T depends on U only, so the six probing solves run at
// F_p = R (U + h T_p): by that invariance Pi(F_p) = Pi(U + h T_p), and the
// base solve's state at F = R U stays a valid warm start for all six.
// Then P_ij,p = (Pi_ij(F_p) - Pi_ij(F)) / h (Eq. tensor_fd), [A] solves
// [A][M][T] = [P] with M = dE/dU, and the spatial stiffness is the push
// forward C = J^-1 F F A F F (Eq. stiffness-push-forward), evaluated in
// Mandel form as [C] = J^-1 [Q][A][Q]^T with [Q] the Mandel matrix of the
// map a -> F a F^T on symmetric tensors.
//
// Mandel convention: index order (11, 22, 33, 23, 13, 12); shear entries of
// a symmetric tensor carry a factor sqrt(2), so inner products are kept.
#pragma once

#include <cuda_runtime.h>

namespace rvegpu {

constexpr int N_MANDEL = 6;  // probing directions

__device__ __forceinline__ void mandel_pair(int I, int& i, int& j) {
  i = I < 3 ? I : (I == 3 ? 1 : 0);
  j = I < 3 ? I : (I == 5 ? 1 : 2);
}
__device__ __forceinline__ double mandel_w(int I) { return I < 3 ? 1.0 : 1.4142135623730951; }

__device__ __forceinline__ double det3(const double a[3][3]) {
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

// inverse by the adjugate; returns the determinant
__device__ __forceinline__ double inv3(const double a[3][3], double o[3][3]) {
  const double d = det3(a);
  const double r = 1.0 / d;
  o[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) * r;
  o[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * r;
  o[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * r;
  o[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) * r;
  o[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * r;
  o[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * r;
  o[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) * r;
  o[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * r;
  o[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * r;
  return d;
}

__device__ __forceinline__ void mul3(const double a[3][3], const double b[3][3], double o[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j] + a[i][2] * b[2][j];
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
// each rotation in the (p, q) plane zeroes a_pq with t = tan(phi) the
// smaller root of t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq).
// On return a is diagonal (the eigenvalues) and the columns of v are the
// eigenvectors.  At most 32 sweeps (quadratic convergence needs < 10).
__device__ void jacobi3(double a[3][3], double v[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (!(off > 1e-32 * dia)) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const double apq = a[p][q];
      if (apq == 0.0) continue;
      const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = 0.0;
      const int r = 3 - p - q;
      const double arp = a[r][p], arq = a[r][q];
      a[r][p] = a[p][r] = c * arp - s * arq;
      a[r][q] = a[q][r] = s * arp + c * arq;
      for (int k = 0; k < 3; ++k) {
        const double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

// F = R U with U = (F^T F)^(1/2) symmetric positive definite
__device__ void polar3(const double F[3][3], double R[3][3], double U[3][3]) {
  double C[3][3], V[3][3], Ui[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  jacobi3(C, V);
  double s[3], si[3];
  for (int k = 0; k < 3; ++k) {
    s[k] = sqrt(fmax(C[k][k], 0.0));
    si[k] = 1.0 / s[k];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double u = 0.0, ui = 0.0;
      for (int k = 0; k < 3; ++k) {
        u += V[i][k] * s[k] * V[j][k];
        ui += V[i][k] * si[k] * V[j][k];
      }
      U[i][j] = u;
      Ui[i][j] = ui;
    }
  mul3(F, Ui, R);
}

// column p of the paper's probing-direction matrix [T], as a symmetric tensor
__device__ __forceinline__ void probe_direction(int p, double T[3][3]) {
  // [T] = 1/2 [[1,0,0,0,r,r],[0,1,0,r,0,r],[0,0,1,r,r,0],[0,0,0,2,0,0],[0,0,0,0,2,0],[0,0,0,0,0,2]], r = sqrt2
  const double r2 = 1.4142135623730951;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (p < 3) {
    v[p] = 0.5;
  } else {
    v[p] = 1.0;
    for (int I = 0; I < 3; ++I) v[I] = (I == p - 3) ? 0.0 : 0.5 * r2;
  }
  for (int I = 0; I < 6; ++I) {
    int i, j;
    mandel_pair(I, i, j);
    T[i][j] = T[j][i] = v[I] / mandel_w(I);
  }
}

__device__ __forceinline__ void load3(const double* p, double a[3][3]) {
  for (int k = 0; k < 9; ++k) a[k / 3][k % 3] = p[k];
}

// F_p = R (U + h T_p)
__device__ void probe_F(const double R[3][3], const double U[3][3], int p, double h, double Fp[3][3]) {
  double T[3][3], W[3][3];
  probe_direction(p, T);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W[i][j] = U[i][j] + h * T[i][j];
  mul3(R, W, Fp);
}

// Pi = J F^-1 sigma F^-T, Mandel form
__device__ void pk2_mandel(const double F[3][3], const double* sigma, double out[6]) {
  double Fi[3][3], S[3][3];
  const double J = inv3(F, Fi);
  load3(sigma, S);
  for (int I = 0; I < 6; ++I) {
    int i, j;
    mandel_pair(I, i, j);
    double acc = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) acc += Fi[i][k] * S[k][l] * Fi[j][l];
    out[I] = mandel_w(I) * J * acc;
  }
}

__global__ void mandel_make_F(const double* __restrict__ F, double* __restrict__ Fp, int64_t n, double h) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    double f[3][3], R[3][3], U[3][3], g[3][3];
    load3(F + 9 * r, f);
    polar3(f, R, U);
    for (int p = 0; p < N_MANDEL; ++p) {
      probe_F(R, U, p, h, g);
      for (int k = 0; k < 9; ++k) Fp[9 * (p * n + r) + k] = g[k / 3][k % 3];
    }
  }
}

// sigma: base stress (9 n); Sd: probe stresses (9 per slot, slot p*n + r);
// C: 36 per RVE, Mandel [I][J] row-major
__global__ void mandel_finish(const double* __restrict__ F, const double* __restrict__ sigma,
                              const double* __restrict__ Sd, const int32_t* __restrict__ Std, int64_t n, double h,
                              double* __restrict__ C, int32_t* __restrict__ status) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    double f[3][3], R[3][3], U[3][3], g[3][3];
    load3(F + 9 * r, f);
    polar3(f, R, U);
    double S0[6], P[6][6];
    pk2_mandel(f, sigma + 9 * r, S0);
    for (int p = 0; p < N_MANDEL; ++p) {
      probe_F(R, U, p, h, g);
      double Sp[6];
      pk2_mandel(g, Sd + 9 * (p * n + r), Sp);
      for (int I = 0; I < 6; ++I) P[I][p] = (Sp[I] - S0[I]) / h;
    }
    // [M] from M_klpq = (d_kq U_pl + d_lq U_pk + d_kp U_ql + d_lp U_qk) / 4, then [M][T]
    double M[6][6], MT[6][6], Tm[6][6];
    for (int I = 0; I < 6; ++I) {
      int k, l;
      mandel_pair(I, k, l);
      for (int J = 0; J < 6; ++J) {
        int p, q;
        mandel_pair(J, p, q);
        const double m = 0.25 * ((k == q ? U[p][l] : 0.0) + (l == q ? U[p][k] : 0.0) + (k == p ? U[q][l] : 0.0) +
                                 (l == p ? U[q][k] : 0.0));
        M[I][J] = mandel_w(I) * mandel_w(J) * m;
      }
    }
    for (int p = 0; p < 6; ++p) {
      double T[3][3];
      probe_direction(p, T);
      for (int I = 0; I < 6; ++I) {
        int i, j;
        mandel_pair(I, i, j);
        Tm[I][p] = mandel_w(I) * T[i][j];
      }
    }
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        double acc = 0.0;
        for (int K = 0; K < 6; ++K) acc += M[I][K] * Tm[K][J];
        MT[I][J] = acc;
      }
    // [A][M T] = [P]  <=>  (M T)^T [A]^T = [P]^T: Gaussian elimination with
    // partial pivoting on G = (M T)^T, right-hand sides Y = [P]^T
    double G[6][6], Y[6][6];
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        G[I][J] = MT[J][I];
        Y[I][J] = P[J][I];
      }
    bool singular = false;
    for (int c = 0; c < 6; ++c) {
      int piv = c;
      for (int i = c + 1; i < 6; ++i)
        if (fabs(G[i][c]) > fabs(G[piv][c])) piv = i;
      if (!(fabs(G[piv][c]) > 0.0)) {
        singular = true;
        break;
      }
      if (piv != c)
        for (int j = 0; j < 6; ++j) {
          double t = G[c][j];
          G[c][j] = G[piv][j];
          G[piv][j] = t;
          t = Y[c][j];
          Y[c][j] = Y[piv][j];
          Y[piv][j] = t;
        }
      for (int i = c + 1; i < 6; ++i) {
        const double m = G[i][c] / G[c][c];
        for (int j = c; j < 6; ++j) G[i][j] -= m * G[c][j];
        for (int j = 0; j < 6; ++j) Y[i][j] -= m * Y[c][j];
      }
    }
    double At[6][6];  // [A]^T
    for (int j = 0; j < 6; ++j)
      for (int i = 5; i >= 0; --i) {
        double acc = Y[i][j];
        for (int k = i + 1; k < 6; ++k) acc -= G[i][k] * At[k][j];
        At[i][j] = singular ? 0.0 : acc / G[i][i];
      }
    // [Q]: Mandel matrix of a -> F a F^T;  [C] = J^-1 [Q][A][Q]^T
    double Q[6][6], QA[6][6];
    for (int I = 0; I < 6; ++I) {
      int i, j;
      mandel_pair(I, i, j);
      for (int J = 0; J < 6; ++J) {
        int k, l;
        mandel_pair(J, k, l);
        Q[I][J] = (k == l) ? mandel_w(I) * f[i][k] * f[j][k]
                           : mandel_w(I) * (f[i][k] * f[j][l] + f[i][l] * f[j][k]) / mandel_w(J);
      }
    }
    const double Jinv = 1.0 / det3(f);
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        double acc = 0.0;
        for (int K = 0; K < 6; ++K) acc += Q[I][K] * At[J][K];  // [A]_KJ = At[J][K]
        QA[I][J] = acc;
      }
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        double acc = 0.0;
        for (int K = 0; K < 6; ++K) acc += QA[I][K] * Q[J][K];
        C[36 * r + 6 * I + J] = Jinv * acc;
      }
    if (status) {
      int w = status[r];
      for (int p = 0; p < N_MANDEL; ++p) {
        const int sp = Std[p * n + r];
        w = max(w, sp == RVE_STATUS_EMPTY ? 0 : sp);
      }
      if (singular && w == RVE_STATUS_CONVERGED) w = RVE_STATUS_NONFINITE;
      status[r] = w;
    }
  }
}

}  // namespace rvegpu
