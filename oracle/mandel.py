"""The paper's material tangent by 6 forward-difference solves (oracle side).

Test infrastructure only (see the package header).

Sec. 3.2 ("material stiffness"), in the paper's order and notation:

1. F = R U (polar decomposition).  The second Piola-Kirchhoff stress
   Pi = J F^-1 sigma F^-T does not change under a rotation of F, so it is a
   function of the stretch U alone, and dPi/dE = dPi/dU : dU/dE.
2. M_klpq = dE_kl/dU_pq = (d_kq U_pl + d_lq U_pk + d_kp U_ql + d_lp U_qk)/4
   for E = (U U - I)/2; both E and U are symmetric, so M has the minor
   symmetries and is written as a 6x6 Mandel matrix [M].
3. Six probing directions T_p, the columns of the Mandel matrix [T] the
   paper prints; forward differences
       P_ij,p = (Pi_ij(U + h T_p) - Pi_ij(U)) / h      (Eq. tensor_fd),
   six microscale solves, each warm-started from the solve at U.
4. [P] = [A][M][T], so solve ([M][T])^T [A]^T = [P]^T for [A] (the 6x6
   Mandel form of A_ijkl = dPi_ij/dE_kl).
5. Push forward, Eq. stiffness-push-forward:
       C_mnpq = J^-1 F_mi F_nj A_ijrs F_pr F_qs.

Mandel convention: index order (11, 22, 33, 23, 13, 12); a symmetric
second-order tensor a maps to (a11, a22, a33, sqrt2 a23, sqrt2 a13,
sqrt2 a12); a fourth-order tensor with minor symmetries maps to
[A]_IJ = w_I w_J A_(I)(J) with w = 1 for the normal and sqrt2 for the shear
indices, so that [A](a) is the Mandel image of A : a.
"""
from __future__ import annotations

import numpy as np

from .newton import solve

MANDEL_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
_W = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])


def to_mandel2(a):
    """Symmetric 3x3 -> Mandel 6-vector."""
    a = np.asarray(a, np.float64)
    return np.array([_W[I] * a[i, j] for I, (i, j) in enumerate(MANDEL_PAIRS)])


def from_mandel2(v):
    """Mandel 6-vector -> symmetric 3x3."""
    a = np.zeros((3, 3))
    for I, (i, j) in enumerate(MANDEL_PAIRS):
        a[i, j] = a[j, i] = v[I] / _W[I]
    return a


def to_mandel4(A):
    """3x3x3x3 tensor with minor symmetries -> 6x6 Mandel matrix."""
    A = np.asarray(A, np.float64)
    out = np.zeros((6, 6))
    for I, (i, j) in enumerate(MANDEL_PAIRS):
        for J, (k, l) in enumerate(MANDEL_PAIRS):
            out[I, J] = _W[I] * _W[J] * A[i, j, k, l]
    return out


def from_mandel4(m):
    """6x6 Mandel matrix -> 3x3x3x3 tensor with minor symmetries."""
    A = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(MANDEL_PAIRS):
        for J, (k, l) in enumerate(MANDEL_PAIRS):
            v = m[I, J] / (_W[I] * _W[J])
            for a, b in ((i, j), (j, i)):
                for c, d in ((k, l), (l, k)):
                    A[a, b, c, d] = v
    return A


def polar(F):
    """F = R U with U symmetric positive definite (eigen-decomposition of F^T F)."""
    F = np.asarray(F, np.float64).reshape(3, 3)
    lam, Q = np.linalg.eigh(F.T @ F)
    U = Q @ np.diag(np.sqrt(lam)) @ Q.T
    R = F @ np.linalg.inv(U)
    return R, U


def M_tensor(U):
    """dE/dU for E = (U U - I)/2 and symmetric U (step 2)."""
    d = np.eye(3)
    return 0.25 * (np.einsum("kq,pl->klpq", d, U) + np.einsum("lq,pk->klpq", d, U)
                   + np.einsum("kp,ql->klpq", d, U) + np.einsum("lp,qk->klpq", d, U))


def T_mandel():
    """The paper's probing directions: column p of this matrix is direction T_p (Mandel form)."""
    s = np.sqrt(2.0)
    return 0.5 * np.array([[1, 0, 0, 0, s, s],
                           [0, 1, 0, s, 0, s],
                           [0, 0, 1, s, s, 0],
                           [0, 0, 0, 2, 0, 0],
                           [0, 0, 0, 0, 2, 0],
                           [0, 0, 0, 0, 0, 2]], np.float64)


def pk2(F, sigma):
    """Pi = J F^-1 sigma F^-T."""
    F = np.asarray(F, np.float64).reshape(3, 3)
    Fi = np.linalg.inv(F)
    return np.linalg.det(F) * Fi @ np.asarray(sigma).reshape(3, 3) @ Fi.T


def push_forward(F, A):
    """C_mnpq = J^-1 F_mi F_nj A_ijrs F_pr F_qs (A as a 3x3x3x3 tensor)."""
    F = np.asarray(F, np.float64).reshape(3, 3)
    return np.einsum("mi,nj,ijrs,pr,qs->mnpq", F, F, A, F, F) / np.linalg.det(F)


def mandel_tangent(X, conn, L0, EA, B, is_boundary, F, V0=1.0, h=1e-6, tol=1e-12, h0_U=None):
    """Returns (sigma at F, [A] 6x6, [C] 6x6) by the paper's six-solve procedure.

    ``h0_U`` (N,3) optionally warm-starts the base solve at U (a fluctuation
    x - U X), so that the tangent is taken at a given equilibrium when the
    network has several stable ones."""
    F = np.asarray(F, np.float64).reshape(3, 3)
    Xr = np.asarray(X, np.float64).reshape(-1, 3)
    R, U = polar(F)                                                           # step 1
    base = solve(X, conn, L0, EA, B, is_boundary, U, V0=V0, tol=tol, h0=h0_U)
    if not base.stable:
        raise ValueError("base state is not a stable equilibrium")
    Pi0 = pk2(U, base.sigma)
    h0 = base.x - Xr @ U.T
    Tm = T_mandel()
    P = np.zeros((6, 6))
    for p in range(6):                                                        # step 3
        Up = U + h * from_mandel2(Tm[:, p])
        sp_ = solve(X, conn, L0, EA, B, is_boundary, Up, V0=V0, tol=tol, h0=h0, check_stability=False)
        P[:, p] = to_mandel2((pk2(Up, sp_.sigma) - Pi0) / h)
    MT = to_mandel4(M_tensor(U)) @ Tm                                         # step 2
    A = np.linalg.solve(MT.T, P.T).T                                          # step 4
    C = to_mandel4(push_forward(F, from_mandel4(A)))                         # step 5
    sigma = R @ base.sigma @ R.T  # sigma(F) = R sigma(U) R^T (objectivity)
    return sigma, A, C
