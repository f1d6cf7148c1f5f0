"""Finite-difference stress tangent (oracle side).

Sec. 3.2 obtains the material stiffness from finite-difference directional
derivatives of extra microscale solves because the dynamic-relaxation
solver has no Jacobian.  The quantity here is the central-difference
derivative of the Cauchy stress with respect to the deformation gradient,
    dsigma_ij/dF_kl = (sigma_ij(F + h E_kl) - sigma_ij(F - h E_kl)) / (2 h),
E_kl = e_k (x) e_l, nine directions, 18 perturbed solves, each warm-started
from the base equilibrium's fluctuation.  Output layout [ij][kl], i.e. a
9x9 matrix with row 3i+j and column 3k+l.
"""
from __future__ import annotations

import numpy as np

from .newton import solve


def dsigma_dF(X, conn, L0, EA, B, is_boundary, F, V0=1.0, h=1e-4, tol=1e-12, base=None):
    F = np.asarray(F, np.float64).reshape(3, 3)
    if base is None:
        base = solve(X, conn, L0, EA, B, is_boundary, F, V0=V0, tol=tol)
    Xr = np.asarray(X, np.float64).reshape(-1, 3)
    h0 = base.x - Xr @ F.T
    D = np.zeros((9, 9))
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = 1.0
            sp_ = solve(X, conn, L0, EA, B, is_boundary, F + h * E, V0=V0, tol=tol, h0=h0,
                        check_stability=False)
            sm_ = solve(X, conn, L0, EA, B, is_boundary, F - h * E, V0=V0, tol=tol, h0=h0,
                        check_stability=False)
            D[:, 3 * k + l] = ((sp_.sigma - sm_.sigma) / (2.0 * h)).ravel()
    return base.sigma, D
