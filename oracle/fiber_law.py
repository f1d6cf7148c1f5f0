"""Fiber constitutive law of the truss network (oracle side).

The paper only says the microscale is a large-displacement truss model of
collagen fibers (Sec. 3.2) whose elasticity alone fixes the static answer.
The law used throughout is the exponential one of the workload
description: with the Green-Lagrange fiber strain
    eps_G = (l^2 / L0^2 - 1) / 2,
the current axial force is
    N = (EA / B) (exp(B eps_G) - 1)        (B > 0),   N = EA eps_G (B = 0),
evaluated with expm1 so small strains keep full relative precision.
"""
from __future__ import annotations

import numpy as np

_GL_T, _GL_W = np.polynomial.legendre.leggauss(16)


def green_strain(l, L0):
    """eps_G = (l^2/L0^2 - 1)/2."""
    return 0.5 * (np.square(l) / np.square(L0) - 1.0)


def axial_force(eps, EA, B):
    """N(eps_G) = (EA/B) expm1(B eps_G); the B -> 0 limit EA*eps_G."""
    eps = np.asarray(eps, dtype=np.float64)
    EA = np.broadcast_to(np.asarray(EA, np.float64), eps.shape)
    B = np.broadcast_to(np.asarray(B, np.float64), eps.shape)
    pos = B > 0
    safeB = np.where(pos, B, 1.0)
    return np.where(pos, EA * np.expm1(safeB * eps) / safeB, EA * eps)


def axial_stiffness(l, L0, EA, B):
    """dN/dl = EA exp(B eps_G) l / L0^2 (chain rule through eps_G)."""
    eps = green_strain(l, L0)
    return EA * np.exp(np.asarray(B) * eps) * l / np.square(L0)


def fiber_energy(l, L0, EA, B):
    """Stored energy w(l) = integral of N from L0 to l (16-point Gauss-Legendre).

    The exponential law has no elementary antiderivative in l; the
    integrand is smooth, so 16 nodes give the integral to rounding for the
    strains met here.  Used only as the line-search merit of the Newton
    solve and in its energy/force consistency pin.
    """
    l = np.asarray(l, np.float64)
    L0 = np.asarray(L0, np.float64)
    mid = 0.5 * (l + L0)
    half = 0.5 * (l - L0)
    lk = mid[..., None] + half[..., None] * _GL_T
    Nk = axial_force(green_strain(lk, L0[..., None]), np.asarray(EA)[..., None], np.asarray(B)[..., None])
    return half * (Nk @ _GL_W)
