"""Microstructure outputs (oracle side): the RVE orientation tensor and the
degree of alignment.

Test infrastructure only (see the package header).

Sec. 4 sends the RVE's orientation tensor to the macroscale with each
converged step; Sec. 5 measures alignment by the second Legendre
polynomial P2 = <3 cos^2(theta) - 1> / 2, theta the angle between a fiber's
direction and a reference direction, <.> the average over the fibers of the
RVE.  Reading: the orientation tensor is Omega = <n (x) n> over the same
fibers, n = (x_j - x_i)/|x_j - x_i| at the current positions, so that
<cos^2 theta> = a . Omega . a and P2(a) = (3 a . Omega . a - 1)/2 for a unit
reference direction a; the fibers are those kept after pruning (dangling
fibers carry no load and have no defined equilibrium direction).
"""
from __future__ import annotations

import math

import numpy as np

from .network import prune


def orientation_tensor(x, conn, is_boundary):
    """Omega (3x3) of one RVE at node positions x (N,3); zeros if no fiber is kept."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    conn = np.asarray(conn, np.int64).reshape(-1, 2)
    kept, _ = prune(conn, np.asarray(is_boundary))
    c = conn[kept]
    if c.shape[0] == 0:
        return np.zeros((3, 3))
    d = x[c[:, 1]] - x[c[:, 0]]
    n = d / np.linalg.norm(d, axis=1)[:, None]
    om = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            om[a, b] = math.fsum(n[:, a] * n[:, b]) / c.shape[0]
    return om


def p2(omega, a):
    """Degree of alignment along direction a from the orientation tensor."""
    a = np.asarray(a, np.float64)
    a = a / np.linalg.norm(a)
    return 0.5 * (3.0 * a @ np.asarray(omega) @ a - 1.0)
