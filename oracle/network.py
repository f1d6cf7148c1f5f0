"""Network topology, forces, tangent and stress (oracle side)."""
from __future__ import annotations

import math
from collections import deque

import numpy as np
import scipy.sparse as sp

from .fiber_law import axial_force, axial_stiffness, fiber_energy, green_strain


def prune(conn, is_boundary):
    """Remove free nodes that carry no force at equilibrium.

    Returns (kept_fiber_mask, free_node_mask).  Two rules, both leaving the
    equilibrium stress unchanged:
      1. free nodes with no fiber path to a boundary node (floating
         clusters relax to their stress-free shape, so their fibers end with
         N = 0);
      2. free nodes of degree <= 1, repeatedly (a dangling fiber ends with
         N = 0 at equilibrium, and removing it may expose the next one).
    The free/fixed grouping follows Sec. 3.2 (vector operations act on free
    DOFs only; fixed positions feed the force computation).
    """
    conn = np.asarray(conn).reshape(-1, 2)
    nb = np.asarray(is_boundary).astype(bool)
    n = nb.shape[0]
    alive = np.ones(conn.shape[0], bool)
    node_ok = np.ones(n, bool)
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(conn):
        adj[a].append(e)
        adj[b].append(e)
    # rule 2: strip leaves (boundary nodes are never stripped)
    deg = np.zeros(n, np.int64)
    np.add.at(deg, conn[:, 0], 1)
    np.add.at(deg, conn[:, 1], 1)
    q = deque(i for i in range(n) if not nb[i] and deg[i] <= 1)
    while q:
        i = q.popleft()
        if not node_ok[i]:
            continue
        node_ok[i] = False
        for e in adj[i]:
            if alive[e]:
                alive[e] = False
                for j in conn[e]:
                    if j != i and node_ok[j]:
                        deg[j] -= 1
                        if not nb[j] and deg[j] <= 1:
                            q.append(j)
    # rule 1: keep only free nodes reachable from the boundary
    seen = np.zeros(n, bool)
    q = deque(i for i in range(n) if nb[i])
    for i in q:
        seen[i] = True
    while q:
        i = q.popleft()
        for e in adj[i]:
            if alive[e]:
                for j in conn[e]:
                    if not seen[j] and node_ok[j]:
                        seen[j] = True
                        q.append(j)
    node_ok &= seen | nb
    alive &= node_ok[conn[:, 0]] & node_ok[conn[:, 1]]
    free = node_ok & ~nb
    return alive, free


def fiber_kinematics(x, conn):
    d = x[conn[:, 1]] - x[conn[:, 0]]
    l = np.sqrt(np.einsum("ij,ij->i", d, d))
    return d, l


def internal_forces(x, conn, L0, EA, B):
    """Nodal internal force f_i = sum_e N_e (x_j - x_i)/l_e (getInternalForces, Algorithm 2).

    A fiber e = (i, j) in tension pulls i toward j and j toward i.
    Equilibrium of a free node is f_i = 0 (f_ext = 0, Sec. 3.2).
    """
    d, l = fiber_kinematics(x, conn)
    N = axial_force(green_strain(l, L0), EA, B)
    fe = (N / l)[:, None] * d
    f = np.zeros_like(x)
    np.add.at(f, conn[:, 0], fe)
    np.add.at(f, conn[:, 1], -fe)
    return f


def total_energy(x, conn, L0, EA, B):
    d, l = fiber_kinematics(x, conn)
    return math.fsum(fiber_energy(l, L0, EA, B))


def stiffness_free(x, conn, L0, EA, B, free_index, n_free):
    """K = -df/dx restricted to free DOFs, assembled from 3x3 fiber blocks.

    Per fiber S = (dN/dl) n n^T + (N/l)(I - n n^T); K_ii += S, K_jj += S,
    K_ij = K_ji -= S.  Material (axial) plus geometric part, the truss
    analogue of Eq. tangent-stiffness.
    """
    d, l = fiber_kinematics(x, conn)
    N = axial_force(green_strain(l, L0), EA, B)
    k = axial_stiffness(l, L0, EA, B)
    nvec = d / l[:, None]
    nn = nvec[:, :, None] * nvec[:, None, :]
    S = k[:, None, None] * nn + (N / l)[:, None, None] * (np.eye(3)[None] - nn)
    rows, cols, vals = [], [], []
    a = free_index[conn[:, 0]]
    b = free_index[conn[:, 1]]
    r3 = np.arange(3)
    RR, CC = np.meshgrid(r3, r3, indexing="ij")

    def put(ia, ib, sign, mask):
        m = np.nonzero(mask)[0]
        if m.size == 0:
            return
        rows.append((3 * ia[m][:, None, None] + RR[None]).ravel())
        cols.append((3 * ib[m][:, None, None] + CC[None]).ravel())
        vals.append((sign * S[m]).ravel())

    fa, fb = a >= 0, b >= 0
    put(a, a, 1.0, fa)
    put(b, b, 1.0, fb)
    put(a, b, -1.0, fa & fb)
    put(b, a, -1.0, fa & fb)
    n3 = 3 * n_free
    if not rows:
        return sp.csc_matrix((n3, n3))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n3, n3))
    return K.tocsc()


def fiber_virial_stress(x, conn, L0, EA, B, volume):
    """sigma = (1/v) sum_e N_e d_e (x) d_e / l_e  (fiber form of the volume average
    after Eq. hill-mandel), each component summed exactly rounded (math.fsum)."""
    d, l = fiber_kinematics(x, conn)
    N = axial_force(green_strain(l, L0), EA, B)
    terms = (N / l)[:, None, None] * d[:, :, None] * d[:, None, :]
    s = np.array([[math.fsum(terms[:, i, j]) for j in range(3)] for i in range(3)])
    return s / volume


def boundary_virial_stress(x, conn, L0, EA, B, is_boundary, volume):
    """sigma_b = (1/v) sum_b t_b (x) x_b with t_b = -f_b the reaction applied at
    boundary node b: the traction form of the volume average (after Eq.
    hill-mandel).  Equals the fiber virial when free nodes are in equilibrium."""
    f = internal_forces(x, conn, L0, EA, B)
    bidx = np.nonzero(np.asarray(is_boundary).astype(bool))[0]
    terms = (-f[bidx])[:, :, None] * x[bidx][:, None, :]
    s = np.array([[math.fsum(terms[:, i, j]) for j in range(3)] for i in range(3)])
    return s / volume


def reference_force_scale(X, conn, L0, EA, B, F):
    """R_aff = ||(N_e(a_e))_e||_2, the 2-norm of the fiber forces under the
    affine map x = F X (a_e the fiber's Green strain there).

    R_aff depends on F and the network only, never on the iterate or on a
    warm start.  Convergence (the residual test R < eps of Algorithm 2,
    made relative) is ||f_free||_2 <= convergence_threshold(tol, ...).
    """
    d = (X[conn[:, 1]] - X[conn[:, 0]]) @ np.asarray(F).T
    l = np.sqrt(np.einsum("ij,ij->i", d, d))
    N = axial_force(green_strain(l, L0), EA, B)
    return math.sqrt(math.fsum(N * N))


def convergence_threshold(tol, R_aff, EA):
    """max(tol * R_aff, 1e-16 * sum_e EA_e): the absolute floor sits at the
    rounding level of double-precision fiber forces, so a rigid rotation
    (R_aff ~ 0) is converged at the affine start."""
    return max(tol * R_aff, 1e-16 * math.fsum(np.asarray(EA, np.float64)))
