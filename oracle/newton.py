"""Load-incremented Newton-Raphson equilibrium solve (oracle side).

Sec. 3.2 names two microscale solvers: an implicit updated-Lagrangian
Newton method and dynamic relaxation (Algorithm 2).  Both target the same
static state; the oracle takes the implicit route in plain double
precision:

  1. split F = R U (polar decomposition) and walk the load path
     F_k = R_k U_k, k = 1..K (intermediate increments converged to 1e-6
     only), with R_k the rotation by k/K of R's angle
     about its axis and U_k = I + (k/K)(U - I);
  2. at each increment pin boundary nodes to x = F_k X (Eq. affine-bc) and
     predict free nodes as F_k X + h, h the previous fluctuation
     (Eq. micro_coords);
  3. Newton on f_free(x) = 0 with a sparse direct solver (SuperLU,
     symmetric mode, diagonal pivots): the tangent K_ff is shifted by the
     smallest mu in {0, 1e-12, 1e-11, ...} x mean diag K_ff that makes
     K_ff + mu I positive definite (Levenberg-Marquardt-style regularisation
     of floppy and compressed directions), so the step descends the stored
     energy W; a backtracking line search halves the step until W drops by
     the Armijo fraction 1e-4 of its predicted first-order decrease (once
     that decrease reaches the rounding level of W, until ||f|| drops);
  4. stop at ||f_free||_2 <= max(tol * R_aff, 1e-16 sum EA) (R_aff from
     ``network.reference_force_scale``); after the last increment check
     that the state is an energy minimum, not a saddle: K_ff + s I with the
     fixed shift s = 1e-9 x mean diag K_ff must factor with no negative pivot
     (inertia by Sylvester's law); the lowest eigenvalue of K_ff can be
     recorded beside the verdict.  At a saddle, push along the
     lowest-curvature direction and re-solve, at most three times.  The
     verdict is taken for solves converged to a relative residual of 1e-8 or
     below (by default; it needs the state converged well below the shift);
  5. return sigma from the fiber virial and, as a self-check, from the
     boundary reactions (the two forms of the average after Eq. hill-mandel).

The default is one increment (K = 1): the microscale solve of Algorithm 2
starts from the affine state of the full F (h = 0, or a warm start), and a
sub-isostatic network can hold several stable equilibria with different
stresses; starting the energy descent from the same state as the method is
the reading that makes the oracle's answer the method's answer.  K > 1
follows the quasi-static load path instead (used in tests where the
minimum is unique).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as sla
from scipy.spatial.transform import Rotation

from .network import (boundary_virial_stress, convergence_threshold, fiber_virial_stress,
                      internal_forces, prune, reference_force_scale, stiffness_free, total_energy)


@dataclass
class Solution:
    sigma: np.ndarray              # (3,3) fiber-virial Cauchy stress
    sigma_boundary: np.ndarray     # (3,3) boundary-reaction form (self-check)
    x: np.ndarray                  # (N,3) positions; pruned nodes left at F X
    residual: float                # ||f_free||_2 at return
    R_ref: float
    converged: bool
    newton_iters: int
    stable: bool | None            # K_ff positive semi-definite at x
    saddle_escapes: int
    kept: np.ndarray               # fiber mask after pruning
    free: np.ndarray               # free-node mask after pruning
    info: dict = field(default_factory=dict)


def _factor(K, mu):
    n = K.shape[0]
    A = (K + mu * sp.identity(n, format="csc")).tocsc()
    try:
        lu = sla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                      options=dict(SymmetricMode=True))
    except RuntimeError:  # exactly singular: not positive definite
        return None, False, -1
    # with symmetric (diagonal) pivots U = D L^T, so the signs of diag(U) give
    # the inertia (Sylvester); after an off-diagonal pivot they do not (-1)
    symmetric_pivots = np.array_equal(lu.perm_r, lu.perm_c)
    neg = int((lu.U.diagonal() <= 0).sum()) if symmetric_pivots else -1
    return lu, symmetric_pivots and neg == 0, neg


def _load_path(F, increments):
    R, U = scipy.linalg.polar(F, side="right")
    rv = Rotation.from_matrix(R).as_rotvec()
    out = []
    for k in range(1, increments + 1):
        t = k / increments
        Rk = Rotation.from_rotvec(t * rv).as_matrix()
        Uk = np.eye(3) + t * (U - np.eye(3))
        out.append(Rk @ Uk)
    out[-1] = np.array(F, dtype=np.float64)  # the last increment is F itself
    return out


class _Problem:
    def __init__(self, X, conn, L0, EA, B, free):
        self.X, self.conn, self.L0, self.EA, self.B = X, conn, L0, EA, B
        self.free_ids = np.nonzero(free)[0]
        self.free_index = -np.ones(X.shape[0], np.int64)
        self.free_index[self.free_ids] = np.arange(self.free_ids.size)

    def place(self, x, xf):
        y = x.copy()
        y[self.free_ids] = xf.reshape(-1, 3)
        return y

    def residual(self, x):
        return internal_forces(x, self.conn, self.L0, self.EA, self.B)[self.free_ids].ravel()

    def energy(self, x):
        return total_energy(x, self.conn, self.L0, self.EA, self.B)

    def tangent(self, x):
        return stiffness_free(x, self.conn, self.L0, self.EA, self.B, self.free_index, self.free_ids.size)


def _newton(pb, x, tol_abs, max_iter):
    """Energy-descending Newton on the free DOFs; returns (x, iters, ||r||, ok).

    Each iteration factors K + mu I with the smallest mu of the sequence
    0, 1e-12 d, 1e-11 d, ... (d = mean diag K) that gives a positive definite
    factor (the search starts a decade below the previous iteration's shift),
    solves (K + mu I) p = r (r = -grad W), and backtracks along p:
    the first step length a in 1, 1/2, 1/4, ... with
    W(x + a p) <= W(x) - 1e-4 a (r . p) is taken; when a (r . p) is at the
    rounding level of W, a step that lowers ||r|| is taken instead.
    """
    it = 0
    r = pb.residual(x)
    rn = float(np.linalg.norm(r))
    W0 = pb.energy(x)
    mu_rel = 0.0  # last shift that worked, relative to mean diag K (the search starts a decade below it)
    while rn > tol_abs and it < max_iter:
        it += 1
        K = pb.tangent(x)
        dscale = max(float(np.abs(K.diagonal()).mean()), 1e-300)
        mu = 0.1 * mu_rel * dscale if mu_rel >= 1e-11 else 0.0
        for _ in range(40):
            lu, pd, _neg = _factor(K, mu)
            if pd:
                break
            mu = 1e-12 * dscale if mu == 0.0 else 10.0 * mu
        else:
            return x, it, rn, False
        mu_rel = mu / dscale
        p = lu.solve(r)
        slope = float(r @ p)  # predicted first-order decrease of W per unit step
        a = 1.0
        for _ in range(60):
            xt = pb.place(x, x[pb.free_ids].ravel() + a * p)
            with np.errstate(over="ignore", invalid="ignore"):  # a wild trial step is rejected below
                Wt = pb.energy(xt)
                rt = pb.residual(xt)
                rtn = float(np.linalg.norm(rt))
            if np.isfinite(rtn) and np.isfinite(Wt):
                if a * slope > 1e-12 * max(abs(W0), 1e-300):
                    if Wt <= W0 - 1e-4 * a * slope:
                        break
                elif rtn < rn:
                    break
            a *= 0.5
        else:
            return x, it, rn, False
        x, r, rn, W0 = xt, rt, rtn, Wt
    return x, it, rn, rn <= tol_abs


STAB_SHIFT = 1e-9  # fixed stability shift, relative to mean diag K_ff
STAB_TOL = 1e-8    # solves at or below this relative residual assess stability by default


def lowest_eigenvalue(K):
    """Lowest eigenvalue of the symmetric sparse K (dense up to 3000 DOF,
    else a bounded Lanczos search; None if it does not converge)."""
    n = K.shape[0]
    if n == 0:
        return None
    if n <= 3000:
        return float(np.linalg.eigvalsh(K.toarray())[0])
    try:
        return float(sla.eigsh(K, k=1, which="SA", tol=1e-8, maxiter=2000, return_eigenvectors=False)[0])
    except sla.ArpackNoConvergence:
        return None


def stability(pb, x, with_lambda=True):
    """(stable, lambda_min, negative pivots) of the free-DOF tangent at x
    (lambda_min None unless with_lambda).

    Stable means K_ff + s I, s = STAB_SHIFT * mean diag K_ff, has no negative
    pivot in its symmetric factorisation, i.e. (Sylvester's law of inertia)
    no eigenvalue of K_ff below -s: a local minimum of the stored energy up
    to that fixed tolerance, which does not depend on the residual."""
    K = pb.tangent(x)
    dscale = max(float(np.abs(K.diagonal()).mean()), 1e-300)
    _, pd, neg = _factor(K, STAB_SHIFT * dscale)
    return bool(pd), (lowest_eigenvalue(K) if with_lambda else None), int(neg)


def _lowest_mode(K):
    """A direction of lowest curvature for the saddle escape.  Exact for small
    K; otherwise a bounded Lanczos search: on sub-isostatic networks K has a
    large cluster of near-zero eigenvalues (floppy modes), no single lowest
    mode converges in reasonable time, and any direction of the cluster's
    best Ritz vector (or a fixed direction) serves the escape step."""
    n = K.shape[0]
    if n <= 3000:
        w, V = np.linalg.eigh(K.toarray())
        return w[0], V[:, 0]
    try:
        w, V = sla.eigsh(K, k=1, which="SA", tol=1e-6, maxiter=300)
        return w[0], V[:, 0]
    except sla.ArpackNoConvergence as err:  # take the best Ritz vector, else a fixed direction
        if err.eigenvectors is not None and err.eigenvectors.shape[1] > 0:
            return err.eigenvalues[0], err.eigenvectors[:, 0]
        v = np.cos(np.arange(n) * 0.7)
        return 0.0, v / np.linalg.norm(v)


def solve(X, conn, L0, EA, B, is_boundary, F, V0=1.0, tol=1e-12, increments=1,
          h0=None, max_newton=50000, check_stability=None, mid_tol=1e-6, record_lambda=False) -> Solution:
    """Equilibrium and Cauchy stress of one RVE under deformation gradient F.

    X (N,3), conn (E,2) RVE-local ids, L0/EA/B (E,), is_boundary (N,),
    F (3,3) with det F > 0.  ``h0`` (N,3) warm-starts the fluctuation
    h = x - F X; with a warm start the load is applied in one increment.
    ``check_stability`` None assesses stability (and escapes saddles) when
    tol <= STAB_TOL only: a fixed-shift inertia verdict needs a state converged
    well below the shift, and at looser tolerances ``stable`` stays None.
    ``record_lambda`` adds the lowest eigenvalue of K_ff at the returned state
    to ``info['lambda_min']`` (a dense or Lanczos eigensolve: a diagnostic).
    """
    X = np.asarray(X, np.float64).reshape(-1, 3)
    conn = np.asarray(conn).reshape(-1, 2).astype(np.int64)
    L0 = np.asarray(L0, np.float64)
    EA = np.broadcast_to(np.asarray(EA, np.float64), L0.shape).copy()
    B = np.broadcast_to(np.asarray(B, np.float64), L0.shape).copy()
    nb = np.asarray(is_boundary).astype(bool)
    F = np.asarray(F, np.float64).reshape(3, 3)
    detF = float(np.linalg.det(F))
    if not detF > 0:
        raise ValueError("det F must be positive")
    kept, free = prune(conn, nb)
    c, l0, ea, b = conn[kept], L0[kept], EA[kept], B[kept]
    pb = _Problem(X, c, l0, ea, b, free)
    R_ref = reference_force_scale(X, c, l0, ea, b, F)
    volume = detF * V0

    if h0 is None:
        path = _load_path(F, increments)
        h = np.zeros_like(X)
    else:
        path = [F]
        h = np.asarray(h0, np.float64).reshape(-1, 3).copy()
    total_it = 0
    ok = True
    x = X @ F.T
    for k, Fk in enumerate(path):
        last = k == len(path) - 1
        x = X @ Fk.T
        x[pb.free_ids] += h[pb.free_ids]
        tol_k = tol if last else max(tol, mid_tol)
        Rk = reference_force_scale(X, c, l0, ea, b, Fk)
        if pb.free_ids.size:
            x, it, rn, ok = _newton(pb, x, convergence_threshold(tol_k, Rk, ea), max_newton)
            total_it += it
        h = x - X @ Fk.T
    escapes = 0
    stable = None
    lam_min = None
    if check_stability is None:
        check_stability = tol <= STAB_TOL
    if pb.free_ids.size and check_stability:
        for escapes in range(4):
            stable, lam_min, _ = stability(pb, x, with_lambda=record_lambda)
            if stable or escapes == 3:
                break
            _, vec = _lowest_mode(pb.tangent(x))
            step = 1e-3 * float(np.mean(l0)) * vec / max(np.abs(vec).max(), 1e-300)
            x = pb.place(x, x[pb.free_ids].ravel() + step)
            x, it, rn, ok = _newton(pb, x, convergence_threshold(tol, R_ref, ea), max_newton)
            total_it += it
    r = pb.residual(x) if pb.free_ids.size else np.zeros(0)
    rn = float(np.linalg.norm(r))
    sigma = fiber_virial_stress(x, c, l0, ea, b, volume)
    sigma_b = boundary_virial_stress(x, c, l0, ea, b, nb, volume)
    return Solution(sigma=sigma, sigma_boundary=sigma_b, x=x, residual=rn, R_ref=R_ref,
                    converged=bool(rn <= convergence_threshold(tol, R_ref, ea)), newton_iters=total_it, stable=stable,
                    saddle_escapes=escapes, kept=kept, free=free,
                    info=dict(n_free=int(pb.free_ids.size), n_fibers=int(kept.sum()), lambda_min=lam_min,
                              energy=float(pb.energy(x))))


def solve_network(net, F, **kw) -> Solution:
    """``solve`` on an ``rvegen.Network``-like object (X, conn, L0, EA, B, is_boundary, V0)."""
    return solve(net.X, net.conn, net.L0, net.EA, net.B, net.is_boundary, F, V0=net.V0, **kw)
