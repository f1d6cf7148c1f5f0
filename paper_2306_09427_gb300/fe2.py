"""Macroscale FE² driver on the host (the paper's Algorithm 1, Sec. 3.1).

A box of trilinear hexahedra with 2x2x2 Gauss points; one RVE per Gauss
point supplies the constitutive response: the batched solver returns the
Cauchy stress sigma and its derivative dsigma/dF for every Gauss point at
once (18 perturbed solves, warm-started), and every RVE keeps its converged
state on the device between Newton iterations and load steps.

The paper's macroscale is updated-Lagrangian with the spatial tangent C
pushed forward from dS/dE (Eq. stiffness-push-forward).  This driver uses
the equivalent total-Lagrangian statement of the same equilibrium:
    R_aI = sum_gp w |J0| P_iJ dN_a/dX_J,  P = J sigma F^-T,
    K = sum_gp w |J0| dN_a/dX_J (dP_iJ/dF_kL) dN_b/dX_L,
with dP/dF from dsigma/dF (chain rule through J and F^-T).  Boundary
conditions (uniaxial extension along z): u_z = 0 on z = 0, u_z = lambda L_z
on z = L_z, u_x = u_y = 0 at the origin node and u_y = 0 at (L_x, 0, 0);
the lateral faces are traction free.

    python -m paper_2306_09427_gb300.fe2 --nx 10 --ny 10 --nz 40 --steps 8 --strain 0.2
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import rvegen

from ._lib import RVE_PREC_MIXED, RveBatch

_GP = np.array([-1.0, 1.0]) / np.sqrt(3.0)


class HexBox:
    """nx x ny x nz trilinear hexahedra on [0,Lx]x[0,Ly]x[0,Lz]."""

    def __init__(self, nx, ny, nz, Lx=1.0, Ly=1.0, Lz=4.0):
        self.n = (nx, ny, nz)
        h = np.array([Lx / nx, Ly / ny, Lz / nz])
        self.L = np.array([Lx, Ly, Lz])
        ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
        self.X = np.stack([ii.ravel() * h[0], jj.ravel() * h[1], kk.ravel() * h[2]], 1)
        nid = lambda i, j, k: (i * (ny + 1) + j) * (nz + 1) + k
        ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
        corners = [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
        self.conn = np.stack([nid(ei + a, ej + b, ek + c) for (a, b, c) in corners], 1)
        self.nodes_ref = np.array(corners, np.float64) * 2.0 - 1.0  # reference corner coords
        # shape-function gradients dN_a/dX_J at the 8 Gauss points (same for every element)
        gps = np.array([(x, y, z) for x in _GP for y in _GP for z in _GP])
        G = np.zeros((8, 8, 3))
        for g, (xi, eta, zeta) in enumerate(gps):
            for a, (sa, ta, ua) in enumerate(self.nodes_ref):
                dxi = np.array([sa * (1 + ta * eta) * (1 + ua * zeta), ta * (1 + sa * xi) * (1 + ua * zeta),
                                ua * (1 + sa * xi) * (1 + ta * eta)]) / 8.0
                G[g, a] = dxi * 2.0 / h  # d(xi)/dX = 2/h
        self.G = G
        self.vol = np.prod(h) / 8.0  # |J0| x weight (1) per Gauss point
        self.ne = self.conn.shape[0]
        self.nn = self.X.shape[0]

    def deformation_gradients(self, u):
        ue = u[self.conn]  # (ne, 8, 3)
        return np.eye(3)[None, None] + np.einsum("eai,gaJ->egiJ", ue, self.G)  # (ne, 8, 3, 3)


def first_pk_and_tangent(F, sigma, dsdF):
    """P = J sigma F^-T and A = dP/dF from sigma and dsigma/dF ([ij][kl] layout)."""
    J = np.linalg.det(F)
    Fi = np.linalg.inv(F)
    P = J[:, None, None] * np.einsum("nik,nJk->niJ", sigma, Fi)
    D = dsdF.reshape(-1, 3, 3, 3, 3)  # d sigma_ik / d F_mN
    A = (J[:, None, None, None, None] * (np.einsum("nNm,nik,nJk->niJmN", Fi, sigma, Fi, optimize=True)
                                          + np.einsum("nikmN,nJk->niJmN", D, Fi)
                                          - np.einsum("nik,nJm,nNk->niJmN", sigma, Fi, Fi, optimize=True)))
    return P, A


class RveMaterial:
    """One RVE per Gauss point on the GPU: sigma and dsigma/dF by rve_tangent."""

    def __init__(self, n_points, rve_side=8, p=0.6, precision=RVE_PREC_MIXED, tol=1e-7, seed_config=4, device=0):
        nets = [rvegen.grid_network(rve_side, p, rvegen.Stream(rvegen.rve_seed(seed_config, r)))
                for r in range(n_points)]
        self.batch = RveBatch(rvegen.pack(nets), device=device, precision=precision, tol=tol, warm_start=1)
        self.n = n_points

    def tangent(self, F):
        import torch
        Fd = torch.tensor(F.reshape(-1, 9), dtype=torch.float64, device=f"cuda:{self.batch.device}")
        s, D, st = self.batch.tangent(Fd)
        torch.cuda.synchronize()
        return s.cpu().numpy().reshape(-1, 3, 3), D.cpu().numpy(), st.cpu().numpy()


class FE2:
    def __init__(self, box: HexBox, material):
        self.box = box
        self.material = material
        self.n_rve = box.ne * 8
        nd = 3 * box.nn
        X = box.X
        fixed = {}
        for n in np.nonzero(np.isclose(X[:, 2], 0.0))[0]:
            fixed[3 * n + 2] = 0.0
        self.top = np.nonzero(np.isclose(X[:, 2], box.L[2]))[0]
        o = int(np.nonzero(np.all(np.isclose(X, 0.0), axis=1))[0][0])
        xa = int(np.nonzero(np.isclose(X[:, 0], box.L[0]) & np.isclose(X[:, 1], 0) & np.isclose(X[:, 2], 0))[0][0])
        fixed[3 * o] = fixed[3 * o + 1] = 0.0
        fixed[3 * xa + 1] = 0.0
        self.base_fixed = fixed
        self.nd = nd
        self.u = np.zeros((box.nn, 3))
        # element DOF indices for assembly
        edof = (3 * box.conn[:, :, None] + np.arange(3)[None, None]).reshape(box.ne, 24)
        self.rows = np.repeat(edof, 24, axis=1).ravel()
        self.cols = np.tile(edof, (1, 24)).ravel()
        self.edof = edof

    def constitutive(self, F):
        return self.material.tangent(F)

    def residual_and_tangent(self, u):
        box = self.box
        F = box.deformation_gradients(u)
        sigma, D, st = self.constitutive(F.reshape(-1, 3, 3))
        P, A = first_pk_and_tangent(F.reshape(-1, 3, 3), sigma, D)
        P = P.reshape(box.ne, 8, 3, 3)
        A = A.reshape(box.ne, 8, 3, 3, 3, 3)
        R = np.zeros((box.nn, 3))
        Re = box.vol * np.einsum("egiJ,gaJ->eai", P, box.G)
        np.add.at(R, box.conn, Re)
        Ke = box.vol * np.einsum("gaJ,egiJkL,gbL->eaibk", box.G, A, box.G, optimize=True).reshape(box.ne, 24, 24)
        K = sp.coo_matrix((Ke.ravel(), (self.rows, self.cols)), shape=(self.nd, self.nd)).tocsr()
        return R.ravel(), K, sigma, st

    def run(self, strain=0.2, steps=8, newton_tol=1e-6, max_newton=12, log=print):
        box = self.box
        history = []
        for step in range(1, steps + 1):
            lam = strain * step / steps
            fixed = dict(self.base_fixed)
            for n in self.top:
                fixed[3 * n + 2] = lam * box.L[2]
            fdofs = np.array(sorted(fixed))
            fvals = np.array([fixed[d] for d in fdofs])
            free = np.setdiff1d(np.arange(self.nd), fdofs)
            # predictor: the previous field scaled by the load ratio (the affine
            # extension on the first step), so the increment is not concentrated
            # in the top layer of elements
            if step == 1:
                u = np.zeros((box.nn, 3))
                u[:, 2] = lam * box.X[:, 2]
                u = u.ravel()
            else:
                u = (self.u * (lam / (strain * (step - 1) / steps))).ravel()
            u[fdofs] = fvals
            norms = []
            for it in range(max_newton):
                t0 = time.perf_counter()
                R, K, sigma, st = self.residual_and_tangent(u.reshape(-1, 3))
                t_micro = time.perf_counter() - t0
                rf = R[free]
                ref = max(np.linalg.norm(R[fdofs]), 1e-300)
                norms.append(float(np.linalg.norm(rf) / ref))
                log(f"step {step} it {it}: |R_free|/|R_fixed| = {norms[-1]:.2e}  micro {t_micro:.2f}s  "
                    f"status!=0: {int((st != 0).sum())}")
                if norms[-1] <= newton_tol:
                    break
                du = sla.spsolve(K[free][:, free].tocsc(), -rf)
                u[free] += du
            self.u = u.reshape(-1, 3)
            reaction = float(R[3 * self.top + 2].sum())
            history.append(dict(step=step, strain=lam, newton=norms, reaction_z=reaction,
                                sigma_zz_mean=float(sigma[:, 2, 2].mean())))
        return history


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=10)
    ap.add_argument("--ny", type=int, default=10)
    ap.add_argument("--nz", type=int, default=40)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--strain", type=float, default=0.2)
    ap.add_argument("--rve-side", type=int, default=8)
    a = ap.parse_args()
    box = HexBox(a.nx, a.ny, a.nz, 1.0, 1.0, 4.0)
    t0 = time.perf_counter()
    fe = FE2(box, RveMaterial(box.ne * 8, rve_side=a.rve_side))
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = fe.run(strain=a.strain, steps=a.steps)
    print(json.dumps(dict(elements=box.ne, rves=fe.n_rve, setup_s=t_setup, run_s=time.perf_counter() - t0,
                          history=hist)))


if __name__ == "__main__":
    main()
