"""Write oracle-computed expected stresses for the GPU parity tests.

Every value stored here comes from ``oracle/`` (the FP64 Newton solve) on
inputs from ``rvegen``; nothing is read back from the CUDA path.  The paper
prints no numeric worked example, so these files are regression anchors of
the oracle, not values quoted from the paper.  Each row records the stress,
the relative residual, the stability verdict with the lowest eigenvalue of
the free-DOF tangent and the stored energy of the returned equilibrium.

Sets:
  single_6    the 6^3 RVE under F = I + 0.1 e1 (x) e1 (relative residual 1e-13);
  uniform_10  the first 64 RVEs of the 1024 x 10^3 uniform batch (1e-10);
  uneven      the first 64 RVEs of the 4096-RVE uneven batch (1e-10);
  fe2_8       16 RVEs of 8^3 (the FE2 strip's networks) stepped through the
              strip's uniaxial load path, F_k = diag(1 - 0.35 e_k, 1 - 0.35 e_k,
              1 + e_k), e_k = 0.025 k, k = 1..8, each step started from the
              previous step's equilibrium (the warm start the GPU keeps).

    python tests/golden/make_golden.py [--jobs N] [--only NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import rvegen  # noqa: E402
from oracle.newton import solve_network  # noqa: E402

FE2_STEPS = 8


def fe2_F(k: int) -> np.ndarray:
    """Macroscale deformation gradient of load step k (1-based) of the strip."""
    e = 0.025 * k
    return np.diag([1.0 - 0.35 * e, 1.0 - 0.35 * e, 1.0 + e])


def fe2_network(i: int):
    return rvegen.grid_network(8, 0.6, rvegen.Stream(rvegen.rve_seed(4, i)))


SETS = {
    # name: (builder, indices, tol)
    "single_6": (lambda i: rvegen.config_single(), [0], 1e-13),
    "uniform_10": (lambda i: rvegen.config_uniform(1, first=i), list(range(64)), 1e-10),
    "uneven": (lambda i: rvegen.config_uneven(1, first=i), list(range(64)), 1e-10),
    "fe2_8": (None, list(range(16)), 1e-10),
}


def _row(name, i, net, s, t, tol, **extra):
    d = dict(set=name, index=i, sigma=s.sigma.ravel().tolist(), sigma_boundary=s.sigma_boundary.ravel().tolist(),
             residual_rel=s.residual / max(s.R_ref, 1e-300), converged=s.converged, stable=s.stable,
             lambda_min=s.info["lambda_min"], energy=s.info["energy"], saddle_escapes=s.saddle_escapes,
             newton_iters=s.newton_iters, seconds=time.time() - t, n_free=s.info["n_free"],
             n_fibers=s.info["n_fibers"], side=int(net.meta["n"]), p=float(net.meta["p"]), tol=tol)
    d.update(extra)
    return d


def _job(args):
    name, i = args
    build, _, tol = SETS[name]
    if name == "fe2_8":
        net = fe2_network(i)
        rows, h = [], None
        for k in range(1, FE2_STEPS + 1):
            F = fe2_F(k)
            t = time.time()
            s = solve_network(net, F, tol=tol, h0=h, record_lambda=True)
            h = s.x - net.X @ F.T
            rows.append(_row(name, i, net, s, t, tol, step=k, F=F.ravel().tolist()))
        return rows
    nets, F = build(i)
    t = time.time()
    s = solve_network(nets[0], F[0], tol=tol, record_lambda=True)
    return [_row(name, i, nets[0], s, t, tol)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    names = a.only.split(",") if a.only else list(SETS)
    tasks = [(n, i) for n in names for i in SETS[n][1]]
    tasks.sort(key=lambda t: t[0] != "uneven")  # the slowest set first
    with get_context("spawn").Pool(a.jobs) as pool:
        res = [r for rows in pool.imap_unordered(_job, tasks, chunksize=1) for r in rows]
    for n in names:
        rows = sorted([r for r in res if r["set"] == n], key=lambda r: (r["index"], r.get("step", 0)))
        with open(os.path.join(HERE, f"oracle_{n}.json"), "w") as f:
            json.dump(dict(source="oracle.newton.solve_network (FP64 Newton, this repository)",
                           generator="rvegen", rows=rows), f, indent=1)
        print(n, "max seconds", max(r["seconds"] for r in rows), "all converged", all(r["converged"] for r in rows),
              "all stable", all(r["stable"] for r in rows))


if __name__ == "__main__":
    main()
