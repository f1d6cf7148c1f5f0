"""Write oracle-computed expected stresses for the GPU parity tests.

Every value stored here comes from ``oracle/`` (the FP64 Newton solve) on
inputs from ``rvegen``; nothing is read back from the CUDA path.  The paper
prints no numeric worked example, so these files are regression anchors of
the oracle, not values quoted from the paper.

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

SETS = {
    # name: (builder, indices, tol)
    "single_6": (lambda i: rvegen.config_single(), [0], 1e-13),
    "uniform_10": (lambda i: rvegen.config_uniform(1, first=i), list(range(16)), 1e-12),
    "uneven": (lambda i: rvegen.config_uneven(1, first=i), list(range(24)), 1e-11),
}


def _job(args):
    name, i = args
    build, _, tol = SETS[name]
    nets, F = build(i)
    t = time.time()
    s = solve_network(nets[0], F[0], tol=tol)
    return dict(set=name, index=i, sigma=s.sigma.ravel().tolist(), sigma_boundary=s.sigma_boundary.ravel().tolist(),
                residual_rel=s.residual / max(s.R_ref, 1e-300), converged=s.converged, stable=s.stable,
                newton_iters=s.newton_iters, seconds=time.time() - t, n_free=s.info["n_free"],
                n_fibers=s.info["n_fibers"], side=int(nets[0].meta["n"]), p=float(nets[0].meta["p"]), tol=tol)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    names = [a.only] if a.only else list(SETS)
    tasks = [(n, i) for n in names for i in SETS[n][1]]
    with get_context("spawn").Pool(a.jobs) as pool:
        res = pool.map(_job, tasks, chunksize=1)
    for n in names:
        rows = sorted([r for r in res if r["set"] == n], key=lambda r: r["index"])
        with open(os.path.join(HERE, f"oracle_{n}.json"), "w") as f:
            json.dump(dict(source="oracle.newton.solve_network (FP64 Newton, this repository)",
                           generator="rvegen", rows=rows), f, indent=1)
        print(n, "max seconds", max(r["seconds"] for r in rows), "all converged", all(r["converged"] for r in rows))


if __name__ == "__main__":
    main()
