"""Throughput of the batched solve on the other workloads (one JSON line each).

    python -m paper_2306_09427_gb300.measure single    # one 6^3 RVE, F = I + 0.1 e1 (x) e1
    python -m paper_2306_09427_gb300.measure uneven    # 4096 RVEs, side 6..16, p 0.5..0.8
    python -m paper_2306_09427_gb300.measure tangent   # 32,000 8^3 RVEs, sigma + dsigma/dF, and the six-solve C
    python -m paper_2306_09427_gb300.measure orientation  # orientation tensors of 1024 x 10^3 RVEs (HBM-bound)
    python -m paper_2306_09427_gb300.measure streamed  # 152 RVEs of side 15-16 (streamed kernel variants)

Option --kernel node runs the node-centric kernels (clusters for RVEs too
large for one CTA) instead of the two-phase kernel.

Each line gives the batched mixed-precision path (one solve of the whole
batch, CUDA events on a created stream, warm-up excluded, median of the
timed repeats) and the plain FP64 per-RVE path on a subset of the same RVEs
at the same tolerance; the iteration counts show the work per solve.  The
uniform 1024 x 10^3 workload is bench.py's; the serving stream is
``paper_2306_09427_gb300.serve`` and the FE^2 strip ``paper_2306_09427_gb300.fe2``.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import rvegen

from ._lib import (RVE_KERNEL_AUTO, RVE_KERNEL_NODE, RVE_KERNEL_TWO_PHASE, RVE_PREC_BATCHED_F64, RVE_PREC_MIXED,
                   RVE_PREC_PLAIN_F64, RveBatch)


def _time_solves(b, Fd, reps, stream, tangent=False):
    import torch
    out = []
    for k in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if tangent == "mandel":
            res = b.tangent_mandel(Fd, stream=stream)
        else:
            res = b.tangent(Fd, stream=stream) if tangent else b.solve(Fd, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            out.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(out)), res


def _plain(pk_sub, Fs_sub, tol, device, damping_scale=1.0):
    import torch
    b = RveBatch(pk_sub, device=device, precision=RVE_PREC_PLAIN_F64, tol=tol, damping_scale=damping_scale)
    Fd = torch.tensor(Fs_sub.reshape(-1, 9), dtype=torch.float64, device=f"cuda:{device}")
    b.solve(Fd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, it, st = b.solve(Fd)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    b.close()
    return Fs_sub.shape[0] / dt, it.cpu().numpy()


def _orientation(b, Fd, stream, reps, res):
    """Time rve_orientation after a solve, L2 flushed before each launch;
    algorithmic bytes: per active fiber its reference chord (24 B) and packed
    endpoints (4 B), per boundary fiber its chord, per free node its state
    (24 B), per RVE F and Omega (144 B)."""
    import torch
    b.solve(Fd, stream=stream)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=Fd.device)
    ts = []
    for k in range(reps + 3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        om = b.orientation(Fd, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            ts.append(e0.elapsed_time(e1) / 1e3)
    nf, na, nb = b.sizes()
    bytes_alg = float(28 * na.sum() + 24 * nb.sum() + 24 * nf.sum() + 144 * b.n_rve)
    t = float(np.median(ts))
    res.update(orientation_s=t, algorithmic_bytes=bytes_alg, achieved_gbs=bytes_alg / t / 1e9,
               trace_max_dev=float((om.diagonal(dim1=1, dim2=2).sum(-1) - 1).abs().max()))
    b.close()
    return res


KERNELS = {"auto": RVE_KERNEL_AUTO, "two-phase": RVE_KERNEL_TWO_PHASE, "node": RVE_KERNEL_NODE}


def run(config: str, reps: int = 5, plain_subset: int = 32, tol: float = 3e-7, autotune: bool = True,
        device: int = 0, damping_scale: float = 1.0, kernel: str = "auto") -> dict:
    import torch
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream()
    if config == "single":
        nets, Fs = rvegen.config_single()
        tol_m, tol_d = 1e-8, 1e-8
    elif config == "uneven":
        nets, Fs = rvegen.config_uneven(4096)
        tol_m = tol_d = tol
    elif config == "streamed":
        # RVEs too large for one CTA's shared memory: fiber data and CSR stream from L2/HBM (MODE 1/2)
        nets, Fs = rvegen.config_uneven(152, side_lo=15, side_hi=16)
        tol_m = tol_d = tol
    elif config == "orientation":
        nets, Fs = rvegen.config_uniform(1024)
        tol_m = tol_d = tol
    elif config == "tangent":
        nets = [rvegen.grid_network(8, 0.6, rvegen.Stream(rvegen.rve_seed(4, r))) for r in range(32000)]
        Fs = np.stack([rvegen.random_F(rvegen.Stream(rvegen.rve_seed(4, 1 << 19 | r))) for r in range(32000)])
        tol_m = tol_d = tol
    else:
        raise ValueError(config)
    t0 = time.perf_counter()
    pk = rvegen.pack(nets)
    n = len(nets)
    prec = RVE_PREC_BATCHED_F64 if config == "single" else RVE_PREC_MIXED
    b = RveBatch(pk, device=device, precision=prec, tol=tol_m, graphs=1, warm_start=int(config == "tangent"),
                 damping_scale=damping_scale, kernel=KERNELS[kernel])
    t_create = time.perf_counter() - t0
    Fd = torch.tensor(Fs.reshape(-1, 9), dtype=torch.float64, device=f"cuda:{device}")
    res = {"config": config, "n_rve": n, "create_s": t_create, "precision": "f64 batched" if config == "single"
           else "mixed", "tol_rel_residual": tol_m, "damping_scale": damping_scale, "kernel": kernel}
    if config == "orientation":
        return _orientation(b, Fd, stream, reps, res)
    if config == "tangent":
        b.solve(Fd, stream=stream)  # base state to warm-start from, as inside a load step
        torch.cuda.synchronize()
        dt, (s, D, st) = _time_solves(b, Fd, reps, stream, tangent=True)
        st = st.cpu().numpy()
        res.update(tangent_s=dt, rve_tangents_per_s=n / dt, rve_solves_per_s=19 * n / dt,
                   converged_frac=float((st == 0).mean()))
        # the paper's six-solve tangent (7 solves per RVE) on the same batch
        dtm, (_, _, stm) = _time_solves(b, Fd, reps, stream, tangent="mandel")
        res.update(mandel_tangent_s=dtm, mandel_tangents_per_s=n / dtm,
                   mandel_converged_frac=float((stm.cpu().numpy() == 0).mean()))
    else:
        if autotune and config == "uneven":
            before, after = b.autotune(Fd, reps=1, stream=stream)
            res["autotune_ms"] = [before, after]
        dt, (s, it, st) = _time_solves(b, Fd, reps, stream)
        it = it.cpu().numpy()
        res.update(batch_s=dt, rve_solves_per_s=n / dt, iters_mean=float(it.mean()), iters_max=int(it.max()),
                   converged_frac=float((st.cpu().numpy() == 0).mean()), bins=b.bins())
    m = min(plain_subset, n)
    if m == 0:
        b.close()
        return res
    sub = rvegen.pack(nets[:m])
    pv, pit = _plain(sub, Fs[:m], tol_d, device, damping_scale)
    # the plain path solves from the affine start; for the tangent the batched
    # solves are warm-started, so the ratio there compares unlike solves
    res.update(plain_fp64_subset=m, plain_fp64_solves_per_s=pv, plain_iters_mean=float(pit.mean()),
               plain_start="cold")
    res["speedup_vs_plain"] = res["rve_solves_per_s"] / pv
    b.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["single", "uneven", "tangent", "orientation", "streamed"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--plain-subset", type=int, default=32)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--damping-scale", type=float, default=1.0, help="s in c = s * 2 sqrt(lambda), both paths")
    ap.add_argument("--kernel", choices=sorted(KERNELS), default="auto",
                    help="batched kernel: two-phase (auto) or node-centric with clusters for large RVEs (node)")
    a = ap.parse_args()
    print(json.dumps(run(a.config, a.reps, a.plain_subset, autotune=not a.no_autotune,
                         damping_scale=a.damping_scale, kernel=a.kernel)))


if __name__ == "__main__":
    main()
