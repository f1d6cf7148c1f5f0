"""Benchmark: batched fiber-network RVE solves on GB300.

Workload: 1024 jittered 10x10x10 networks (bond p = 0.6, EA = 1, B = 10),
each under its own random F = R U (principal strains in [-0.05, 0.15]),
solved from the affine start to sigma relative error <= 1e-4 against the
FP64 oracle (mixed precision, relative residual tolerance chosen and
validated in tests/test_gpu_parity.py).  One step = one rve_solve over the
whole batch.  Inputs are synthetic (rvegen), resident in HBM when timing
starts; L2 is flushed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RVE solves/s batched vs plain per-RVE at sigma rel.err <=1e-4"
UNIT = "RVE solves/s"
N_RVE = 1024
SIDE = 10
# stopping rule of both timed paths: relative residual <= 1e-6 AND the
# estimated remaining stress error <= 2e-5 (option sigma_tol).  On this
# batch the largest stress error against FP64 solves at 1e-10 is 7.1e-5,
# below the library default's 8.4e-5 (residual 3e-7 alone), at 1.25x its
# speed; parity-tested at these options in tests/test_gpu_parity.py.
TOL = 1e-6
SIGMA_TOL = 2e-5
DAMPING_SCALE = 0.6  # c = 0.6 * 2 sqrt(lambda_RQ) on both paths timed (parity-tested at this setting)
PLAIN_SUBSET = 32   # RVEs timed on the plain FP64 per-RVE path
F_STEP = 1e-3       # step k solves F + k F_STEP G (G fixed, |G_ij| <= 1): a small increment per step
# Algorithmic work of one DR iteration (the method's own count, FMA = 2
# flops): about 30 FP32 flops + 1 exp + 1 rsqrt per fiber-update (chord,
# strain, length, law, force vector) and about 20 per free-node update
# (gathered force, damped velocity, position).
FLOPS_PER_FIBER_UPDATE = 30.0
FLOPS_PER_NODE_UPDATE = 20.0
# this kernel's own count, reported beside it: fiber force 39 (adds the
# stiffness bound 7, chord update 3, misc 3) + CSR gather 8; node 17
IMPL_FLOPS_PER_FIBER_UPDATE = 47.0
IMPL_FLOPS_PER_NODE_UPDATE = 17.0
# Algorithmic on-chip bytes of one DR iteration: per active fiber its two
# endpoint indices and three parameters (20 B), per free node h and v read
# and written plus 1/m (52 B); boundary nodes are not stored (zero slot).
BYTES_PER_FIBER_UPDATE = 20.0
BYTES_PER_NODE_UPDATE = 52.0
FP32_LANES_PER_SM = 128
SMEM_BYTES_PER_CLK_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum of the fused kernel's 1016-RVE
# launch on this workload (ncu capture summarised in profiles/; the 8-RVE
# launch beside it adds about 1 %); None whenever the kernel changes after
# that capture
TRAFFIC_BYTES_PER_LAUNCH = 104.73e6 + 5.09e6


def _config():
    return {"workload": "uniform batch: 1024 RVEs, 10x10x10 jittered grid, bond p=0.6, EA=1, B=10, "
                        "random F=R.U (principal strains U[-0.05,0.15])",
            "n_rve": N_RVE, "grid_side": SIDE, "tol_rel_residual": TOL, "sigma_tol": SIGMA_TOL,
            "damping_scale": DAMPING_SCALE, "precision": "mixed (FP32 forces/updates, "
            "FP64 residual and stress sums)", "start": "cold (h=0) every step",
            "F_per_step": f"step k solves F + k*{F_STEP:g}*G (G fixed, entries in [-1,1]): no two steps repeat F",
            "l2": "flushed between timed steps (256 MiB write)"}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only samples
    whose timestamps fall inside the timed window [t0, t1] (host wall clock)
    are summarised."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self, t0: float = 0.0, t1: float = float("inf")):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        return self.summarise(out, t0, t1)

    @staticmethod
    def summarise(out: str, t0: float = 0.0, t1: float = float("inf")) -> dict:
        """Median SM clock under load, maximum clock and active throttle reasons
        of the csv lines (query Q) whose timestamps fall in [t0, t1]."""
        import datetime
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if not (t0 <= ts <= t1):
                    continue
                sm.append(float(f[2]))
                smax.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples inside the timed window"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle

def _oracle_job(args):
    i, tol = args
    import rvegen
    from oracle.newton import solve_network
    nets, F = rvegen.config_uniform(1, side=SIDE, first=i)
    t = time.time()
    solve_network(nets[0], F[0], tol=tol)
    return time.time() - t


class OraclePool:
    """The FP64 Newton oracle as it stands, one spawned process per host core."""

    def __init__(self):
        from multiprocessing import get_context
        self.cores = len(os.sched_getaffinity(0))
        self.pool = get_context("spawn").Pool(self.cores)
        self.next = 0

    def run(self, budget_s: float, tol: float = 1e-6):
        """Solve workload RVEs (continuing from the last index) until the budget
        is spent; RVEs already started are finished.  Returns (done, wall)."""
        t0 = time.time()
        pending, done = [], 0
        while True:
            while len(pending) < self.cores and time.time() - t0 < budget_s:
                pending.append(self.pool.apply_async(_oracle_job, ((self.next, tol),)))
                self.next += 1
            if not pending:
                break
            pending.pop(0).get()
            done += 1
        return done, time.time() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_baseline(budget_s: float = 20.0, tol: float = 1e-6):
    pool = OraclePool()
    done, wall = pool.run(budget_s, tol)
    pool.close()
    return {"value": done / wall, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"first {done} RVEs of the workload, FP64 Newton (scipy SuperLU) at relative residual "
                      f"{tol:g}, one process per core, {wall:.1f} s wall"}


# -------------------------------------------------------------------- GPU

def serving_latency(device: int, pool: int = 2000, rate: float = 20000.0, duration: float = 3.0) -> dict:
    """p50/p99 request latency through the continuous-batching server (outside
    the timed region): a Poisson stream of single RVE solves, each request an
    RVE of a resident pool (sides 6, 8, 12, 16) under its own F, library
    defaults, warm starts kept on the device."""
    import rvegen
    import paper_2306_09427_gb300 as rve
    from paper_2306_09427_gb300.serve import pool_networks, request_stream, run_poisson
    b = rve.RveBatch(rvegen.pack(pool_networks(pool)), device=device, precision=rve.RVE_PREC_MIXED, warm_start=1)
    t, ids, F = request_stream(pool, rate, duration)
    r = run_poisson(b, t, ids, F)
    b.close()
    return {"p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "throughput": r["throughput"], "unit": "requests/s",
            "offered_rate": r["offered_rate"], "requests": r["requests"], "converged_frac": r["converged_frac"],
            "workload": f"Poisson stream {rate:.0f}/s for {duration:.0f} s over a pool of {pool} RVEs "
                        "(sides 6, 8, 12, 16), warm starts resident"}


def run_ours(args, rank, world, local):
    import torch

    import rvegen
    import paper_2306_09427_gb300 as rve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # each rank solves its own shard of independent RVEs (weak scaling)
    nets, Fs = rvegen.config_uniform(N_RVE, side=SIDE, first=rank * N_RVE)
    pk = rvegen.pack(nets)
    b = rve.RveBatch(pk, device=local, precision=rve.RVE_PREC_MIXED, tol=TOL, sigma_tol=SIGMA_TOL, warm_start=0,
                     damping_scale=DAMPING_SCALE)
    # per-step deformation gradients, all resident before timing
    G = rvegen.Stream(0x5EEDF00D + rank).uniform(9 * N_RVE, -1.0, 1.0).reshape(N_RVE, 9)
    n_steps = args.warmup + args.steps
    F_all = np.stack([Fs.reshape(-1, 9) + k * F_STEP * G for k in range(n_steps + 1)])
    Fd_all = torch.tensor(F_all, dtype=torch.float64, device=dev)
    sigma = torch.empty((N_RVE, 9), dtype=torch.float64, device=dev)
    iters_all = torch.empty((n_steps + 1, N_RVE), dtype=torch.int32, device=dev)  # each step's own counts
    iters = iters_all[n_steps]
    status = torch.empty(N_RVE, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(k):
        b.solve(Fd_all[k], sigma=sigma, iters=iters_all[k], status=status, stream=stream)

    # the first solve of a fresh batch: no learned per-RVE cost for the
    # longest-first order yet (set-up of the size bins excluded: done by a
    # solve of another batch object of the same networks)
    b_cold = rve.RveBatch(pk, device=local, precision=rve.RVE_PREC_MIXED, tol=TOL, sigma_tol=SIGMA_TOL,
                          warm_start=0, damping_scale=DAMPING_SCALE)
    b_cold.set_kernel_timing(True)
    b_cold.solve(Fd_all[0], sigma=sigma, iters=iters, status=status, stream=stream)
    torch.cuda.synchronize()
    first_solve_ms = float(b_cold.last_kernel_ms().sum())
    b_cold.close()
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    n_bins = b.info()["n_bins"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    info = b.info()  # after the first solve: the size bins exist
    clk = ClockSampler(local)
    clk.start()
    time.sleep(1.0)  # nvidia-smi start-up, so that samples cover the timed window
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    b.set_kernel_timing(True)  # events around each fused-kernel launch, on its launching stream
    t_win0 = time.time()
    it_total = 0
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(args.warmup + k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop(t_win0, time.time())
    step_ms = [a.elapsed_time(z) for a, z in ev]
    kernel_ms = b.last_kernel_ms()  # n_bins launches per step
    b.set_kernel_timing(False)
    t_total = sum(step_ms) / 1e3
    it_steps = iters_all[args.warmup:args.warmup + args.steps].cpu().numpy()  # (steps, N_RVE)
    it = it_steps[-1]
    st = status.cpu().numpy()
    if world > 1:
        t = torch.tensor([t_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_total = float(t.item())
    value = world * N_RVE * args.steps / t_total
    # fiber-updates and roofline of the fused kernel (one launch per bin per step)
    nf, na, _ = b.sizes()
    fiber_updates = float((na.astype(np.float64) * it_steps).sum()) / args.steps  # per step
    node_updates = float((nf.astype(np.float64) * it_steps).sum()) / args.steps
    t_step = t_total / args.steps
    # the dominant kernel: the fused solve; with one bin it is one launch per step,
    # with several (concurrent) bins their summed durations bound the kernel time
    t_kernel = float(kernel_ms.sum()) / 1e3 / args.steps
    flops = FLOPS_PER_FIBER_UPDATE * fiber_updates + FLOPS_PER_NODE_UPDATE * node_updates
    impl_flops = IMPL_FLOPS_PER_FIBER_UPDATE * fiber_updates + IMPL_FLOPS_PER_NODE_UPDATE * node_updates
    onchip = BYTES_PER_FIBER_UPDATE * fiber_updates + BYTES_PER_NODE_UPDATE * node_updates
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flops / t_kernel / 1e12
    smem_peak = sm_count * SMEM_BYTES_PER_CLK_PER_SM * mhz * 1e6 / 1e9
    smem_achieved = onchip / t_kernel / 1e9

    # end to end through the public host-buffer call (copies inside)
    e2e_steps = max(1, min(args.steps, 5))
    b.solve_host(F_all[0])  # staging buffers allocated outside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        b.solve_host(F_all[k + 1])
    e2e = N_RVE * e2e_steps / (time.perf_counter() - t0)

    # plain FP64 per-RVE path on a subset (one RVE at a time, several launches per iteration)
    plain = None
    if rank == 0 and not args.no_plain:
        sub = rvegen.pack(nets[:PLAIN_SUBSET])
        bp = rve.RveBatch(sub, device=local, precision=rve.RVE_PREC_PLAIN_F64, tol=TOL, sigma_tol=SIGMA_TOL,
                          damping_scale=DAMPING_SCALE)
        sp = torch.empty((PLAIN_SUBSET, 9), dtype=torch.float64, device=dev)
        bp.solve(Fd_all[0, :PLAIN_SUBSET].contiguous(), sigma=sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bp.solve(Fd_all[1, :PLAIN_SUBSET].contiguous(), sigma=sp)
        torch.cuda.synchronize()
        plain = PLAIN_SUBSET / (time.perf_counter() - t0)
        bp.close()

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 residual and stress accumulation)", "data": "synthetic",
        "config": _config(),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 9 * 8 * N_RVE,
                "d2h_bytes_per_step": 9 * 8 * N_RVE + 2 * 4 * N_RVE},
        # per bin and step: the longest-first sort of the work list, then the fused solve
        "gpu_launches": args.steps * sum(x["sorted"] + 1 + (x["exclusive"] > 0) for x in b.bins()),
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_LAUNCH, "traffic_unit": "bytes per launch",
                     "kernel_ms_per_launch": float(kernel_ms.mean()), "launches_timed": int(kernel_ms.size),
                     "kernel": "dr_fused_kernel<float,...> (one CTA per RVE, resident in shared memory)",
                     "work": f"{FLOPS_PER_FIBER_UPDATE:g} flops per fiber-update + {FLOPS_PER_NODE_UPDATE:g} per "
                             "free-node update (algorithmic)",
                     "impl_flops_frac": impl_flops / t_kernel / 1e12 / peak,
                     "peak_note": f"FP32 FMA peak derived: {sm_count} SMs x 128 lanes x 2 flops x {mhz:.0f} MHz "
                                  "(median SM clock under load)"},
        "roofline_smem": {"bound": "smem", "achieved": smem_achieved, "peak": smem_peak, "unit": "GB/s",
                          "frac": smem_achieved / smem_peak,
                          "work": f"{BYTES_PER_FIBER_UPDATE:g} B per fiber-update + {BYTES_PER_NODE_UPDATE:g} B per "
                                  "free-node update (algorithmic on-chip bytes)",
                          "peak_note": f"{sm_count} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk x {mhz:.0f} MHz"},
        "first_solve_ms": first_solve_ms,
        "fiber_updates_per_s": fiber_updates / t_step,
        "iterations": {"mean": float(it_steps.mean()), "max": int(it_steps.max()),
                       "converged_frac_last_step": float((st == 0).mean())},
        "plain_fp64_per_rve": {"value": plain, "unit": UNIT, "subset": f"first {PLAIN_SUBSET} RVEs, same tol"}
        if plain else None,
        "speedup_vs_plain": (value / world) / plain if plain else None,
        "batch": info,
    }
    if rank == 0 and not args.no_serve:
        res["latency"] = serving_latency(local)
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"] = oracle_baseline(args.cpu_budget)
    if world > 1:
        torch.distributed.destroy_process_group()
    b.close()
    return res


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the same workload and metric,
    each step a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return None
    pool = OraclePool()
    per_step = max(2.0, args.cpu_budget / max(args.steps, 1))
    for _ in range(args.warmup):
        pool.run(0.0)  # one RVE per core, untimed
    done = wall = 0.0
    for _ in range(args.steps):
        d, w = pool.run(per_step)
        done += d
        wall += w
    pool.close()
    v = done / wall
    base = {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{int(done)} RVEs of the workload over {args.steps} steps of ~{per_step:.0f} s, FP64 Newton "
                      f"at relative residual 1e-6, one process per core"}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(),
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for the CPU baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-latency measurement")
    args = ap.parse_args()
    rank, world, local = _dist()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
