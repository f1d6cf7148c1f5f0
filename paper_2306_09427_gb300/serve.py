"""Serving driver: Poisson stream of RVE solve requests through ``RveServer``
(iteration-level waves of WAVE_ITERS DR iterations by default).

Requests arrive with exponential inter-arrival times (counter-based stream,
reproducible), each naming an RVE of a resident pool and its deformation
gradient.  Request k on RVE r uses F = F_r + 0.002 G_k: a base gradient of
the RVE (random R U as in the uniform workload) plus a small per-request
increment, the pattern successive macroscale Newton iterations produce, so
the resident warm-start state of each RVE is useful.  Latency is measured
from the scheduled arrival time to the moment the driver sees the result.

    python -m paper_2306_09427_gb300.serve --pool 2000 --rate 20000 --duration 5
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import rvegen

from ._lib import RVE_PREC_MIXED, RveBatch, RveServer


def pool_networks(n: int, sides=(6, 8, 12, 16)):
    return [rvegen.config_serving_network(r, sides) for r in range(n)]


def request_stream(n_pool: int, rate: float, duration: float, seed: int = 5):
    """Arrival times (s), RVE ids and per-request F (n, 9)."""
    st = rvegen.Stream(seed)
    n = int(rate * duration * 1.2) + 16
    gaps = -np.log(1.0 - st.uniform(n)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    n = t.shape[0]
    rve = np.minimum((st.uniform(n) * n_pool).astype(np.int64), n_pool - 1)
    base = np.stack([rvegen.random_F(rvegen.Stream(rvegen.rve_seed(5, 1 << 19 | r))) for r in range(n_pool)])
    G = st.uniform(9 * n, -1.0, 1.0).reshape(n, 3, 3)
    F = base[rve] + 0.002 * G
    return t, rve, F.reshape(n, 9)


WAVE_ITERS = 200  # DR iterations per wave (solves park and resume between waves)


def run_poisson(batch: RveBatch, t_arr, rve, F, n_slots: int = 4, max_wave: int = 2048,
                hbm_cap_bytes: float = 150e9, wave_iters: int = WAVE_ITERS) -> dict:
    srv = RveServer(batch, n_slots=n_slots, max_wave=max_wave, hbm_cap_bytes=hbm_cap_bytes, wave_iters=wave_iters)
    n = t_arr.shape[0]
    done_t = np.full(n, np.nan)
    sigma = np.full((n, 9), np.nan)
    status = np.full(n, -1, np.int32)
    iters = np.zeros(n, np.int32)
    nxt = 0
    got = 0
    t0 = time.perf_counter()
    while got < n:
        now = time.perf_counter() - t0
        while nxt < n and t_arr[nxt] <= now:
            srv.submit(int(rve[nxt]), F[nxt], nxt)
            nxt += 1
        srv.step()
        tags, s, it, st, _ = srv.poll()
        if tags.size:
            tnow = time.perf_counter() - t0
            done_t[tags] = tnow
            sigma[tags] = s
            iters[tags] = it
            status[tags] = st
            got += tags.size
        if nxt >= n and got < n and srv.stats()["in_flight"] == 0 and srv.stats()["queued"] == 0:
            srv.drain()
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = done_t - t_arr
    return {"requests": int(n), "wall_s": wall, "throughput": n / wall, "offered_rate": n / float(t_arr[-1]),
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_iters": float(iters.mean()), "converged_frac": float((status == 0).mean()),
            "waves": int(stats["waves"]), "wave_iters": wave_iters, "sigma": sigma, "status": status,
            "latency_s": lat}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pool", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=20000.0)
    ap.add_argument("--duration", type=float, default=5.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-wave", type=int, default=2048)
    ap.add_argument("--precision", type=int, default=RVE_PREC_MIXED, help="0 plain FP64 per RVE, 1 mixed, 2 FP64")
    ap.add_argument("--wave-iters", type=int, default=WAVE_ITERS, help="DR iterations per wave (0: whole solves)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="0 two-phase kernel, 2 node-centric kernels (clusters for RVEs too large for one CTA)")
    a = ap.parse_args()
    nets = pool_networks(a.pool)
    b = RveBatch(rvegen.pack(nets), precision=a.precision, warm_start=1, kernel=a.kernel)
    t, rve, F = request_stream(a.pool, a.rate, a.duration)
    wave = a.wave_iters if a.precision != 0 else 0
    res = run_poisson(b, t, rve, F, n_slots=a.slots, max_wave=a.max_wave, wave_iters=wave)
    out = {k: v for k, v in res.items() if not isinstance(v, np.ndarray)}
    out.update(pool=a.pool, slots=a.slots, max_wave=a.max_wave, precision=a.precision, kernel=a.kernel)
    print(json.dumps(out))
    b.close()


if __name__ == "__main__":
    main()
