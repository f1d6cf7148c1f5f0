"""Serving loop (rve_server_*): continuous batching over a resident pool.

CPU part: the request stream is reproducible and Poisson.  GPU part: every
request's result is the same whether it is solved alone or inside the mix
of overlapping waves; latencies are accounted; admission honours the cap."""
import numpy as np
import pytest

import rvegen


def test_request_stream_is_poisson_and_reproducible():
    import __graft_entry__ as g
    g.build()
    from paper_2306_09427_gb300.serve import request_stream
    t1, r1, F1 = request_stream(50, 4000.0, 2.0, seed=3)
    t2, r2, F2 = request_stream(50, 4000.0, 2.0, seed=3)
    assert np.array_equal(t1, t2) and np.array_equal(r1, r2) and np.array_equal(F1, F2)
    gaps = np.diff(t1)
    assert abs(gaps.mean() * 4000.0 - 1.0) < 0.05          # mean inter-arrival 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05      # exponential: CV = 1
    assert r1.min() >= 0 and r1.max() < 50
    assert np.abs(np.linalg.det(F1.reshape(-1, 3, 3)) - 1.0).max() < 0.6


@pytest.fixture(scope="module")
def rve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2306_09427_gb300 as rve
    return rve


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix(rve):
    import torch
    nets = [rvegen.config_serving_network(r, sides=(6, 8)) for r in range(40)]
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, warm_start=0)
    rng = np.random.default_rng(0)
    n = 300
    ids = rng.integers(0, 40, n)
    Fs = np.stack([rvegen.random_F(rvegen.Stream(900 + k)) for k in range(n)])
    srv = rve.RveServer(b, n_slots=3, max_wave=16)
    for k in range(n):
        srv.submit(int(ids[k]), Fs[k], k)
        if k % 7 == 0:
            srv.step()
    srv.drain()
    tags, sig, it, st, lat = srv.poll(10 * n)
    assert sorted(tags.tolist()) == list(range(n))
    assert (st == 0).all() and (lat > 0).all()
    stats = srv.stats()
    assert stats["completed"] == n and stats["waves"] > 1
    order = np.argsort(tags)
    sig = sig[order]
    for k in range(0, n, 23):  # solved alone
        s1, _, _ = b.solve_subset(np.array([ids[k]]), torch.tensor(Fs[k].reshape(1, 9), device="cuda:0"))
        assert np.array_equal(s1.cpu().numpy()[0], sig[k]), k
    srv.close()
    b.close()


@pytest.mark.gpu
def test_poisson_stream_latency_and_warm_history(rve):
    from paper_2306_09427_gb300.serve import pool_networks, request_stream, run_poisson
    nets = pool_networks(60, sides=(6, 8))
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, warm_start=1)
    t, ids, F = request_stream(60, 3000.0, 0.5)
    res = run_poisson(b, t, ids, F, n_slots=4, max_wave=256)
    assert res["converged_frac"] == 1.0
    assert np.isfinite(res["latency_s"]).all() and (res["latency_s"] > 0).all()
    assert res["p99_ms"] >= res["p50_ms"] > 0
    assert res["waves"] > 1
    b.close()


@pytest.mark.gpu
def test_admission_cap(rve):
    nets = [rvegen.config_serving_network(r, sides=(6,)) for r in range(8)]
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED)
    with pytest.raises(rve.RveError) as e:
        rve.RveServer(b, n_slots=2, max_wave=8, hbm_cap_bytes=1e3)
    assert e.value.code == rve.RVE_EADMIT
    b.close()
