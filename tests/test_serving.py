"""Serving loop (rve_server_*): continuous batching over a resident pool.

CPU part: the request stream is reproducible and Poisson.  GPU part: every
request's result is the same whether it is solved alone or inside the mix
of overlapping waves, with whole-solve waves and with iteration-level waves
(solves parked and resumed between waves); served stresses match the
oracle; latencies are accounted; admission honours the cap at creation and
when RVE topologies are admitted or removed mid-stream."""
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


def _mix(rve, b, ids, Fs, wave_iters, n_slots=3, max_wave=16):
    srv = rve.RveServer(b, n_slots=n_slots, max_wave=max_wave, wave_iters=wave_iters)
    for k in range(len(ids)):
        srv.submit(int(ids[k]), Fs[k], k)
        if k % 5 == 0:
            srv.step()
    srv.drain()
    tags, sig, it, st, lat = srv.poll(10 * len(ids))
    stats = srv.stats()
    srv.close()
    order = np.argsort(tags)
    assert sorted(tags.tolist()) == list(range(len(ids)))
    return sig[order], it[order], st[order], stats


@pytest.mark.gpu
def test_iteration_waves_same_alone_and_in_the_mix(rve):
    """Waves of 100 DR iterations: solves park and resume between waves,
    finished ones retire and queued ones take their slots; every result is
    bit-identical to the same request served alone, and within the mixed
    path's tolerance of a solve that runs to the end in one launch."""
    import torch
    nets = [rvegen.config_serving_network(r, sides=(6, 8, 12)) for r in range(30)]
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, warm_start=0)
    rng = np.random.default_rng(1)
    n = 120
    ids = rng.integers(0, 30, n)
    Fs = np.stack([rvegen.random_F(rvegen.Stream(5000 + k)) for k in range(n)])
    sig, it, st, stats = _mix(rve, b, ids, Fs, wave_iters=100)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    assert (it > 100).mean() > 0.5          # most solves spanned several waves
    assert stats["waves"] > n // 16 and stats["wave_iters"] == 100 and stats["in_flight"] == 0
    for k in range(0, n, 11):
        s1, it1, st1, _ = _mix(rve, b, ids[k:k + 1], Fs[k:k + 1], wave_iters=100, n_slots=1, max_wave=1)
        assert np.array_equal(s1[0], sig[k]) and it1[0] == it[k], k
        s2, _, _ = b.solve_subset(np.array([ids[k]]), torch.tensor(Fs[k].reshape(1, 9), device="cuda:0"))
        s2 = s2.cpu().numpy()[0]
        assert np.linalg.norm(s2 - sig[k]) <= 1e-4 * np.linalg.norm(s2), k
    b.close()


@pytest.mark.gpu
def test_served_stresses_match_the_oracle(rve):
    """Stresses returned by the server (iteration-level waves, cold starts)
    against the FP64 oracle: its own equilibrium, or a verified other stable
    minimum reached from the state the served solve left on the device."""
    from oracle.newton import solve_network
    from tests.parity import classify
    nets = [rvegen.config_serving_network(r, sides=(6, 8)) for r in range(12)]
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, warm_start=0)
    ids = np.arange(12)
    Fs = np.stack([rvegen.random_F(rvegen.Stream(7000 + k)) for k in range(12)])
    sig, it, st, _ = _mix(rve, b, ids, Fs, wave_iters=150, n_slots=2, max_wave=4)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    items = []
    for k in range(12):
        ref = solve_network(nets[k], Fs[k], tol=1e-10)
        items.append(dict(k=k, net=nets[k], F=Fs[k], sigma=sig[k].reshape(3, 3), ref=ref.sigma,
                          ref_energy=ref.info["energy"]))
    print("served vs oracle:", classify(b, rve.RVE_PREC_MIXED, items, 1e-4, "served"))
    b.close()


@pytest.mark.gpu
def test_admission_of_new_rves_mid_stream(rve):
    """The pool grows while requests are served: a group of new topologies is
    admitted under the cap and served; one that would exceed the cap is
    refused with RVE_EADMIT and nothing changes; removing an idle group frees
    its memory so the refused group fits."""
    base = [rvegen.config_serving_network(r, sides=(6,)) for r in range(8)]
    b = rve.RveBatch(rvegen.pack(base), precision=rve.RVE_PREC_MIXED, warm_start=1)
    small = rvegen.pack([rvegen.config_serving_network(100 + r, sides=(8,)) for r in range(16)])
    big = rvegen.pack([rvegen.config_serving_network(200 + r, sides=(12,)) for r in range(24)])
    probe = rve.RveServer(b, n_slots=2, max_wave=8, hbm_cap_bytes=0.0)
    bytes_base = probe.stats()["pool_device_bytes"] + probe.stats()["device_bytes"]
    f_small = probe.add_rves(small)
    bytes_small = probe.stats()["pool_device_bytes"] + probe.stats()["device_bytes"] - bytes_base
    first_big = probe.add_rves(big)
    bytes_big = probe.stats()["pool_device_bytes"] + probe.stats()["device_bytes"] - bytes_base - bytes_small
    probe.close()
    assert first_big == f_small + 16 and bytes_big > bytes_small > 0
    # room for the base pool with either group alone, not with both
    cap = bytes_base + bytes_big + 0.5 * bytes_small
    srv = rve.RveServer(b, n_slots=2, max_wave=8, hbm_cap_bytes=cap, wave_iters=200)
    F = rvegen.random_F(rvegen.Stream(11))
    for k in range(8):
        srv.submit(k, F, k)
    srv.step()
    first = srv.add_rves(small)                      # admitted while waves run
    assert first == 8 and srv.stats()["pool_rves"] == 24
    for k in range(16):
        srv.submit(first + k, F, 100 + k)
    with pytest.raises(rve.RveError) as e:
        srv.add_rves(big)
    assert e.value.code == rve.RVE_EADMIT
    assert srv.stats()["pool_rves"] == 24
    with pytest.raises(rve.RveError):
        srv.submit(first + 16, F, 999)               # not in the pool
    with pytest.raises(rve.RveError):
        srv.remove_rves(first)                       # requests queued or in flight
    srv.drain()
    tags, sig, it, st, lat = srv.poll(100)
    assert sorted(tags.tolist()) == list(range(8)) + list(range(100, 116))
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    srv.remove_rves(first)
    assert srv.stats()["pool_rves"] == 8
    with pytest.raises(rve.RveError):
        srv.submit(first, F, 0)                       # removed
    first2 = srv.add_rves(big)                       # fits once the small group is gone
    assert first2 == first + 16                       # ids are never reused
    for k in range(24):
        srv.submit(first2 + k, F, 200 + k)
    srv.drain()
    tags, sig, it, st, lat = srv.poll(100)
    assert sorted(tags.tolist()) == list(range(200, 224)) and (st == rve.RVE_STATUS_CONVERGED).all()
    srv.close()
    b.close()
