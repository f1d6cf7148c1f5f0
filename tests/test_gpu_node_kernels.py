"""GPU parity of the node-centric kernels (option kernel = RVE_KERNEL_NODE):
the one-CTA node-centric kernel for RVEs that fit one CTA's shared memory
and the thread-block-cluster kernel for larger ones, against the FP64
oracle (stored goldens; the acceptance rule of tests/parity.py where a
network holds several stable equilibria), against the two-phase kernel,
alone and inside a batch, and under iteration-level serving waves."""
import json
import os

import numpy as np
import pytest

import rvegen
from tests.parity import classify, rel

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def rve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2306_09427_gb300 as rve
    return rve


def _F(F):
    import torch
    return torch.tensor(np.asarray(F).reshape(-1, 9), dtype=torch.float64, device="cuda:0")


def _rows(name):
    rows = json.load(open(os.path.join(HERE, "golden", f"oracle_{name}.json")))["rows"]
    assert all(r["converged"] and r["stable"] for r in rows)
    return rows


def _solve(b, Fs):
    s, it, st = b.solve(_F(Fs))
    return s.cpu().numpy().reshape(-1, 3, 3), it.cpu().numpy(), st.cpu().numpy()


def test_node_kernel_uniform_against_the_oracle(rve):
    rows = _rows("uniform_10")
    n = max(r["index"] for r in rows) + 1
    nets, Fs = rvegen.config_uniform(n)
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, kernel=rve.RVE_KERNEL_NODE)
    s, it, st = _solve(b, Fs)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    assert {x["kernel"] for x in b.bins()} == {1}  # every 10^3 RVE fits one CTA
    items = [dict(k=r["index"], net=nets[r["index"]], F=Fs[r["index"]], sigma=s[r["index"]],
                  ref=np.array(r["sigma"]).reshape(3, 3), ref_energy=r["energy"]) for r in rows]
    c = classify(b, rve.RVE_PREC_MIXED, items, 1e-4, "node kernel, uniform")
    print("node kernel, uniform 64 vs oracle:", c)
    assert c["other"] <= 10
    b.close()


def test_node_kernels_fp64_match_the_two_phase_kernel(rve):
    """FP64 to relative residual 1e-10: both kernels take Algorithm 2's
    iterates and differ only in the order of the force sums at a node."""
    nets, Fs = rvegen.config_uneven(24, side_hi=12)
    out = {}
    for kern in (rve.RVE_KERNEL_TWO_PHASE, rve.RVE_KERNEL_NODE):
        b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-10, max_iter=2_000_000,
                         kernel=kern)
        s, it, st = _solve(b, Fs)
        assert (st == rve.RVE_STATUS_CONVERGED).all()
        out[kern] = s
        b.close()
    e = max(rel(a, b_) for a, b_ in zip(out[rve.RVE_KERNEL_NODE], out[rve.RVE_KERNEL_TWO_PHASE]))
    print("node vs two-phase kernel, FP64 at 1e-10: max sigma difference %.2e" % e)
    assert e <= 1e-8


def test_cluster_kernel_large_rves_against_the_oracle(rve):
    """The uneven goldens' RVEs too large for one CTA (side 13-16) on
    thread-block clusters, against the stored oracle solves."""
    rows = _rows("uneven")
    nets_all, Fs_all = rvegen.config_uneven(max(r["index"] for r in rows) + 1)
    big = [r for r in rows if nets_all[r["index"]].n_nodes >= 13 ** 3]
    assert len(big) >= 8
    nets = [nets_all[r["index"]] for r in big]
    Fs = np.stack([Fs_all[r["index"]] for r in big])
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, kernel=rve.RVE_KERNEL_NODE)
    s, it, st = _solve(b, Fs)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    bins = b.bins()
    assert any(x["kernel"] == 2 and 2 <= x["cluster"] <= 8 for x in bins), bins
    items = [dict(k=j, net=nets[j], F=Fs[j], sigma=s[j], ref=np.array(r["sigma"]).reshape(3, 3),
                  ref_energy=r["energy"]) for j, r in enumerate(big)]
    c = classify(b, rve.RVE_PREC_MIXED, items, 1e-4, "cluster kernel, large RVEs")
    print(f"cluster kernel, {len(big)} large uneven RVEs vs oracle:", c,
          [(x["cluster"], x["nodes_per_thread"], x["n_rve"]) for x in bins if x["kernel"] == 2])
    assert c["other"] <= len(big) // 4
    # the same RVEs on the streamed two-phase kernel
    b2 = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, kernel=rve.RVE_KERNEL_TWO_PHASE)
    s2, _, _ = _solve(b2, Fs)
    d = max(rel(x, y) for x, y in zip(s, s2))
    print("cluster vs streamed two-phase kernel: max sigma difference %.2e" % d)
    b2.close()
    b.close()


def test_node_kernels_alone_equal_in_batch(rve):
    """Deterministic force sums: a result does not depend on the rest of the
    batch, for the one-CTA kernel and for the cluster kernel."""
    nets, Fs = rvegen.config_uneven(30, side_lo=6, side_hi=16)
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, tol=1e-6, kernel=rve.RVE_KERNEL_NODE)
    s_all, _, st = _solve(b, Fs)
    s_again, _, _ = _solve(b, Fs)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    assert np.array_equal(s_all, s_again)
    # one-CTA node-centric and cluster bins both present (a resident bin whose
    # node-centric layout does not fit one CTA keeps the two-phase kernel)
    kinds = {x["kernel"] for x in b.bins()}
    assert {1, 2} <= kinds, b.bins()
    assert all(x["mode"] == 0 for x in b.bins() if x["kernel"] == 0), b.bins()
    b.close()
    sizes = [n.n_nodes for n in nets]
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        b1 = rve.RveBatch(rvegen.pack([nets[k]]), precision=rve.RVE_PREC_MIXED, tol=1e-6, kernel=rve.RVE_KERNEL_NODE)
        s1, _, _ = _solve(b1, Fs[k:k + 1])
        assert np.array_equal(s1[0], s_all[k]), k
        b1.close()


def test_node_kernels_under_iteration_waves(rve):
    """Serving waves of 100 DR iterations with the node-centric kernels:
    solves park and resume; each result is bit-identical to the same request
    served alone and within 1e-4 of a solve that runs to the end."""
    import torch
    nets = [rvegen.config_serving_network(r, sides=(6, 8, 16)) for r in range(12)]
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, warm_start=0, kernel=rve.RVE_KERNEL_NODE)
    rng = np.random.default_rng(2)
    n = 40
    ids = rng.integers(0, 12, n)
    Fs = np.stack([rvegen.random_F(rvegen.Stream(7000 + k)) for k in range(n)])

    def mix(idx, F, n_slots, max_wave):
        srv = rve.RveServer(b, n_slots=n_slots, max_wave=max_wave, wave_iters=100)
        for k in range(len(idx)):
            srv.submit(int(idx[k]), F[k], k)
            if k % 5 == 0:
                srv.step()
        srv.drain()
        tags, sig, it, st, lat = srv.poll(10 * len(idx))
        srv.close()
        order = np.argsort(tags)
        return sig[order], it[order], st[order]

    sig, it, st = mix(ids, Fs, 3, 8)
    assert (st == rve.RVE_STATUS_CONVERGED).all()
    assert (it > 100).mean() > 0.5
    big = [k for k in range(n) if nets[ids[k]].n_nodes == 16 ** 3]
    assert big, "no request on a cluster-sized RVE"
    for k in sorted(set(range(0, n, 9)) | set(big[:2])):
        s1, it1, _ = mix(ids[k:k + 1], Fs[k:k + 1], 1, 1)
        assert np.array_equal(s1[0], sig[k]) and it1[0] == it[k], k
        s2, _, _ = b.solve_subset(np.array([ids[k]]), torch.tensor(Fs[k].reshape(1, 9), device="cuda:0"))
        s2 = s2.cpu().numpy()[0]
        assert np.linalg.norm(s2 - sig[k]) <= 1e-4 * np.linalg.norm(s2), k
    b.close()
