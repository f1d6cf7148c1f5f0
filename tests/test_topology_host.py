"""The library's host-side set-up (validation, pruning, renumbering, the
node CSR and the bank-aware orders) on the CPU: compiled with g++ together
with tests/topology_shim.cpp and checked against the oracle's pruning rules
and the definitions the kernels rely on."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import rvegen
from oracle.network import prune
from tests import nets as tnets

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2306_09427_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    out = str(tmp_path_factory.mktemp("topo") / "libtopo.so")
    cmd = [gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-I", CUDA_INC, os.path.join(CSRC, "topology.cpp"), os.path.join(HERE, "topology_shim.cpp"),
           "-o", out, "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    lib.shim_error.restype = C.c_char_p
    return lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def build(lib, nets_):
    pk = rvegen.pack(nets_)
    n = len(nets_)
    arrs = [np.ascontiguousarray(pk.node_off, np.int64), np.ascontiguousarray(pk.X, np.float64),
            np.ascontiguousarray(pk.fiber_off, np.int64), np.ascontiguousarray(pk.conn, np.int32),
            np.ascontiguousarray(pk.L0, np.float64), np.ascontiguousarray(pk.EA, np.float64),
            np.ascontiguousarray(pk.B, np.float64), np.ascontiguousarray(pk.is_boundary, np.uint8)]
    sizes = np.zeros(6, np.int64)
    rc = lib.shim_build(C.c_int64(n), *[_ptr(a) for a in arrs], _ptr(sizes))
    if rc != 0:
        return rc, lib.shim_error().decode()
    nfa, nfb, ncsr_len, nnodes, nfree, pruned = (int(x) for x in sizes)
    meta = np.zeros((n, 8), np.int32)
    fa = np.zeros((max(nfa, 1), 7))
    fij = np.zeros(max(nfa, 1), np.uint32)
    csr = np.zeros(max(ncsr_len, 1), np.uint16)
    ncsr = np.zeros(max(nnodes, 1), np.uint32)
    ncap = np.zeros(max(nnodes, 1), np.float32)
    fid = np.zeros(max(nfree, 1), np.int32)
    nord = np.zeros(max(nnodes, 1), np.uint16)
    lib.shim_meta(_ptr(meta))
    lib.shim_fa(_ptr(fa))
    lib.shim_fij(_ptr(fij))
    lib.shim_csr(_ptr(csr))
    lib.shim_ncsr(_ptr(ncsr))
    lib.shim_ncap(_ptr(ncap))
    lib.shim_free_ids(_ptr(fid))
    lib.shim_nord(_ptr(nord))
    return 0, dict(meta=meta, fa=fa, fij=fij, csr=csr, ncsr=ncsr, ncap=ncap, fid=fid, nord=nord, pruned=pruned)


def wavefronts(idx):
    """16-byte shared loads of a warp: 4 phases of 8 lanes; different rows
    whose indices agree mod 8 in one phase are served one after another."""
    w = 0
    for ph in range(4):
        lanes = [x for x in idx[8 * ph:8 * ph + 8] if x >= 0]
        if lanes:
            cls = {}
            for x in set(lanes):
                cls.setdefault(x % 8, set()).add(x)
            w += max(len(v) for v in cls.values())
    return w


def check_rve(T, r, net):
    nf, na, nb, node_off, fa_off, fb_off, csr_off, csr_len = (int(x) for x in T["meta"][r])
    conn = np.asarray(net.conn, np.int64)
    kept, free = prune(conn, net.is_boundary)
    # free nodes: the oracle's kept free set, in input order
    fid = T["fid"][node_off:node_off + nf]
    assert list(fid) == list(np.nonzero(free)[0])
    loc = -np.ones(net.X.shape[0], np.int64)
    loc[fid] = np.arange(nf)
    # active and boundary fibers: the oracle's kept fibers with >= 1 / 0 free ends
    c = conn[kept]
    act = free[c[:, 0]] | free[c[:, 1]]
    assert na == int(act.sum()) and nb == int((~act).sum())
    want = sorted((int(i), int(j), round(float(l0), 12)) for (i, j), l0 in zip(c[act], net.L0[kept][act]))
    fa = T["fa"][fa_off:fa_off + na]
    ij = T["fij"][fa_off:fa_off + na].astype(np.int64)
    ii, jj = ij & 0xFFFF, ij >> 16
    got = []
    for e in range(na):
        gi = int(fid[ii[e]]) if ii[e] < nf else None
        gj = int(fid[jj[e]]) if jj[e] < nf else None
        # a boundary end reads the zero slot nf; recover it from the chord
        X = net.X
        if gi is None:
            cand = [int(a) for (a, b) in c[act] if b == gj and np.allclose(X[gj] - X[a], fa[e, :3], atol=1e-14)]
            gi = cand[0]
        if gj is None:
            cand = [int(b) for (a, b) in c[act] if a == gi and np.allclose(X[b] - X[gi], fa[e, :3], atol=1e-14)]
            gj = cand[0]
        assert np.allclose(net.X[gj] - net.X[gi], fa[e, :3], atol=1e-14)
        assert fa[e, 6] == 0.5 / (fa[e, 3] * fa[e, 3])
        got.append((gi, gj, round(float(fa[e, 3]), 12)))
    assert sorted(got) == want
    # CSR: every active fiber at each free end once, with the end's flag; runs
    # padded to a multiple of 4 with the zero slot na, 8-byte aligned
    assert csr_off % 4 == 0
    seen = np.zeros(na, np.int64)
    csr = T["csr"][csr_off:csr_off + csr_len].astype(np.int64)
    for a in range(nf):
        w = int(T["ncsr"][node_off + a])
        begin, cnt = w >> 8, w & 0xFF
        assert begin % 4 == 0 and cnt % 4 == 0 and cnt >= 4
        run = csr[begin:begin + cnt]
        lmin = np.inf
        for x in run:
            e, is_j = x >> 1, x & 1
            if e == na:
                assert is_j == 0
                continue
            assert (jj[e] if is_j else ii[e]) == a
            seen[e] += 1
            lmin = min(lmin, fa[e, 3])
        assert T["ncap"][node_off + a] == np.float32(0.1 * lmin)
    assert (seen == (ii < nf).astype(int) + (jj < nf).astype(int)).all()
    # modelled bank conflicts of the two gathers the kernels issue
    fw = fi = 0
    for e0 in range(0, na, 32):
        a_ = list(ii[e0:e0 + 32]) + [-1] * (32 - len(ii[e0:e0 + 32]))
        b_ = list(jj[e0:e0 + 32]) + [-1] * (32 - len(jj[e0:e0 + 32]))
        fw += wavefronts(a_) + wavefronts(b_)
        fi += 8
    return fw / max(fi, 1)


def test_uniform_networks(shim):
    nets_, _ = rvegen.config_uniform(4)
    rc, T = build(shim, nets_)
    assert rc == 0
    ratios = [check_rve(T, r, n) for r, n in enumerate(nets_)]
    # the bank-aware fiber order keeps the H gathers near one wavefront per phase
    assert max(ratios) <= 1.3, ratios


def test_uneven_and_pruned_networks(shim):
    nets_, _ = rvegen.config_uneven(6, side_hi=9)
    hand = [tnets.tiny("one"), tnets.tiny("two"), tnets.tiny("three"), tnets.lattice(3)]
    # a dangling chain and an isolated island that pruning removes
    d = tnets.lattice(3, p=0.8, jitter=0.2, seed=5)
    X = np.vstack([d.X, [[0.05, 0.05, 0.05], [0.08, 0.02, 0.0], [0.3, 0.3, 0.3], [0.32, 0.3, 0.3]]])
    n0 = d.X.shape[0]
    interior = int(np.nonzero(d.is_boundary == 0)[0][0])
    extra = np.array([[interior, n0], [n0, n0 + 1], [n0 + 2, n0 + 3]])
    conn = np.vstack([d.conn, extra]).astype(np.int32)
    L0 = np.linalg.norm(X[conn[:, 1]] - X[conn[:, 0]], axis=1)
    nb = np.concatenate([d.is_boundary, np.zeros(4, np.uint8)])
    E = conn.shape[0]
    dang = rvegen.Network(X=X, conn=conn, L0=L0, EA=np.ones(E), B=np.full(E, 10.0), is_boundary=nb, V0=1.0)
    all_nets = list(nets_) + hand + [dang]
    rc, T = build(shim, all_nets)
    assert rc == 0
    for r, n in enumerate(all_nets):
        check_rve(T, r, n)
    assert T["pruned"] >= 3


def test_invalid_input_is_rejected(shim):
    net = tnets.lattice(3)
    bad = rvegen.Network(X=net.X, conn=np.vstack([net.conn, [[0, 10_000]]]).astype(np.int32),
                         L0=np.concatenate([net.L0, [1.0]]), EA=np.concatenate([net.EA, [1.0]]),
                         B=np.concatenate([net.B, [1.0]]), is_boundary=net.is_boundary, V0=1.0)
    rc, msg = build(shim, [bad])
    assert rc == -1 and "out of range" in msg


def node_rank(q, t, nt):
    """Position of thread t's q-th node in the decreasing-degree order (the
    snake dealing of the node-centric kernels)."""
    return (q + 1) * nt - 1 - t if q & 1 else q * nt + t


def test_degree_order_and_node_dealing(shim):
    """The node-centric kernels deal free nodes to threads in decreasing-degree
    order: the order is a permutation of the free nodes sorted by decreasing
    degree (ties by index), the snake dealing gives every node exactly one
    (thread, slot), and it balances each thread's total degree."""
    nets_, _ = rvegen.config_uniform(3)
    nets_ += list(rvegen.config_uneven(3, side_hi=11)[0])
    rc, T = build(shim, nets_)
    assert rc == 0
    for r in range(len(nets_)):
        nf, na, _, node_off, _, _, csr_off, _ = (int(x) for x in T["meta"][r])
        csr = T["csr"][csr_off:]
        deg = np.zeros(nf, int)
        for a in range(nf):
            w = int(T["ncsr"][node_off + a])
            run = csr[w >> 8:(w >> 8) + (w & 0xff)].astype(int)
            deg[a] = int(((run >> 1) < na).sum())
        order = T["nord"][node_off:node_off + nf].astype(int)
        assert sorted(order.tolist()) == list(range(nf))
        assert (np.diff(deg[order]) <= 0).all()
        for k in range(nf - 1):  # ties by index
            if deg[order[k]] == deg[order[k + 1]]:
                assert order[k] < order[k + 1]
        for nt in (64, 128, 256):
            npt = max(1, -(-nf // nt))
            npt = 1 if npt <= 1 else (2 if npt <= 2 else 4)
            if nf > nt * npt:
                continue
            seen = set()
            load = np.zeros(nt, int)
            for t in range(nt):
                for q in range(npt):
                    k = node_rank(q, t, nt)
                    if k < nf:
                        assert k not in seen
                        seen.add(k)
                        load[t] += deg[order[k]]
            assert seen == set(range(nf))
            if npt == 2 and nf == 2 * nt:
                # pairs of a high and a low degree: the spread of the loads is at
                # most the spread of the degrees
                assert load.max() - load.min() <= deg.max() - deg.min()
