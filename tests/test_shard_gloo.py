"""Multi-rank path on CPU: two gloo ranks split a batch of RVEs by cost,
each solves its own range (oracle on the host), and the gathered stresses
equal a single-process solve; the partition covers every RVE once."""
import os
import socket

import numpy as np
import pytest

import rvegen


def test_partition_properties():
    import importlib.util
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2306_09427_gb300",
                        "shard.py")
    spec = importlib.util.spec_from_file_location("_shard", path)
    shard = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(shard)
    rng = np.random.default_rng(1)
    for world in (1, 2, 3, 8):
        costs = rng.uniform(1, 100, 257)
        parts = shard.partition(costs, world)
        assert parts[0][0] == 0 and parts[-1][1] == 257
        assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
        loads = [costs[a:b].sum() for a, b in parts]
        assert max(loads) - min(loads) <= 2 * costs.max()
    assert shard.partition([], 3) == [(0, 0)] * 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import importlib.util
    import sys

    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    spec = importlib.util.spec_from_file_location("_shard", os.path.join(root, "paper_2306_09427_gb300", "shard.py"))
    shard = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(shard)
    import rvegen as g
    from oracle.newton import solve_network
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    nets, Fs = g.config_uniform(6, side=4)
    costs = [n.n_fibers for n in nets]
    a, b = shard.partition(costs, world)[rank]
    local = np.zeros((6, 9))
    for k in range(a, b):
        local[k] = solve_network(nets[k], Fs[k]).sigma.ravel()
    import torch
    t = torch.tensor(local)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)  # ranges are disjoint: the sum gathers them
    n = torch.tensor([float(b - a)])
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    if rank == 0:
        q.put((t.numpy(), float(n.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    import multiprocessing as mp

    from oracle.newton import solve_network
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    sig, n = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    nets, Fs = rvegen.config_uniform(6, side=4)
    ref = np.stack([solve_network(nets[k], Fs[k]).sigma.ravel() for k in range(6)])
    assert n == 6.0
    assert np.abs(sig - ref).max() <= 1e-13 * np.abs(ref).max()
