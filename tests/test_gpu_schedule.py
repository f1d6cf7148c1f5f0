"""Batch scheduling: CUDA-graph replay and the autotuner (GPU)."""
import numpy as np
import pytest

import rvegen

pytestmark = pytest.mark.gpu


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


def test_graph_replay_matches_plain_launches(rve):
    import torch
    nets, Fs = rvegen.config_uneven(48, side_hi=11)
    pk = rvegen.pack(nets)
    ref = rve.RveBatch(pk, precision=rve.RVE_PREC_MIXED)
    gb = rve.RveBatch(pk, precision=rve.RVE_PREC_MIXED, graphs=1)
    Fd = _F(Fs)
    sig = torch.empty((48, 9), dtype=torch.float64, device="cuda:0")
    it = torch.empty(48, dtype=torch.int32, device="cuda:0")
    st = torch.empty(48, dtype=torch.int32, device="cuda:0")
    s0, i0, _ = ref.solve(Fd)
    stream = torch.cuda.Stream()  # graphs need a created stream
    torch.cuda.synchronize()
    for _ in range(3):  # first call runs and records, the others replay
        gb.solve(Fd, sigma=sig, iters=it, status=st, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(sig, s0) and torch.equal(it, i0)
    F2 = Fs + 0.003 * np.eye(3)
    Fd.copy_(_F(F2))  # same pointer, new contents: the replay reads them
    torch.cuda.synchronize()
    gb.solve(Fd, sigma=sig, iters=it, status=st, stream=stream)
    s2, _, _ = ref.solve(_F(F2))
    torch.cuda.synchronize()
    assert torch.equal(sig, s2)
    ref.close()
    gb.close()


def test_autotuner_keeps_results(rve):
    nets, Fs = rvegen.config_uneven(96, side_hi=12)
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED)
    Fd = _F(Fs)
    s0, _, st0 = b.solve(Fd)
    before_bins = b.bins()
    t_before, t_after = b.autotune(Fd, reps=1)
    after_bins = b.bins()
    assert t_after <= t_before * 1.05
    assert len(after_bins) == len(before_bins)
    for x in after_bins:
        assert x["threads"] in (64, 128, 256, 512, 1024) and x["check_every"] in (25, 50, 100) or x["n_rve"] == 0
    s1, _, st1 = b.solve(Fd)
    s0, s1 = s0.cpu().numpy(), s1.cpu().numpy()
    assert (st1.cpu().numpy() == 0).all()
    e = np.linalg.norm(s1 - s0, axis=1) / np.linalg.norm(s0, axis=1)
    print("autotune: %.2f -> %.2f ms; sigma change max %.2e" % (t_before, t_after, e.max()))
    assert (e <= 1e-4).mean() >= 0.95
    b.close()


def test_kernel_timing_records_every_launch(rve):
    import torch
    nets, Fs = rvegen.config_uneven(40, side_hi=11)
    b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, graphs=1)
    Fd = _F(Fs)
    stream = torch.cuda.Stream()
    s0, _, _ = b.solve(Fd, stream=stream)
    n_bins = sum(1 for x in b.bins() if x["n_rve"] > 0)
    b.set_kernel_timing(True)
    for _ in range(3):
        s1, _, _ = b.solve(Fd, stream=stream)  # timing forces uncaptured launches
    t = b.last_kernel_ms()
    assert t.shape == (3 * n_bins,) and (t > 0).all() and np.isfinite(t).all()
    torch.cuda.synchronize()
    assert torch.equal(s0, s1)
    b.set_kernel_timing(False)
    assert b.last_kernel_ms().shape == (0,)
    b.solve(Fd, stream=stream)
    assert b.last_kernel_ms().shape == (0,)
    b.close()


def test_costliest_rves_on_their_own_sms_keep_results(rve):
    """A whole-batch solve of a large resident bin launches the head of its
    longest-first list on SMs of its own (high-priority stream); a subset
    solve of the same RVEs runs one launch.  Same kernel and arithmetic, so
    the stresses and iteration counts are identical, with and without a
    captured graph."""
    import torch
    nets, Fs = rvegen.config_uniform(512, side=8)
    Fd = _F(Fs)
    for graphs in (0, 1):
        b = rve.RveBatch(rvegen.pack(nets), precision=rve.RVE_PREC_MIXED, graphs=graphs)
        assert len(b.bins()) in (0, 1)
        stream = torch.cuda.Stream()
        s_all, i_all, st = b.solve(Fd, stream=stream)   # learns the per-RVE cost
        s_all, i_all, st = b.solve(Fd, stream=stream)   # longest first, costliest on their own SMs
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == rve.RVE_STATUS_CONVERGED).all()
        ids = np.arange(512)
        s_sub, i_sub, _ = b.solve_subset(ids, Fd, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(s_all, s_sub) and torch.equal(i_all, i_sub)
        b.close()
