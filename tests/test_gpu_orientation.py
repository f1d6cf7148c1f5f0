"""Parity of the orientation-tensor kernel (Sec. 4, Sec. 5) against the
oracle's definition evaluated at the same positions."""
import numpy as np
import pytest

import rvegen
from oracle.newton import solve_network
from oracle.orientation import orientation_tensor, p2
from tests import nets

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


@pytest.mark.parametrize("precision", ["mixed", "fp64", "plain"])
def test_matches_oracle_at_gpu_positions(rve, precision):
    prec = {"mixed": rve.RVE_PREC_MIXED, "fp64": rve.RVE_PREC_BATCHED_F64, "plain": rve.RVE_PREC_PLAIN_F64}[precision]
    nets_, Fs = rvegen.config_uneven(12, side_hi=9)
    b = rve.RveBatch(rvegen.pack(nets_), precision=prec, tol=1e-8)
    Fd = _F(Fs)
    b.solve(Fd)
    om = b.orientation(Fd).cpu().numpy()
    for k, net in enumerate(nets_):
        x = b.positions(k, Fs[k], net.n_nodes)
        ref = orientation_tensor(x, net.conn, net.is_boundary)
        assert np.abs(om[k] - ref).max() <= 2e-6, (k, np.abs(om[k] - ref).max())
        assert abs(np.trace(om[k]) - 1.0) <= 1e-6 and np.allclose(om[k], om[k].T)
    b.close()


def test_before_any_solve_is_affine_and_lattice_closed_form(rve):
    net = nets.lattice(5)
    F = nets.F_tension_shear()
    b = rve.RveBatch(rvegen.pack([net]), precision=rve.RVE_PREC_MIXED)
    om0 = b.orientation(_F(F[None])).cpu().numpy()[0]  # no solve yet: x = F X
    ref = np.zeros((3, 3))
    for a in range(3):
        t = F[:, a] / np.linalg.norm(F[:, a])
        ref += np.outer(t, t) / 3.0
    assert np.abs(om0 - ref).max() <= 1e-6
    b.solve(_F(F[None]))
    om1 = b.orientation(_F(F[None])).cpu().numpy()[0]  # the lattice's equilibrium is affine
    assert np.abs(om1 - ref).max() <= 1e-6
    b.close()


def test_p2_after_solve_matches_oracle_solve(rve):
    # a fully bonded jittered lattice is rigid: its equilibrium positions are
    # unique.  (On a sub-isostatic network the unloaded parts can sit anywhere
    # along their floppy modes without changing sigma, so Omega is compared
    # at the same positions instead, as above.)
    net = nets.lattice(6, p=1.0, jitter=0.3, seed=4)
    F = rvegen.random_F(rvegen.Stream(17))
    sol = solve_network(net, F)
    b = rve.RveBatch(rvegen.pack([net]), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-11)
    s, _, _ = b.solve(_F(F[None]))
    assert np.linalg.norm(s.cpu().numpy().reshape(3, 3) - sol.sigma) <= 1e-8 * np.linalg.norm(sol.sigma)
    om = b.orientation(_F(F[None])).cpu().numpy()[0]
    om_o = orientation_tensor(sol.x, net.conn, net.is_boundary)
    for a in ([1, 0, 0], [0, 1, 0], [0.2, 0.3, 0.9]):
        assert abs(p2(om, a) - p2(om_o, a)) <= 3e-6
    b.close()
