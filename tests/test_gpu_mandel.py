"""Parity of the six-solve material tangent (Sec. 3.2) on the GPU against
the oracle's implementation of the same procedure."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import rvegen
from oracle.mandel import from_mandel2, from_mandel4, mandel_tangent, polar, to_mandel2, to_mandel4
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _args(net):
    return net.X, net.conn, net.L0, net.EA, net.B, net.is_boundary


def oracle_at_gpu_state(b, k, net, F, sig_gpu, h):
    """The oracle's six-solve tangent at the equilibrium the GPU reached.
    Same minimum as the oracle's own cold solve: that one.  Otherwise (a
    sub-isostatic network can hold several stable equilibria) the oracle
    starts from the GPU's base positions, rotated to U; its base solve must
    be stable and reproduce the GPU's sigma."""
    C_o = mandel_tangent(*_args(net), F, h=h, tol=1e-12)
    if rel(sig_gpu, C_o[0]) <= 1e-9:
        return C_o
    R, U = polar(F)
    x = b.positions(k, F, net.n_nodes) @ R  # x_U = R^T x_F per node
    C_o = mandel_tangent(*_args(net), F, h=h, tol=1e-12, h0_U=x - net.X @ U.T)
    assert rel(sig_gpu, C_o[0]) <= 1e-9, rel(sig_gpu, C_o[0])
    print("  RVE %d: other stable minimum than the oracle's cold solve" % k)
    return C_o


def _case(seed=9):
    net = nets.lattice(5, p=0.7, jitter=0.3, seed=seed, B=8.0)
    F = rvegen.random_F(rvegen.Stream(31 + seed))
    return net, F


@pytest.mark.parametrize("seed", [9, 12])
def test_fp64_matches_oracle_single(rve, seed):
    net, F = _case(seed)
    h = 1e-5
    b = rve.RveBatch(rvegen.pack([net]), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-12)
    sig, C, st = b.tangent_mandel(_F(F[None]), h=h)
    C = C.cpu().numpy()[0]
    assert int(st[0]) == rve.RVE_STATUS_CONVERGED
    sig_o, A_o, C_o = oracle_at_gpu_state(b, 0, net, F, sig.cpu().numpy().reshape(3, 3), h)
    print("C rel err FP64: %.2e" % rel(C, C_o))
    assert rel(C, C_o) <= 1e-4
    b.close()


def test_mixed_precision_accuracy(rve):
    net = nets.lattice(5, p=0.7, jitter=0.3, seed=9, B=8.0)
    F = rvegen.random_F(rvegen.Stream(31))  # a case whose equilibrium the oracle and the DR share
    h = 1e-3
    sig_o, A_o, C_o = mandel_tangent(*_args(net), F, h=h, tol=1e-12)
    b = rve.RveBatch(rvegen.pack([net]), precision=rve.RVE_PREC_MIXED, tol=1e-7)
    sig, C, st = b.tangent_mandel(_F(F[None]), h=h)
    assert int(st[0]) == rve.RVE_STATUS_CONVERGED
    assert rel(sig.cpu().numpy().reshape(3, 3), sig_o) <= 1e-4
    e = rel(C.cpu().numpy()[0], C_o)
    print("C rel err mixed (h=1e-3): %.2e" % e)
    # FP32 stresses differenced over h = 1e-3
    assert e <= 2e-2
    b.close()


def test_uneven_batch_each_rve_matches_oracle(rve):
    nets_, Fs = rvegen.config_uneven(6, side_hi=8)
    h = 1e-5
    b = rve.RveBatch(rvegen.pack(nets_), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-12, max_iter=2_000_000)
    sig, C, st = b.tangent_mandel(_F(Fs), h=h)
    C = C.cpu().numpy()
    st = st.cpu().numpy()
    sig = sig.cpu().numpy().reshape(-1, 3, 3)
    for k in range(3):  # the oracle side is six Newton solves per RVE
        if st[k] != rve.RVE_STATUS_CONVERGED:
            continue
        _, _, C_o = oracle_at_gpu_state(b, k, nets_[k], Fs[k], sig[k], h)
        print("RVE %d: C rel err %.2e" % (k, rel(C[k], C_o)))
        assert rel(C[k], C_o) <= 1e-3
    assert (st == rve.RVE_STATUS_CONVERGED).mean() >= 0.8
    b.close()


def test_consistent_with_central_difference_tangent(rve):
    """A : dE from the six-solve route equals dPi/dF : dF from the GPU's own
    nine-direction central-difference dsigma/dF (different solves)."""
    net, F = _case(12)
    b = rve.RveBatch(rvegen.pack([net]), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-12)
    sig, Cm, _ = b.tangent_mandel(_F(F[None]), h=1e-6)
    sig2, D, _ = b.tangent(_F(F[None]), h=1e-5)
    sig = sig.cpu().numpy().reshape(3, 3)
    D = D.cpu().numpy().reshape(9, 9)
    C4 = from_mandel4(Cm.cpu().numpy()[0])
    J = np.linalg.det(F)
    Fi = np.linalg.inv(F)
    # pull C back to A: A_ijrs = J Fi_im Fi_jn C_mnpq Fi_rp Fi_sq
    A = to_mandel4(J * np.einsum("im,jn,mnpq,rp,sq->ijrs", Fi, Fi, C4, Fi, Fi))
    rng = np.random.default_rng(3)
    for _ in range(3):
        dF = rng.normal(size=(3, 3)) * 0.5
        dsig = (D @ dF.ravel()).reshape(3, 3)
        dJ = J * np.trace(Fi @ dF)
        dFi = -Fi @ dF @ Fi
        dPi = dJ * Fi @ sig @ Fi.T + J * (dFi @ sig @ Fi.T + Fi @ dsig @ Fi.T + Fi @ sig @ dFi.T)
        dE = 0.5 * (dF.T @ F + F.T @ dF)
        lhs = from_mandel2(A @ to_mandel2(dE))
        assert np.abs(lhs - dPi).max() <= 2e-4 * np.abs(dPi).max()
    b.close()


def test_objectivity_of_C(rve):
    net, F = _case(9)
    R = Rotation.from_rotvec([0.4, -0.2, 0.1]).as_matrix()
    b = rve.RveBatch(rvegen.pack([net, net]), precision=rve.RVE_PREC_BATCHED_F64, tol=1e-12)
    sig, C, st = b.tangent_mandel(_F(np.stack([F, R @ F])), h=1e-5)
    C = C.cpu().numpy()
    C_rot = to_mandel4(np.einsum("ma,nb,abcd,pc,qd->mnpq", R, R, from_mandel4(C[0]), R, R))
    assert rel(C[1], C_rot) <= 1e-6
    b.close()
