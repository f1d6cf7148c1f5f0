"""Pins of the FP64 oracle against closed forms, invariants, brute force and
an independent linear-elastic solve (none of them re-uses the oracle's
Newton path)."""
import math

import numpy as np
import pytest
import scipy.optimize as so
from scipy.spatial.transform import Rotation

import rvegen
from oracle.fiber_law import axial_force
from oracle.network import internal_forces, prune, stiffness_free, total_energy
from oracle.newton import solve, solve_network
from tests import nets


def _closed_form_fiber_stress(Xa, Xb, F, EA, B, V0):
    d = F @ (np.asarray(Xb) - np.asarray(Xa))
    L0 = np.linalg.norm(np.asarray(Xb) - np.asarray(Xa))
    l = np.linalg.norm(d)
    N = (EA / B) * math.expm1(B * 0.5 * (l * l / (L0 * L0) - 1.0))
    return N * np.outer(d, d) / l / (np.linalg.det(F) * V0)


def test_single_fiber_uniaxial():
    # one boundary-to-boundary fiber along e1, F = I + 0.1 e1 (x) e1:
    # l = 1.1 L0, eps_G = 0.105, sigma_11 = N l / v with v = det F V0 = 1.1
    X = np.array([[-0.25, 0, 0], [0.25, 0, 0]])
    F = rvegen.F_UNIAXIAL_10
    s = solve(X, [[0, 1]], [0.5], [1.0], [10.0], [1, 1], F)
    N = (math.exp(1.05) - 1.0) / 10.0
    assert abs(s.sigma[0, 0] - N * 0.55 / 1.1) < 1e-15
    assert np.abs(s.sigma - np.diag([s.sigma[0, 0], 0, 0])).max() == 0.0


def test_single_fiber_general_direction():
    rng = np.random.default_rng(3)
    Xa, Xb = rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.5, 0.5, 3)
    F = np.eye(3) + rng.uniform(-0.1, 0.1, (3, 3))
    L0 = np.linalg.norm(Xb - Xa)
    s = solve(np.stack([Xa, Xb]), [[0, 1]], [L0], [1.7], [7.0], [1, 1], F, V0=0.8)
    ref = _closed_form_fiber_stress(Xa, Xb, F, 1.7, 7.0, 0.8)
    assert np.abs(s.sigma - ref).max() <= 1e-14 * np.abs(ref).max()


def _lattice_closed_form(n, F, EA=1.0, B=10.0):
    # regular lattice, every bond kept: opposite bonds balance at every node,
    # so x = F X is the equilibrium and sigma sums n^2(n-1) bonds per axis.
    s = 1.0 / (n - 1)
    sig = np.zeros((3, 3))
    for k in range(3):
        g = F[:, k] * s
        l = np.linalg.norm(g)
        N = (EA / B) * math.expm1(B * 0.5 * (l * l / (s * s) - 1.0))
        sig += n * n * (n - 1) * N * np.outer(g, g) / l
    return sig / np.linalg.det(F)


@pytest.mark.parametrize("n", [3, 5])
def test_affine_regular_lattice(n):
    net = nets.lattice(n)
    F = nets.F_tension_shear()
    s = solve_network(net, F)
    ref = _lattice_closed_form(n, F)
    assert np.abs(s.sigma - ref).max() <= 1e-13 * np.abs(ref).max()
    assert s.newton_iters == 0
    assert s.stable


def test_rigid_rotation_zero_stress():
    net = nets.lattice(5, p=0.7, jitter=0.3, seed=11)
    R = Rotation.from_rotvec([0.3, -0.8, 0.5]).as_matrix()
    s = solve_network(net, R)
    assert np.abs(s.sigma).max() < 1e-14
    assert s.newton_iters == 0


def _jittered(seed, n=5, p=0.7, B=10.0):
    return nets.lattice(n, p=p, jitter=0.3, seed=seed, B=B)


def test_symmetry_objectivity_hill_mandel():
    net = _jittered(21)
    F = rvegen.random_F(rvegen.Stream(99))
    R, U = np.linalg.qr(F)  # any rotation will do for objectivity
    R = R * np.sign(np.linalg.det(R))
    Q = Rotation.from_rotvec([1.1, 0.2, -0.4]).as_matrix()
    s1 = solve_network(net, F)
    s2 = solve_network(net, Q @ F)
    assert s1.converged and s2.converged
    scale = np.abs(s1.sigma).max()
    assert np.abs(s1.sigma - s1.sigma.T).max() <= 1e-12 * scale
    assert np.abs(s2.sigma - Q @ s1.sigma @ Q.T).max() <= 1e-10 * scale
    # Hill-Mandel: fiber virial equals boundary-reaction virial at equilibrium
    assert np.abs(s1.sigma - s1.sigma_boundary).max() <= 1e-9 * scale
    # interior force residual
    conn = net.conn[s1.kept]
    f = internal_forces(s1.x, conn, net.L0[s1.kept], net.EA[s1.kept], net.B[s1.kept])
    assert np.abs(f[s1.free]).max() < 1e-10


def test_translation_invariance():
    net = _jittered(5)
    F = rvegen.random_F(rvegen.Stream(7))
    s1 = solve_network(net, F)
    net2 = rvegen.Network(X=net.X + np.array([3.0, -1.0, 0.5]), conn=net.conn, L0=net.L0, EA=net.EA,
                          B=net.B, is_boundary=net.is_boundary)
    s2 = solve_network(net2, F)
    assert np.abs(s1.sigma - s2.sigma).max() <= 1e-11 * np.abs(s1.sigma).max()


def test_prune_rules_on_hand_graph():
    # nodes 0,1 boundary; 2-3-4 chain off node 2 (free, attached to both
    # boundaries); 5-6-7 floating triangle; 8 isolated
    conn = np.array([[0, 2], [2, 1], [2, 3], [3, 4], [5, 6], [6, 7], [7, 5], [0, 1]])
    nb = np.array([1, 1, 0, 0, 0, 0, 0, 0, 0], np.uint8)
    kept, free = prune(conn, nb)
    assert kept.tolist() == [True, True, False, False, False, False, False, True]
    assert free.tolist() == [False, False, True, False, False, False, False, False, False]


def test_pruned_parts_do_not_change_stress():
    net = _jittered(8)
    F = rvegen.random_F(rvegen.Stream(8))
    s1 = solve_network(net, F)
    # attach a dangling two-fiber chain to a kept free node and add a floating triangle
    i = int(np.nonzero(s1.free)[0][0])
    N0 = net.X.shape[0]
    extra_X = np.array([net.X[i] + [0.05, 0.02, 0.01], net.X[i] + [0.09, 0.05, 0.0],
                        [0.1, 0.1, 0.1], [0.15, 0.1, 0.1], [0.1, 0.16, 0.12]])
    extra_c = np.array([[i, N0], [N0, N0 + 1], [N0 + 2, N0 + 3], [N0 + 3, N0 + 4], [N0 + 4, N0 + 2]])
    X = np.vstack([net.X, extra_X])
    conn = np.vstack([net.conn, extra_c])
    L0 = np.concatenate([net.L0, np.linalg.norm(X[extra_c[:, 1]] - X[extra_c[:, 0]], axis=1)])
    EA = np.concatenate([net.EA, np.ones(5)])
    B = np.concatenate([net.B, np.full(5, 10.0)])
    nb = np.concatenate([net.is_boundary, np.zeros(5, np.uint8)])
    s2 = solve(X, conn, L0, EA, B, nb, F)
    assert np.abs(s1.sigma - s2.sigma).max() <= 1e-12 * np.abs(s1.sigma).max()


@pytest.mark.parametrize("kind", ["one", "two", "three"])
def test_brute_force_tiny(kind):
    net = nets.tiny(kind, seed=4)
    F = np.array([[1.08, 0.03, -0.02], [0.01, 0.97, 0.04], [0.0, -0.03, 1.05]])
    s = solve_network(net, F)
    assert s.converged and s.stable
    free = np.nonzero(net.is_boundary == 0)[0]
    xb = net.X @ F.T

    def energy(z):
        x = xb.copy()
        x[free] = z.reshape(-1, 3)
        return total_energy(x, net.conn.astype(np.int64), net.L0, net.EA, net.B)

    def residual(z):
        x = xb.copy()
        x[free] = z.reshape(-1, 3)
        return internal_forces(x, net.conn.astype(np.int64), net.L0, net.EA, net.B)[free].ravel()

    # independent routes: energy minimisation (BFGS) and root finding (least squares)
    best = None
    rng = np.random.default_rng(0)
    for trial in range(4):
        z0 = xb[free].ravel() + rng.normal(0, 0.01, 3 * free.size)
        m = so.minimize(energy, z0, method="BFGS", options=dict(gtol=1e-13, maxiter=5000))
        ls = so.least_squares(residual, m.x, xtol=1e-15, ftol=1e-15, gtol=1e-15)
        if best is None or energy(ls.x) < energy(best):
            best = ls.x
    x = xb.copy()
    x[free] = best.reshape(-1, 3)
    assert np.abs(residual(best)).max() < 1e-11
    assert np.abs(x[free] - s.x[free]).max() < 1e-9
    d = x[net.conn[:, 1]] - x[net.conn[:, 0]]
    l = np.linalg.norm(d, axis=1)
    N = axial_force(0.5 * (l * l / net.L0 ** 2 - 1.0), net.EA, net.B)
    sig = np.einsum("e,ei,ej->ij", N / l, d, d) / np.linalg.det(F)
    assert np.abs(sig - s.sigma).max() <= 1e-9 * np.abs(sig).max()


def test_force_is_minus_energy_gradient_and_tangent_is_force_jacobian():
    net = _jittered(13, B=14.0)
    F = rvegen.random_F(rvegen.Stream(5))
    conn = net.conn.astype(np.int64)
    rng = np.random.default_rng(1)
    x = net.X @ F.T + rng.normal(0, 0.004, net.X.shape)
    free = np.nonzero(net.is_boundary == 0)[0]
    fidx = -np.ones(net.X.shape[0], np.int64)
    fidx[free] = np.arange(free.size)
    f = internal_forces(x, conn, net.L0, net.EA, net.B)
    K = stiffness_free(x, conn, net.L0, net.EA, net.B, fidx, free.size)
    for _ in range(3):
        v = np.zeros_like(x)
        v[free] = rng.normal(size=(free.size, 3))
        h = 1e-6
        dW = (total_energy(x + h * v, conn, net.L0, net.EA, net.B)
              - total_energy(x - h * v, conn, net.L0, net.EA, net.B)) / (2 * h)
        assert abs(dW + np.sum(f * v)) < 1e-6 * max(1.0, abs(dW))
        df = (internal_forces(x + h * v, conn, net.L0, net.EA, net.B)
              - internal_forces(x - h * v, conn, net.L0, net.EA, net.B))[free].ravel() / (2 * h)
        Kv = K @ v[free].ravel()
        assert np.linalg.norm(df + Kv) <= 1e-6 * np.linalg.norm(Kv)


def test_linear_elastic_limit():
    # over-constrained jittered lattice (every bond kept): K0 is positive
    # definite, so the first-order response is the unique linear solve
    net = nets.lattice(4, p=1.0, jitter=0.3, seed=17)
    G = np.array([[0.3, -0.2, 0.5], [0.1, 0.7, -0.4], [-0.6, 0.2, 0.1]])
    delta = 1e-6
    s = solve_network(net, np.eye(3) + delta * G)
    X, conn = net.X, net.conn
    dX = X[conn[:, 1]] - X[conn[:, 0]]
    L0 = np.linalg.norm(dX, axis=1)
    n = dX / L0[:, None]
    k0 = net.EA / L0
    Nn = X.shape[0]
    Kfull = np.zeros((3 * Nn, 3 * Nn))
    for e, (a, b) in enumerate(conn):
        S = k0[e] * np.outer(n[e], n[e])
        for (p, q, sg) in ((a, a, 1), (b, b, 1), (a, b, -1), (b, a, -1)):
            Kfull[3 * p:3 * p + 3, 3 * q:3 * q + 3] += sg * S
    fdof = np.concatenate([[3 * i, 3 * i + 1, 3 * i + 2] for i in np.nonzero(net.is_boundary == 0)[0]])
    bdof = np.setdiff1d(np.arange(3 * Nn), fdof)
    u = (X @ G.T).ravel()
    uf = np.linalg.solve(Kfull[np.ix_(fdof, fdof)], -Kfull[np.ix_(fdof, bdof)] @ u[bdof])
    u[fdof] = uf
    u = u.reshape(-1, 3)
    N1 = k0 * np.einsum("ei,ei->e", n, u[conn[:, 1]] - u[conn[:, 0]])
    sig_lin = np.einsum("e,e,ei,ej->ij", N1, L0, n, n)
    assert np.abs(s.sigma / delta - sig_lin).max() <= 1e-4 * np.abs(sig_lin).max()


def test_load_path_irrelevant_for_unique_minimum():
    net = nets.lattice(4, p=1.0, jitter=0.3, seed=2)
    F = rvegen.random_F(rvegen.Stream(4))
    s1 = solve_network(net, F, increments=1)
    s4 = solve_network(net, F, increments=6)
    assert np.abs(s1.sigma - s4.sigma).max() <= 1e-11 * np.abs(s1.sigma).max()


def test_bad_inputs_rejected():
    with pytest.raises(ValueError):
        solve(np.zeros((2, 3)) + [[0, 0, 0], [1, 0, 0]], [[0, 1]], [1.0], [1.0], [1.0], [1, 1],
              np.diag([1.0, 1.0, -1.0]))
