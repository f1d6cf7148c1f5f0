"""Pins of the orientation tensor and P2 (Sec. 4, Sec. 5) against closed
forms, a direct angle average and invariants."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

import rvegen
from oracle.newton import solve_network
from oracle.orientation import orientation_tensor, p2
from tests import nets


def test_regular_lattice_closed_form():
    net = nets.lattice(4)
    F = nets.F_tension_shear()
    x = net.X @ F.T  # the regular lattice's equilibrium is affine
    om = orientation_tensor(x, net.conn, net.is_boundary)
    ref = np.zeros((3, 3))
    for a in range(3):
        t = F[:, a] / np.linalg.norm(F[:, a])
        ref += np.outer(t, t) / 3.0  # equal bond counts along the three axes
    assert np.allclose(om, ref, atol=1e-15)
    assert math.isclose(p2(om, [1, 0, 0]), 0.5 * (3 * ref[0, 0] - 1), rel_tol=1e-14)
    # undeformed: isotropic in the lattice's axes, P2 = 0 along each axis
    om0 = orientation_tensor(net.X, net.conn, net.is_boundary)
    assert np.allclose(om0, np.eye(3) / 3, atol=1e-15)
    assert abs(p2(om0, [0, 0, 1])) < 1e-15


def test_p2_equals_direct_angle_average():
    net = nets.lattice(5, p=0.7, jitter=0.3, seed=2)
    F = rvegen.random_F(rvegen.Stream(7))
    sol = solve_network(net, F)
    om = orientation_tensor(sol.x, net.conn, net.is_boundary)
    from oracle.network import prune
    kept, _ = prune(np.asarray(net.conn, np.int64), net.is_boundary)
    c = net.conn[kept]
    a = np.array([0.3, -0.5, 0.8])
    a /= np.linalg.norm(a)
    vals = []
    for i, j in c:
        d = sol.x[j] - sol.x[i]
        theta = math.acos(max(-1.0, min(1.0, d @ a / np.linalg.norm(d))))
        vals.append(0.5 * (3 * math.cos(theta) ** 2 - 1))
    assert math.isclose(p2(om, a), math.fsum(vals) / len(vals), rel_tol=1e-12, abs_tol=1e-14)
    assert math.isclose(np.trace(om), 1.0, rel_tol=1e-14)
    assert np.allclose(om, om.T)


def test_extremes_and_rotation():
    # every fiber along e1: P2 = 1 along e1, -1/2 across it
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [0, 1.0, 0], [1.0, 1.0, 0], [2.0, 1.0, 0]])
    conn = np.array([[0, 1], [1, 2], [3, 4], [4, 5]])
    nb = np.array([1, 0, 1, 1, 0, 1], np.uint8)
    om = orientation_tensor(X, conn, nb)
    assert math.isclose(p2(om, [1, 0, 0]), 1.0) and math.isclose(p2(om, [0, 1, 0]), -0.5)
    R = Rotation.from_rotvec([0.2, 0.4, -0.3]).as_matrix()
    omr = orientation_tensor(X @ R.T, conn, nb)
    assert np.allclose(omr, R @ om @ R.T, atol=1e-15)


def test_pruned_fibers_do_not_count():
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [1.0, 0.5, 0.3]])
    conn = np.array([[0, 1], [1, 2], [1, 3]])  # node 3 is a dangling free node
    nb = np.array([1, 0, 1, 0], np.uint8)
    om = orientation_tensor(X, conn, nb)
    assert np.allclose(om, np.diag([1.0, 0, 0]))
