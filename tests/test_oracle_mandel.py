"""Pins of the oracle's six-solve material tangent (Sec. 3.2) against the
mathematics it must satisfy: dE/dU by finite differences of E(U), the
Mandel matrix the paper prints, a closed form for the affine lattice, an
independent route through central differences of sigma in F, objectivity
of the push-forward, and the major symmetry of a hyperelastic tangent."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle.mandel import (M_tensor, T_mandel, from_mandel2, from_mandel4, mandel_tangent, pk2, polar,
                           push_forward, to_mandel2, to_mandel4)
from tests import nets


def _sym(rng, scale=0.1):
    G = rng.normal(size=(3, 3))
    return scale * (G + G.T)


def _net_args(net):
    return net.X, net.conn, net.L0, net.EA, net.B, net.is_boundary


def test_mandel_maps_preserve_inner_products_and_contractions():
    rng = np.random.default_rng(1)
    a, b = _sym(rng), _sym(rng)
    assert math.isclose(to_mandel2(a) @ to_mandel2(b), np.tensordot(a, b), rel_tol=1e-14)
    assert np.allclose(from_mandel2(to_mandel2(a)), a, atol=1e-15)
    # a tensor with minor symmetries acting on a symmetric tensor
    A = rng.normal(size=(3, 3, 3, 3))
    A = A + A.transpose(1, 0, 2, 3)
    A = A + A.transpose(0, 1, 3, 2)
    lhs = to_mandel4(A) @ to_mandel2(a)
    rhs = to_mandel2(np.einsum("ijkl,kl->ij", A, a))
    assert np.allclose(lhs, rhs, atol=1e-13)
    assert np.allclose(from_mandel4(to_mandel4(A)), A, atol=1e-14)


def test_dE_dU_matches_finite_differences_of_E():
    """M = dE/dU for E = (U U - I)/2: central differences are exact for a quadratic."""
    rng = np.random.default_rng(2)
    U = np.eye(3) + _sym(rng)
    Mm = to_mandel4(M_tensor(U))
    E = lambda V: 0.5 * (V @ V - np.eye(3))
    for _ in range(4):
        D = _sym(rng, 1.0)
        t = 1e-3
        dE = (E(U + t * D) - E(U - t * D)) / (2 * t)
        assert np.allclose(Mm @ to_mandel2(D), to_mandel2(dE), atol=1e-12)


def test_dE_dU_mandel_equals_the_printed_matrix():
    """The 6x6 matrix the paper prints for [M] (Sec. 3.2), entry by entry."""
    rng = np.random.default_rng(3)
    U = np.eye(3) + _sym(rng)
    s = math.sqrt(2.0)
    U11, U22, U33, U12, U13, U23 = U[0, 0], U[1, 1], U[2, 2], U[0, 1], U[0, 2], U[1, 2]
    printed = 0.5 * np.array([
        [2 * U11, 0, 0, 0, s * U13, s * U12],
        [0, 2 * U22, 0, s * U23, 0, s * U12],
        [0, 0, 2 * U33, s * U23, s * U13, 0],
        [0, s * U23, s * U23, U22 + U33, U12, U13],
        [s * U13, 0, s * U13, U12, U11 + U33, U23],
        [s * U12, s * U12, 0, U13, U23, U11 + U22]])
    assert np.allclose(to_mandel4(M_tensor(U)), printed, atol=1e-15)


def test_probing_directions_span_and_keep_U_positive_definite():
    T = T_mandel()
    assert abs(np.linalg.det(T)) > 0.1
    U = np.diag([1.05, 0.97, 1.1])
    for p in range(6):
        assert np.linalg.eigvalsh(U + 1e-4 * from_mandel2(T[:, p])).min() > 0


def test_polar_decomposition():
    rng = np.random.default_rng(4)
    R0 = Rotation.random(random_state=5).as_matrix()
    U0 = np.eye(3) + _sym(rng)
    R, U = polar(R0 @ U0)
    assert np.allclose(R, R0, atol=1e-12) and np.allclose(U, U0, atol=1e-12)


def _affine_lattice_A(n, U, EA=1.0, B=10.0):
    """Closed form dPi/dE for the regular n^3 lattice, whose equilibrium is affine:
    Pi = sum_e g(eps_e) dX dX^T with g = N / l, eps_e = dX^T E dX / L0^2, so
    A_ijkl = sum_e g'(eps_e) dX_i dX_j dX_k dX_l / L0^2 (unit reference volume)."""
    s = 1.0 / (n - 1)
    E = 0.5 * (U.T @ U - np.eye(3))
    A = np.zeros((3, 3, 3, 3))
    for ax in range(3):
        dX = np.zeros(3)
        dX[ax] = s
        eps = dX @ E @ dX / (s * s)
        l = s * math.sqrt(1.0 + 2.0 * eps)
        N = (EA / B) * math.expm1(B * eps)
        dN = EA * math.exp(B * eps)
        dl = s * s / l
        gp = dN / l - N * dl / (l * l)
        A += n * n * (n - 1) * gp * np.einsum("i,j,k,l->ijkl", dX, dX, dX, dX) / (s * s)
    return to_mandel4(A)


@pytest.mark.parametrize("n", [3, 4])
def test_affine_lattice_closed_form(n):
    net = nets.lattice(n)
    U = np.diag([1.05, 1.08, 1.03])
    sig, A, C = mandel_tangent(*_net_args(net), U, h=1e-7)
    ref = _affine_lattice_A(n, U)
    assert np.abs(A - ref).max() <= 1e-5 * np.abs(ref).max()
    # at F = U (no rotation) C is the push-forward of the same A
    assert np.allclose(C, to_mandel4(push_forward(U, from_mandel4(ref))), rtol=0, atol=1e-5 * np.abs(C).max())


def test_independent_route_through_dsigma_dF():
    """A : dE from the six-solve route equals dPi/dF : dF from central
    differences of sigma in F (nine directions, a different set of solves)."""
    net = nets.lattice(4, p=0.8, jitter=0.25, seed=3, B=6.0)
    F = Rotation.from_rotvec([0.2, -0.1, 0.3]).as_matrix() @ np.array(
        [[1.06, 0.02, 0.0], [0.02, 0.98, 0.01], [0.0, 0.01, 1.04]])
    args = _net_args(net)
    sig, A, C = mandel_tangent(*args, F, h=1e-6)
    sig_c, D = oracle.dsigma_dF(*args, F, h=1e-5)
    assert np.allclose(sig, sig_c, atol=1e-9 * np.abs(sig).max())
    Fi = np.linalg.inv(F)
    J = np.linalg.det(F)
    rng = np.random.default_rng(6)
    for _ in range(3):
        dF = rng.normal(size=(3, 3)) * 0.5
        dsig = (D @ dF.ravel()).reshape(3, 3)
        # Pi = J F^-1 sigma F^-T differentiated along dF
        dJ = J * np.trace(Fi @ dF)
        dFi = -Fi @ dF @ Fi
        dPi = dJ * Fi @ sig @ Fi.T + J * (dFi @ sig @ Fi.T + Fi @ dsig @ Fi.T + Fi @ sig @ dFi.T)
        dE = 0.5 * (dF.T @ F + F.T @ dF)
        lhs = from_mandel2(A @ to_mandel2(dE))
        assert np.abs(lhs - dPi).max() <= 2e-4 * np.abs(dPi).max(), np.abs(lhs - dPi).max() / np.abs(dPi).max()


def test_push_forward_objectivity_and_major_symmetry():
    net = nets.lattice(4, p=0.8, jitter=0.25, seed=3, B=6.0)
    U = np.array([[1.06, 0.02, 0.0], [0.02, 0.98, 0.01], [0.0, 0.01, 1.04]])
    R = Rotation.from_rotvec([0.3, 0.2, -0.4]).as_matrix()
    args = _net_args(net)
    sU, AU, CU = mandel_tangent(*args, U, h=1e-6)
    sF, AF, CF = mandel_tangent(*args, R @ U, h=1e-6)
    assert np.allclose(AF, AU, atol=1e-9 * np.abs(AU).max())  # A depends on U only
    C4 = np.einsum("ma,nb,abcd,pc,qd->mnpq", R, R, from_mandel4(CU), R, R)
    assert np.allclose(CF, to_mandel4(C4), atol=1e-8 * np.abs(CU).max())
    assert np.allclose(sF, R @ sU @ R.T, atol=1e-12 * np.abs(sU).max())
    # a hyperelastic network: A_ijkl = A_klij up to the forward-difference error
    assert np.abs(AU - AU.T).max() <= 1e-4 * np.abs(AU).max()
