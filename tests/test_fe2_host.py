"""Host FE² driver on the CPU with an analytic material in place of the RVE
batch: a compressible neo-Hookean solid under uniaxial extension has a
homogeneous exact solution (lateral stretch a from sigma_xx = 0), which the
driver must reproduce, with quadratic Newton convergence."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

MU, LAM = 1.0, 0.6


def nh_sigma(F):
    J = np.linalg.det(F)
    b = np.einsum("nik,njk->nij", F, F)
    return (MU / J)[:, None, None] * (b - np.eye(3)) + (LAM * np.log(J) / J)[:, None, None] * np.eye(3)


class NeoHooke:
    def tangent(self, F):
        h = 1e-6
        D = np.zeros((F.shape[0], 9, 9))
        for kl in range(9):
            E = np.zeros(9)
            E[kl] = h
            E = E.reshape(3, 3)
            D[:, :, kl] = ((nh_sigma(F + E) - nh_sigma(F - E)) / (2 * h)).reshape(-1, 9)
        return nh_sigma(F), D.reshape(-1, 81), np.zeros(F.shape[0], np.int32)


@pytest.fixture(scope="module")
def fe2mod():
    import __graft_entry__ as g
    g.build()
    from paper_2306_09427_gb300 import fe2
    return fe2


def test_shape_function_gradients_partition_of_unity(fe2mod):
    box = fe2mod.HexBox(2, 1, 3, 1.0, 0.5, 2.0)
    assert np.abs(box.G.sum(axis=1)).max() < 1e-12          # sum_a dN_a/dX = 0
    u = box.X @ np.array([[0.1, 0.02, 0], [0, -0.03, 0.01], [0.05, 0, 0.2]]).T
    F = box.deformation_gradients(u)                         # an affine field is reproduced exactly
    assert np.abs(F - (np.eye(3) + np.array([[0.1, 0.02, 0], [0, -0.03, 0.01], [0.05, 0, 0.2]]))).max() < 1e-12


def test_first_pk_tangent_is_derivative(fe2mod):
    rng = np.random.default_rng(0)
    F = np.eye(3) + 0.1 * rng.normal(size=(4, 3, 3))
    s, D, _ = NeoHooke().tangent(F)
    P, A = fe2mod.first_pk_and_tangent(F, s, D)
    h = 1e-6
    for (m, N) in [(0, 0), (1, 2), (2, 1)]:
        E = np.zeros((3, 3))
        E[m, N] = h
        sp, _, _ = NeoHooke().tangent(F + E)
        sm, _, _ = NeoHooke().tangent(F - E)
        Pp, _ = fe2mod.first_pk_and_tangent(F + E, sp, D)
        Pm, _ = fe2mod.first_pk_and_tangent(F - E, sm, D)
        assert np.abs((Pp - Pm) / (2 * h) - A[:, :, :, m, N]).max() < 1e-6


def test_uniaxial_extension_matches_homogeneous_solution(fe2mod):
    box = fe2mod.HexBox(2, 2, 3, 1.0, 1.0, 2.0)
    fe = fe2mod.FE2(box, NeoHooke())
    hist = fe.run(strain=0.1, steps=2, newton_tol=1e-10, log=lambda *a: None)
    lz = 1.1
    a = brentq(lambda a: nh_sigma(np.diag([a, a, lz])[None])[0, 0, 0], 0.5, 1.5)
    s_zz = nh_sigma(np.diag([a, a, lz])[None])[0, 2, 2]
    # reaction on the top face = sigma_zz x current cross-section
    assert abs(hist[-1]["reaction_z"] - s_zz * a * a * 1.0) < 1e-7
    u = fe.u
    top = np.isclose(box.X[:, 2], 2.0)
    assert np.allclose(u[top, 2], 0.2)
    assert np.allclose(u[:, 0], (a - 1.0) * box.X[:, 0], atol=1e-8)
    # Newton converges quadratically: the last ratios fall fast
    n = hist[-1]["newton"]
    assert n[-1] < 1e-10 and len(n) <= 6
