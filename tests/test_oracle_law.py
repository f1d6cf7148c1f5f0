"""Pins of the fiber law (oracle side): limits, closed-form energy, derivatives."""
import numpy as np
import pytest
from scipy.special import erfi

from oracle.fiber_law import axial_force, axial_stiffness, fiber_energy, green_strain


def test_linear_limit_B_to_zero():
    eps = np.linspace(-0.2, 0.3, 11)
    # B -> 0: N -> EA eps_G; first correction is EA B eps^2 / 2
    N = axial_force(eps, 2.0, 1e-9)
    assert np.allclose(N, 2.0 * eps, rtol=1e-8, atol=1e-15)
    assert np.array_equal(axial_force(eps, 2.0, 0.0), 2.0 * eps)


def test_small_strain_relative_precision():
    # expm1 keeps N/eps -> EA for tiny strains (no cancellation)
    for e in (1e-14, 1e-10, 1e-7):
        N = axial_force(np.array([e]), 1.0, 10.0)[0]
        assert abs(N / e - (1.0 + 5.0 * e)) < 1e-12


def test_known_value():
    # eps = 0.105 (10% stretch), EA = 1, B = 10: N = (e^{1.05} - 1)/10
    N = axial_force(np.array([green_strain(1.1, 1.0)]), 1.0, 10.0)[0]
    assert abs(N - (np.e ** 1.05 - 1.0) / 10.0) < 1e-15


def _energy_closed_form(l, L0, EA, B):
    # integral of (EA/B)(exp(B((t/L0)^2-1)/2) - 1) dt from L0 to l via erfi
    u = np.sqrt(B / 2.0)
    g = L0 * np.exp(-B / 2.0) * np.sqrt(np.pi / (2.0 * B)) * (erfi(u * l / L0) - erfi(u))
    return EA / B * (g - (l - L0))


@pytest.mark.parametrize("B", [2.0, 10.0, 20.0])
def test_energy_matches_erfi_closed_form(B):
    L0 = 0.37
    for ratio in (0.7, 0.95, 1.0, 1.05, 1.3):
        l = ratio * L0
        w = fiber_energy(np.array([l]), np.array([L0]), 1.3, B)[0]
        ref = _energy_closed_form(l, L0, 1.3, B)
        assert abs(w - ref) <= 1e-11 * max(abs(ref), 1e-12) + 1e-15


def test_stiffness_is_derivative_of_force():
    L0, EA, B = 0.3, 1.7, 12.0
    for l in (0.25, 0.3, 0.33, 0.36):
        h = 1e-7
        fd = (axial_force(green_strain(l + h, L0), EA, B) - axial_force(green_strain(l - h, L0), EA, B)) / (2 * h)
        assert abs(axial_stiffness(l, L0, EA, B) - fd) < 1e-6 * abs(fd)


def test_energy_derivative_is_force():
    L0, EA, B = 0.3, 1.7, 12.0
    for l in (0.25, 0.3, 0.33, 0.36):
        h = 1e-6
        fd = (fiber_energy(np.array([l + h]), np.array([L0]), EA, B) - fiber_energy(np.array([l - h]), np.array([L0]), EA, B))[0] / (2 * h)
        assert abs(fd - axial_force(green_strain(l, L0), EA, B)) < 1e-8
