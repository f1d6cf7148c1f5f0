"""Pins of the oracle's stability verdict and saddle escape (Sec. 3.2).

The oracle accepts an equilibrium only if it is a local minimum of the
stored energy (the static state the damped loop of Algorithm 2 settles in;
a saddle is an equilibrium the dynamics leaves).  These tests pin each part
of that decision to something other than the oracle itself:

* the inertia count of the symmetric factorisation against the closed-form
  spectrum of the Dirichlet path Laplacian, 2 - 2 cos(k pi / (n + 1));
* a straight chain of fibers held in compression between two fixed nodes:
  the straight state is an equilibrium by symmetry, and its transverse
  curvature is 2 N / l per free node (N < 0), a saddle with a closed-form
  lowest eigenvalue; the escape must end at a lower-energy stable state;
* a planted "always stable" bug in the factorisation must fail the pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.newton as newton
from oracle.fiber_law import axial_force, green_strain

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _path_laplacian(n):
    return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csc")


@pytest.mark.parametrize("n,c", [(7, 0.0), (7, 1.1), (40, 0.5), (40, 3.9), (200, 2.2)])
def test_inertia_count_matches_closed_form_spectrum(n, c):
    lam = 2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    expected = int((lam - c < 0).sum())
    _, pd, neg = newton._factor(_path_laplacian(n), -c)
    assert neg == expected
    assert pd == (expected == 0)


def test_lowest_eigenvalue_dense_and_lanczos():
    n = 60
    lam = 2.0 - 2.0 * np.cos(np.pi / (n + 1))
    assert newton.lowest_eigenvalue(_path_laplacian(n)) == pytest.approx(lam, rel=1e-9)
    # above the dense limit: a diagonal operator with one isolated negative entry
    d = np.linspace(1.0, 2.0, 3500)
    d[1234] = -0.7
    assert newton.lowest_eigenvalue(sp.diags(d, format="csc")) == pytest.approx(-0.7, rel=1e-8)


def _chain(n_free, gap=0.8, L0=1.0, EA=1.0, B=10.0):
    """A straight chain along x: fixed ends, n_free free nodes, n_free + 1
    fibers of rest length L0 at spacing gap < L0 (every fiber compressed)."""
    m = n_free + 2
    xs = (np.arange(m) - 0.5 * (m - 1)) * gap
    X = np.zeros((m, 3))
    X[:, 0] = xs
    conn = np.array([[k, k + 1] for k in range(m - 1)], np.int32)
    isb = np.zeros(m, np.uint8)
    isb[0] = isb[-1] = 1
    e = m - 1
    return X, conn, np.full(e, L0), np.full(e, EA), np.full(e, B), isb


def _problem(X, conn, L0, EA, B, isb):
    kept, free = newton.prune(conn, isb)
    assert kept.all() and free.sum() == (isb == 0).sum()
    return newton._Problem(X, conn.astype(np.int64), L0, EA, B, free)


def _pin_chain_saddle(n_free):
    X, conn, L0, EA, B, isb = _chain(n_free)
    pb = _problem(X, conn, L0, EA, B, isb)
    x = X.copy()  # F = I: the straight state
    # an equilibrium by symmetry (uniform compression along the chain)
    assert np.abs(pb.residual(x)).max() < 1e-15
    stable, lam, neg = newton.stability(pb, x)
    N = axial_force(green_strain(0.8, 1.0), 1.0, 10.0)
    assert N < 0.0
    # transverse curvature of the chain: the tridiagonal (N/l) [2 -1; -1 2 ...]
    # in y and in z, lowest eigenvalue (N/l)(2 - 2 cos(pi/(n_free+1)))... with N < 0
    # the most negative is (N/l)(2 + 2 cos(pi/(n_free+1)))
    lam_exact = (N / 0.8) * (2.0 + 2.0 * np.cos(np.pi / (n_free + 1)))
    assert lam == pytest.approx(lam_exact, rel=1e-10)
    assert not stable
    assert neg == 2 * n_free  # every transverse mode (y and z) has N/l < 0 curvature
    return pb, x


@pytest.mark.parametrize("n_free", [1, 2, 3])
def test_compressed_chain_is_a_saddle(n_free):
    _pin_chain_saddle(n_free)


@pytest.mark.parametrize("n_free", [1, 2])
def test_escape_from_the_chain_saddle_reaches_a_lower_stable_minimum(n_free):
    X, conn, L0, EA, B, isb = _chain(n_free)
    F = np.eye(3)
    pb, x_saddle = _pin_chain_saddle(n_free)
    W_saddle = pb.energy(x_saddle)
    # without the check the solver stops at the saddle (zero residual at the start)
    s0 = newton.solve(X, conn, L0, EA, B, isb, F, tol=1e-10, check_stability=False)
    assert s0.newton_iters == 0 and s0.stable is None
    assert np.allclose(s0.x, X)
    s = newton.solve(X, conn, L0, EA, B, isb, F, tol=1e-10, record_lambda=True)
    assert s.saddle_escapes >= 1
    assert s.stable is True and s.converged
    assert s.info["energy"] < W_saddle - 1e-3
    # the minima of a chain longer than its span hold every fiber at its rest
    # length (zero energy, zero stress)
    assert s.info["energy"] == pytest.approx(0.0, abs=1e-12)
    lengths = np.linalg.norm(s.x[conn[:, 1]] - s.x[conn[:, 0]], axis=1)
    assert np.allclose(lengths, 1.0, atol=1e-6)
    assert np.abs(s.sigma).max() < 1e-6
    assert s.info["lambda_min"] >= -newton.STAB_SHIFT * 1.0


def test_a_true_minimum_is_stable_with_its_lowest_eigenvalue():
    # the same chain in tension: straight is the unique minimum
    X, conn, L0, EA, B, isb = _chain(2, gap=1.1)
    s = newton.solve(X, conn, L0, EA, B, isb, np.eye(3), tol=1e-12, record_lambda=True)
    assert s.stable is True and s.saddle_escapes == 0
    N = axial_force(green_strain(1.1, 1.0), 1.0, 10.0)
    assert N > 0.0
    lam_exact = (N / 1.1) * (2.0 - 2.0 * np.cos(np.pi / 3))  # transverse, lowest
    assert s.info["lambda_min"] == pytest.approx(lam_exact, rel=1e-9)


def test_planted_always_stable_bug_fails_the_saddle_pin(monkeypatch):
    real = newton._factor

    def always_pd(K, mu):
        lu, _, _ = real(K, mu)
        return lu, True, 0

    monkeypatch.setattr(newton, "_factor", always_pd)
    with pytest.raises(AssertionError):
        _pin_chain_saddle(2)


def test_planted_wrong_inertia_sign_fails_the_spectrum_pin(monkeypatch):
    real = newton._factor

    def flipped(K, mu):
        lu, pd, neg = real(K, mu)
        return lu, pd, K.shape[0] - neg

    monkeypatch.setattr(newton, "_factor", flipped)
    with pytest.raises(AssertionError):
        test_inertia_count_matches_closed_form_spectrum(40, 0.5)
