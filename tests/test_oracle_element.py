"""Pins for the oracle's element operator (Sec. 3) and static condensation
(Sec. 4): exact energy integrals of polynomials, constants, symmetry and
definiteness, the Schur complement's minimum-energy property."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle.element import (boundary_interior, condensed_element, element_operator,
                            local_index, metric)
from oracle.gll import gll


def _poly_energy(P, Q, R, h, lam):
    """lambda int u^2 + int |grad u|^2 over [0,h1]x[0,h2]x[0,h3] for
    u = P(x) Q(y) R(z), by exact polynomial integration."""
    I = lambda f, a: f.integ()(a) - f.integ()(0.0)
    h1, h2, h3 = h
    mass = I(P * P, h1) * I(Q * Q, h2) * I(R * R, h3)
    gx = I(P.deriv() ** 2, h1) * I(Q * Q, h2) * I(R * R, h3)
    gy = I(P * P, h1) * I(Q.deriv() ** 2, h2) * I(R * R, h3)
    gz = I(P * P, h1) * I(Q * Q, h2) * I(R.deriv() ** 2, h3)
    return lam * mass + gx + gy + gz


@pytest.mark.parametrize("p,h,lam", [(2, (1.0, 0.5, 2.0), 3.0), (4, (0.3, 0.7, 0.2), 0.5),
                                     (5, (2.0, 0.25, 0.5), 0.0), (6, (0.1, 0.1, 0.9), 10.0)])
def test_element_energy_exact(p, h, lam):
    """u^T H_e u equals the exact Helmholtz energy for u of degree <= p-1 in each
    direction (all GLL quadratures exact).  Anisotropic widths and degrees pin
    the metric coefficients and which Kronecker factor is direction 1."""
    rng = np.random.default_rng(p)
    degs = [p - 1, max(p - 2, 1), max(p - 3, 0)]
    P, Q, R = (Polynomial(rng.standard_normal(d + 1)) for d in degs)
    xi, _ = gll(p)
    x = h[0] * (xi + 1) / 2
    y = h[1] * (xi + 1) / 2
    z = h[2] * (xi + 1) / 2
    c, b, a = np.meshgrid(range(p + 1), range(p + 1), range(p + 1), indexing="ij")
    u = (P(x[a]) * Q(y[b]) * R(z[c])).ravel()
    H = element_operator(p, h, lam)
    assert u @ H @ u == pytest.approx(_poly_energy(P, Q, R, h, lam), rel=1e-11)


def test_metric_values():
    d = metric(1.0, 0.5, 2.0, 3.0)
    np.testing.assert_allclose(d, [0.375, 0.5, 2.0, 0.125], rtol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_element_constants_and_spd(p):
    h = (0.4, 1.1, 0.7)
    H0 = element_operator(p, h, 0.0)
    assert np.abs(H0 @ np.ones(len(H0))).max() < 1e-12 * np.abs(H0).max()
    H = element_operator(p, h, 2.0)
    np.testing.assert_allclose(H, H.T, atol=1e-14 * np.abs(H).max())
    assert np.linalg.eigvalsh(H)[0] > 0


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_boundary_interior_split(p):
    B, I = boundary_interior(p)
    assert len(I) == (p - 1) ** 3 and len(B) == (p + 1) ** 3 - (p - 1) ** 3
    assert set(B).isdisjoint(I)
    assert local_index(p, 1, 1, 1) in set(I)


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_schur_complement_properties(p):
    h = (0.3, 0.9, 0.6)
    Hh, B, I, H = condensed_element(p, h, 1.5)
    np.testing.assert_allclose(Hh, Hh.T, atol=1e-13 * np.abs(Hh).max())
    assert np.linalg.eigvalsh(Hh)[0] > 0
    # minimum energy: u_B^T Hhat u_B = min over interior extensions of u^T H u
    rng = np.random.default_rng(p)
    uB = rng.standard_normal(len(B))
    uI = -np.linalg.solve(H[np.ix_(I, I)], H[np.ix_(I, B)] @ uB)
    u = np.zeros(len(H))
    u[B], u[I] = uB, uI
    e_min = u @ H @ u
    assert uB @ Hh @ uB == pytest.approx(e_min, rel=1e-11)
    for _ in range(3):
        v = u.copy()
        v[I] += 1e-3 * rng.standard_normal(len(I))
        assert v @ H @ v > e_min
    # lambda = 0: constants are harmonic, so the condensed operator annihilates 1_B
    Hh0, *_ = condensed_element(p, h, 0.0)
    assert np.abs(Hh0 @ np.ones(len(B))).max() < 1e-11 * np.abs(Hh0).max()
