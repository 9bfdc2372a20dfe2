"""Pins for the oracle's 1D basis (Sec. 3): GLL points and weights, the lumped
mass and the exact stiffness matrix, checked against closed forms and exact
polynomial integrals rather than against the oracle itself."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import Legendre, Polynomial

from oracle.gll import diff_matrix, gll, mass_stiffness
from oracle.transform import eigenbasis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_textbook.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        p, x, w = line.split()
        val = lambda s: float(eval(s, {"sqrt": math.sqrt}))
        rows.setdefault(int(p), []).append((val(x), val(w)))
    return rows


@pytest.mark.parametrize("p", [2, 3, 4])
def test_gll_textbook_values(p):
    xs, ws = zip(*_golden()[p])
    x, w = gll(p)
    np.testing.assert_allclose(x, xs, atol=1e-15)
    np.testing.assert_allclose(w, ws, rtol=1e-14)


@pytest.mark.parametrize("p", list(range(1, 33)))
def test_gll_quadrature_exactness(p):
    """Lobatto quadrature is exact for degree <= 2p-1 and not for 2p."""
    x, w = gll(p)
    assert np.all(np.diff(x) > 0) and x[0] == -1.0 and x[-1] == 1.0
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, k
    # degree 2p is not integrated exactly: the GLL rule gives sum w P_p^2 = 2/p,
    # whereas int P_p^2 = 2/(2p+1)
    Pp = Legendre.basis(p)(x)
    assert np.sum(w * Pp * Pp) == pytest.approx(2.0 / p, rel=1e-13)
    assert w[0] == pytest.approx(2.0 / (p * (p + 1)), rel=1e-14)


@pytest.mark.parametrize("p", [2, 5, 8, 16, 32])
def test_diff_matrix_exact_on_polynomials(p):
    x, _ = gll(p)
    D = diff_matrix(x)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(p + 1)
    P = Polynomial(c)
    np.testing.assert_allclose(D @ P(x), P.deriv()(x), atol=1e-9 * np.abs(c).sum() * p * p)


def test_stiffness_p1_closed_form():
    _, K = mass_stiffness(1)
    np.testing.assert_allclose(K, 0.5 * np.array([[1.0, -1.0], [-1.0, 1.0]]), atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 4, 7, 8, 12, 16, 24, 32])
def test_stiffness_properties(p):
    M, K = mass_stiffness(p)
    np.testing.assert_allclose(K, K.T, atol=0)
    assert np.abs(K @ np.ones(p + 1)).max() < 1e-10 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert abs(ev[0]) < 1e-9 * ev[-1] and ev[1] > 1e-6     # one-dimensional null space
    # u^T K u = int_{-1}^{1} u'(x)^2 dx for u of degree <= p (exact integral)
    x, _ = gll(p)
    rng = np.random.default_rng(100 + p)
    P = Polynomial(rng.standard_normal(p + 1))
    dP2 = P.deriv() ** 2
    exact = dP2.integ()(1.0) - dP2.integ()(-1.0)
    u = P(x)
    assert u @ K @ u == pytest.approx(exact, rel=1e-10)
    # lumped mass is the weight diagonal
    np.testing.assert_array_equal(np.diag(np.diag(M)), M)


@pytest.mark.parametrize("p", [2, 4, 8, 16, 32])
def test_generalized_eigenpairs(p):
    """Eq. generalized_eigenvalues with S_II = V^T: S M_II S^T = I, S K_II S^T = Lambda."""
    M, K = mass_stiffness(p)
    lam, V = eigenbasis(p)
    S = V.T
    np.testing.assert_allclose(S @ M[1:p, 1:p] @ S.T, np.eye(p - 1), atol=1e-12)
    np.testing.assert_allclose(S @ K[1:p, 1:p] @ S.T, np.diag(lam), atol=1e-10 * lam[-1])
    assert np.all(np.diff(lam) > 0)
    # canonical sign: first entry positive and well away from zero
    assert np.all(V[0, :] > 1e-3 * np.abs(V).max(axis=0))


def test_lowest_eigenvalue_converges_to_continuous():
    """The smallest eigenvalue of -u'' = Lambda u on (-1, 1) with u(+-1) = 0 is
    (pi/2)^2; the discrete one converges spectrally."""
    errs = [abs(eigenbasis(p)[0][0] - (math.pi / 2) ** 2) for p in (4, 6, 8, 12)]
    assert errs[-1] < 1e-10
    assert all(a > b for a, b in zip(errs, errs[1:]))
