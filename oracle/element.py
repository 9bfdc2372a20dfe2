"""Element operator of the spectral-element Helmholtz discretisation (Sec. 3).

H_e = d0 M(x)M(x)M + d1 M(x)M(x)K + d2 M(x)K(x)M + d3 K(x)M(x)M  (Eq. helmholtz_operator)

with the rightmost Kronecker factor acting on direction 1 (x).  Local nodes of
an element are numbered a + (p+1) (b + (p+1) c) with a, b, c the node indices in
x, y, z: np.kron(A, B) makes the index of B the fastest, so the factor order of
the paper's formula maps directly onto np.kron(M, np.kron(M, K)) etc.

The metric coefficients (Eq. metriccoeffelement) for an element of widths
h1, h2, h3 are d = h1 h2 h3 / 8 * (lambda, 4/h1^2, 4/h2^2, 4/h3^2).

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .gll import mass_stiffness


def metric(h1, h2, h3, lam: float) -> np.ndarray:
    """d = h1 h2 h3 / 8 (lambda, 4/h1^2, 4/h2^2, 4/h3^2); for array widths the
    result has shape (..., 4)."""
    h1, h2, h3 = (np.asarray(v, dtype=np.float64) for v in (h1, h2, h3))
    J = h1 * h2 * h3 / 8.0
    return np.stack([J * lam, J * 4.0 / h1 ** 2, J * 4.0 / h2 ** 2, J * 4.0 / h3 ** 2], axis=-1)


def element_operator(p: int, h, lam: float) -> np.ndarray:
    """Dense (p+1)^3 x (p+1)^3 element Helmholtz operator H_e."""
    M, K = mass_stiffness(p)
    d = metric(*h, lam)
    kron3 = lambda A, B, C: np.kron(A, np.kron(B, C))
    return (d[0] * kron3(M, M, M) + d[1] * kron3(M, M, K)
            + d[2] * kron3(M, K, M) + d[3] * kron3(K, M, M))


def local_index(p: int, a, b, c):
    q = p + 1
    return np.asarray(a) + q * (np.asarray(b) + q * np.asarray(c))


def boundary_interior(p: int):
    """Local indices of the element's boundary nodes B and interior nodes I
    (Sec. 4): interior means all three node indices in 1..p-1."""
    q = p + 1
    c, b, a = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    inner = (a > 0) & (a < p) & (b > 0) & (b < p) & (c > 0) & (c < p)
    idx = local_index(p, a, b, c).ravel()
    inner = inner.ravel()
    return idx[~inner], idx[inner]


def condensed_element(p: int, h, lam: float):
    """Dense Schur complement H_BB - H_BI H_II^-1 H_IB (Eq. condensation_system).

    Returns (Hhat, B, I, H) with B and I the local index sets."""
    H = element_operator(p, h, lam)
    B, I = boundary_interior(p)
    HBB = H[np.ix_(B, B)]
    HBI = H[np.ix_(B, I)]
    HIB = H[np.ix_(I, B)]
    HII = H[np.ix_(I, I)]
    Hhat = HBB - HBI @ np.linalg.solve(HII, HIB)
    return 0.5 * (Hhat + Hhat.T), B, I, H


def local_rhs(p: int, h, f_local) -> np.ndarray:
    """Discrete element right-hand side F_e = J (w(x)w(x)w) o f_e: the GLL
    quadrature of f times each basis function (mass-lumped), J = h1 h2 h3 / 8."""
    from .gll import gll
    _, w = gll(p)
    J = h[0] * h[1] * h[2] / 8.0
    W3 = np.kron(w, np.kron(w, w))
    return J * W3 * np.asarray(f_local)
