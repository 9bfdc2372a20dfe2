"""1D Gauss-Lobatto-Legendre basis (Sec. 3 of the paper).

The nodal basis functions are the Lagrange polynomials through the p+1 GLL
points.  The mass matrix is evaluated by GLL quadrature, which makes it the
diagonal of the weights; the stiffness matrix K_ij = int phi_i' phi_j' has a
polynomial integrand of degree 2p-2 and is therefore integrated exactly by the
same quadrature: K = D^T W D, with D_ij = phi_j'(xi_i).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import functools

import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(p: int, x):
    """P_p(x) and P_p'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    if p == 0:
        return p0, d0
    for k in range(1, p):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1          # P'_{k+1} = P'_{k-1} + (2k+1) P_k
        p0, p1 = p1, p2
        d0, d1 = d1, d2
    return p1, d1


@functools.lru_cache(maxsize=None)
def gll(p: int):
    """GLL nodes (ascending, on [-1, 1]) and weights for degree p >= 1."""
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    # interior nodes: roots of P_p', seeded from the Legendre companion matrix,
    # then polished by Newton with P_p'' from Legendre's equation
    c = np.zeros(p + 1)
    c[p] = 1.0
    r = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    for _ in range(50):
        P, dP = legendre(p, r)
        ddP = (2.0 * r * dP - p * (p + 1) * P) / (1.0 - r * r)
        step = dP / ddP
        r = r - step
        if np.max(np.abs(step)) < 1e-17:
            break
    x = np.concatenate(([-1.0], r, [1.0]))
    P, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * P * P)
    x.setflags(write=False)
    w.setflags(write=False)
    return x, w


def diff_matrix(x) -> np.ndarray:
    """D_ij = phi_j'(x_i) for the Lagrange basis through the points x.

    Written from the product form phi_j(x) = prod_{m!=j} (x - x_m)/(x_j - x_m):
    off the diagonal the derivative at a node reduces to (c_i/c_j)/(x_i - x_j)
    with c_i = prod_{m!=i} (x_i - x_m); on the diagonal to sum_{m!=i} 1/(x_i - x_m).
    """
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    c = np.prod(diff, axis=1)
    D = (c[:, None] / c[None, :]) / diff
    for i in range(n):
        D[i, i] = np.sum(1.0 / (x[i] - np.delete(x, i)))
    return D


@functools.lru_cache(maxsize=None)
def mass_stiffness(p: int):
    """Lumped mass M = diag(w) and stiffness K = D^T diag(w) D, both (p+1)^2."""
    x, w = gll(p)
    D = diff_matrix(x)
    K = D.T @ (w[:, None] * D)
    K = 0.5 * (K + K.T)
    M = np.diag(w)
    M.setflags(write=False)
    K.setflags(write=False)
    return M, K
