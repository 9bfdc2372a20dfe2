"""Gradients of J = 1/2 ||u - u_t||^2 through the discrete Helmholtz solve,
u = A(lambda, h)^-1 M(h) f on the free nodes, by the adjoint method on dense
assembled matrices (tiny meshes only).

  w        = A^-1 (u - u_t)
  dJ/df    = M w
  dJ/dlam  = -w^T (dA/dlam) u,              dA/dlam = M (assembled lumped mass)
  dJ/dh    =  w^T (dF/dh) - w^T (dA/dh) u,  A = sum_e R_e H_e(d(h)) R_e^T,
                                            F = sum_e R_e J(h) (w(x)w(x)w) o f_e

with the derivatives of d = h1h2h3/8 (lambda, 4/h1^2, 4/h2^2, 4/h3^2) and of
J = h1h2h3/8 taken by hand.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dense import assemble_full, rhs_full
from .gll import gll, mass_stiffness
from .mesh import Mesh


def _kron_terms(p):
    M, K = mass_stiffness(p)
    k3 = lambda A, B, C: np.kron(A, np.kron(B, C))
    return [k3(M, M, M), k3(M, M, K), k3(M, K, M), k3(K, M, M)]


def _dd_dh(h, lam, axis):
    """Derivatives of (d0, d1, d2, d3) and of J with respect to h[axis]."""
    h1, h2, h3 = h
    hh = [h1, h2, h3]
    others = [hh[(axis + 1) % 3], hh[(axis + 2) % 3]]
    dJ = others[0] * others[1] / 8.0
    J = h1 * h2 * h3 / 8.0
    dd = [lam * dJ]
    for k in range(3):
        if k == axis:
            # J * 4 / h_k^2 = (product of the other two) / (2 h_k)
            dd.append(-others[0] * others[1] / (2.0 * hh[k] ** 2))
        else:
            dd.append(4.0 * dJ / hh[k] ** 2)
    return np.array(dd), dJ


def solve_and_gradient(mesh: Mesh, lam: float, f_full, u_target):
    """Returns (J, u, dJ/df, dJ/dlam, (dJ/dhx, dJ/dhy, dJ/dhz))."""
    f_full = np.asarray(f_full, float).ravel()
    free = np.flatnonzero(mesh.free_mask)
    A = assemble_full(mesh, lam).tocsc()
    Af = A[free][:, free]
    F = rhs_full(mesh, f_full)
    u = np.zeros(mesh.n_global)
    u[free] = spla.spsolve(Af, F[free])
    g = (u - np.asarray(u_target, float).ravel())
    g[~mesh.free_mask] = 0.0
    J = 0.5 * float(np.sum((u - np.asarray(u_target, float).ravel()) ** 2))
    w = np.zeros(mesh.n_global)
    w[free] = spla.spsolve(Af, g[free])
    # assembled lumped mass
    _, wq = gll(mesh.p)
    m = rhs_full(mesh, np.ones(mesh.n_global))
    df = np.where(mesh.free_mask, m * w, 0.0)
    dlam = -float(np.sum(w * m * u))
    terms = _kron_terms(mesh.p)
    W3 = np.kron(wq, np.kron(wq, wq))
    l2g = mesh.local_to_global
    dh = [np.zeros(mesh.mx), np.zeros(mesh.my), np.zeros(mesh.mz)]
    for e, ex, ey, ez in mesh.elements():
        h = mesh.widths(ex, ey, ez)
        gidx = l2g[e]
        we, ue, fe = w[gidx], u[gidx], f_full[gidx]
        forms = np.array([we @ (T @ ue) for T in terms])
        load = float(np.sum(W3 * we * fe))
        for axis, idx in enumerate((ex, ey, ez)):
            dd, dJ = _dd_dh(h, lam, axis)
            dh[axis][idx] += -float(dd @ forms) + dJ * load
    return J, u, df, dlam, tuple(dh)


def objective(mesh: Mesh, lam: float, f_full, u_target):
    free = np.flatnonzero(mesh.free_mask)
    A = assemble_full(mesh, lam).tocsc()
    F = rhs_full(mesh, np.asarray(f_full, float).ravel())
    u = np.zeros(mesh.n_global)
    u[free] = spla.spsolve(A[free][:, free], F[free])
    return 0.5 * float(np.sum((u - np.asarray(u_target, float).ravel()) ** 2))
