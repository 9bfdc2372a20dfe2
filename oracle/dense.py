"""Assembled dense/sparse operators on tiny meshes: the plain definitions.

* full system       R H_L R^T u_G = R F_L                    (Sec. 3)
* condensed system  Hhat_e = H_BB - H_BI H_II^-1 H_IB, assembled over the
                    skeleton; fhat_e = F_B - H_BI H_II^-1 F_I          (Sec. 4)
* interior recovery u_I = H_II^-1 (F_I - H_IB u_B)            (Algorithm 1)

Every element block is a dense matrix from oracle.element; assembly uses the
global numbering and packed skeleton layout of oracle.mesh.  Only for meshes
small enough that a sparse direct solve finishes in seconds.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import condensed_element, element_operator, local_rhs
from .mesh import Mesh


class _ElementCache:
    """Dense element matrices keyed by the element widths (shared by all
    elements of equal size)."""

    def __init__(self, p, lam):
        self.p, self.lam = p, lam
        self._c = {}

    def get(self, h):
        key = tuple(float(v) for v in h)
        if key not in self._c:
            Hhat, B, I, H = condensed_element(self.p, key, self.lam)
            HII = H[np.ix_(I, I)]
            self._c[key] = dict(Hhat=Hhat, B=B, I=I, H=H, HII=HII,
                                HBI=H[np.ix_(B, I)], HIB=H[np.ix_(I, B)])
        return self._c[key]


def assemble_full(mesh: Mesh, lam: float) -> sp.csr_matrix:
    """A = sum_e R_e H_e R_e^T over all global nodes (Dirichlet rows kept)."""
    cache = _ElementCache(mesh.p, lam)
    rows, cols, vals = [], [], []
    l2g = mesh.local_to_global
    for e, ex, ey, ez in mesh.elements():
        H = cache.get(mesh.widths(ex, ey, ez))["H"]
        g = l2g[e]
        rows.append(np.repeat(g, len(g)))
        cols.append(np.tile(g, len(g)))
        vals.append(H.ravel())
    n = mesh.n_global
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def assemble_condensed(mesh: Mesh, lam: float) -> sp.csr_matrix:
    """Ahat = sum_e Rhat_e Hhat_e Rhat_e^T on the packed skeleton (nodal space)."""
    cache = _ElementCache(mesh.p, lam)
    slot = mesh.skeleton_slot
    rows, cols, vals = [], [], []
    l2g = mesh.local_to_global
    for e, ex, ey, ez in mesh.elements():
        c = cache.get(mesh.widths(ex, ey, ez))
        s = slot[l2g[e][c["B"]]]
        assert np.all(s >= 0)
        rows.append(np.repeat(s, len(s)))
        cols.append(np.tile(s, len(s)))
        vals.append(c["Hhat"].ravel())
    n = mesh.n_skeleton
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def apply_condensed(mesh: Mesh, lam: float, uB: np.ndarray) -> np.ndarray:
    """v = Ahat u on free skeleton entries; Dirichlet entries of u are ignored
    and those of v are zero."""
    A = assemble_condensed(mesh, lam)
    free = mesh.skeleton_free
    u = np.where(free, uB, 0.0)
    return np.where(free, A @ u, 0.0)


def rhs_full(mesh: Mesh, f_full: np.ndarray) -> np.ndarray:
    """F = sum_e R_e F_e with F_e the GLL-quadrature element load vector."""
    F = np.zeros(mesh.n_global)
    f_full = np.asarray(f_full).ravel()
    l2g = mesh.local_to_global
    for e, ex, ey, ez in mesh.elements():
        g = l2g[e]
        np.add.at(F, g, local_rhs(mesh.p, mesh.widths(ex, ey, ez), f_full[g]))
    return F


def condensed_rhs(mesh: Mesh, lam: float, f_full: np.ndarray) -> np.ndarray:
    """fhat = sum_e Rhat_e (F_B - H_BI H_II^-1 F_I) (Eq. condensation_system),
    zero at Dirichlet entries."""
    cache = _ElementCache(mesh.p, lam)
    slot = mesh.skeleton_slot
    fhat = np.zeros(mesh.n_skeleton)
    f_full = np.asarray(f_full).ravel()
    l2g = mesh.local_to_global
    for e, ex, ey, ez in mesh.elements():
        h = mesh.widths(ex, ey, ez)
        c = cache.get(h)
        g = l2g[e]
        Fe = local_rhs(mesh.p, h, f_full[g])
        contrib = Fe[c["B"]] - c["HBI"] @ np.linalg.solve(c["HII"], Fe[c["I"]])
        np.add.at(fhat, slot[g[c["B"]]], contrib)
    return np.where(mesh.skeleton_free, fhat, 0.0)


def recover_interior(mesh: Mesh, lam: float, f_full: np.ndarray, uB: np.ndarray) -> np.ndarray:
    """Full nodal field from skeleton values: u_I = H_II^-1 (F_I - H_IB u_B)
    per element (Algorithm 1, second loop); Dirichlet nodes are zero."""
    cache = _ElementCache(mesh.p, lam)
    u = np.zeros(mesh.n_global)
    uB = np.where(mesh.skeleton_free, uB, 0.0)
    u[mesh.pack_map] = uB
    f_full = np.asarray(f_full).ravel()
    l2g = mesh.local_to_global
    slot = mesh.skeleton_slot
    for e, ex, ey, ez in mesh.elements():
        h = mesh.widths(ex, ey, ez)
        c = cache.get(h)
        g = l2g[e]
        Fe = local_rhs(mesh.p, h, f_full[g])
        ub = uB[slot[g[c["B"]]]]
        u[g[c["I"]]] = np.linalg.solve(c["HII"], Fe[c["I"]] - c["HIB"] @ ub)
    return u


def solve_condensed(mesh: Mesh, lam: float, f_full: np.ndarray):
    """Algorithm 1: condense, solve the skeleton system directly, recover.
    Returns (u_full, uB)."""
    A = assemble_condensed(mesh, lam).tocsc()
    free = np.flatnonzero(mesh.skeleton_free)
    fhat = condensed_rhs(mesh, lam, f_full)
    uB = np.zeros(mesh.n_skeleton)
    uB[free] = spla.spsolve(A[free][:, free], fhat[free])
    return recover_interior(mesh, lam, f_full, uB), uB


def solve_full(mesh: Mesh, lam: float, f_full: np.ndarray) -> np.ndarray:
    """Brute-force direct solve of the uncondensed system on the free nodes."""
    A = assemble_full(mesh, lam).tocsc()
    free = np.flatnonzero(mesh.free_mask)
    F = rhs_full(mesh, f_full)
    u = np.zeros(mesh.n_global)
    u[free] = spla.spsolve(A[free][:, free], F[free])
    return u
