"""Algorithm 4 with the oracle's element-local tier: transformed condensed
load, CG with the diagonal (BT) preconditioner on T Ahat T^T, back-transform
and interior recovery.  Runs at full benchmark sizes (slowly).

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from . import local, transform
from .mesh import Mesh
from .pcg import pcg


def bt_solve(mesh: Mesh, lam: float, f_full, rtol=1e-10, maxit=100000, diag=None, x0=None, callback=None):
    """Returns (u_full, uB_transformed, iterations, residual history)."""
    free = mesh.skeleton_free
    fhat = local.condensed_rhs(mesh, lam, f_full)
    b = np.where(free, transform.load_to_transformed(mesh, fhat), 0.0)
    if diag is None:
        diag = local.transformed_diagonal(mesh, lam)
    P = np.where(free, 1.0 / np.where(free, diag, 1.0), 0.0)

    def apply(ut):
        u = transform.solution_from_transformed(mesh, np.where(free, ut, 0.0))
        v = local.apply_condensed(mesh, lam, u)
        return np.where(free, transform.load_to_transformed(mesh, v), 0.0)

    ut, it, hist = pcg(apply, b, P, rtol=rtol, maxit=maxit, x0=x0, callback=callback)
    uB = transform.solution_from_transformed(mesh, ut)
    return local.recover_interior(mesh, lam, f_full, uB), ut, it, hist
