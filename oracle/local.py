"""Condensed operator, condensed load and interior recovery, element by element.

The same quantities as oracle.dense, computed without forming matrices so
that they run at full benchmark sizes:

* H_e applied to a local (p+1)^3 array as the sum of Kronecker products of
  Eq. helmholtz_operator, each Kronecker product applied as three mode
  products (the identity (A(x)B)v = (A(x)I)(I(x)B)v of Sec. 2);
* H_II^-1 by the fast diagonalisation of Sec. 5: with K_II V = M_II V Lambda and
  V^T M_II V = I, H_II^-1 = (V(x)V(x)V) D^-1 (V(x)V(x)V)^T and
  D = d0 I + d1 I(x)I(x)Lambda + d2 I(x)Lambda(x)I + d3 Lambda(x)I(x)I
  (Eq. hii_diagonal).  V and Lambda come from scipy.linalg.eigh.

The condensed action on an element is Hhat_e u_B = [H_e (u_B, 0)]_B -
[H_e (0, H_II^-1 [H_e (u_B, 0)]_I)]_B, the definition of the Schur complement
written as operator applications.  Everything is in nodal space; local arrays
are indexed [element, c, b, a] (z, y, x; x fastest).  Elements are processed
in chunks to bound memory.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .element import metric
from .gll import gll, mass_stiffness
from .mesh import Mesh
from .transform import eigenbasis

_CHUNK_ENTRIES = 1 << 22


def _mode(U, A, axis):
    """Apply matrix A along ``axis`` of U."""
    return np.moveaxis(np.tensordot(A, U, axes=(1, axis)), 0, axis)


def _chunks(mesh: Mesh):
    q3 = (mesh.p + 1) ** 3
    step = max(1, _CHUNK_ENTRIES // q3)
    E = mesh.n_elements
    for s in range(0, E, step):
        yield s, min(E, s + step)


def _l2g(mesh: Mesh, e0: int, e1: int):
    p, q = mesh.p, mesh.p + 1
    e = np.arange(e0, e1)
    ex = e % mesh.mx
    ey = (e // mesh.mx) % mesh.my
    ez = e // (mesh.mx * mesh.my)
    c, b, a = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    gx = ex[:, None, None, None] * p + a[None]
    gy = ey[:, None, None, None] * p + b[None]
    gz = ez[:, None, None, None] * p + c[None]
    return mesh.gid(gx, gy, gz), ex, ey, ez


def _metric(mesh: Mesh, lam, ex, ey, ez):
    """Per-element d[e, 4] (Eq. metriccoeffelement)."""
    return metric(mesh.hx[ex], mesh.hy[ey], mesh.hz[ez], lam)


def H_apply(p: int, d, U):
    """H_e U for local arrays U[e, c, b, a] and per-element metric d[e, 4]."""
    M, K = mass_stiffness(p)
    w = np.diag(M)
    Wa = w[None, None, None, :]
    Wb = w[None, None, :, None]
    Wc = w[None, :, None, None]
    s = lambda k: d[:, k, None, None, None]
    out = s(0) * (Wc * Wb * Wa * U)
    out += s(1) * (Wc * Wb * _mode(U, K, 3))
    out += s(2) * (Wc * Wa * _mode(U, K, 2))
    out += s(3) * (Wb * Wa * _mode(U, K, 1))
    return out


def HII_solve(p: int, d, Y):
    """H_II^-1 Y for interior arrays Y[e, k, j, i] by fast diagonalisation."""
    lam, V = eigenbasis(p)
    Yh = _mode(_mode(_mode(Y, V.T, 3), V.T, 2), V.T, 1)
    D = (d[:, 0, None, None, None] + d[:, 1, None, None, None] * lam[None, None, None, :]
         + d[:, 2, None, None, None] * lam[None, None, :, None]
         + d[:, 3, None, None, None] * lam[None, :, None, None])
    Z = Yh / D
    return _mode(_mode(_mode(Z, V, 3), V, 2), V, 1)


def _interior(U):
    return U[:, 1:-1, 1:-1, 1:-1]


def _zero_interior(U):
    U = U.copy()
    U[:, 1:-1, 1:-1, 1:-1] = 0.0
    return U


def _local_rhs(mesh: Mesh, f_full, g, ex, ey, ez):
    _, w = gll(mesh.p)
    J = mesh.hx[ex] * mesh.hy[ey] * mesh.hz[ez] / 8.0
    W3 = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :]
    return J[:, None, None, None] * W3 * f_full[g]


def apply_condensed(mesh: Mesh, lam: float, uB: np.ndarray) -> np.ndarray:
    """Assembled condensed operator in nodal space on the packed skeleton."""
    p = mesh.p
    ug = mesh.unpack(np.where(mesh.skeleton_free, uB, 0.0))
    vg = np.zeros(mesh.n_global)
    for e0, e1 in _chunks(mesh):
        g, ex, ey, ez = _l2g(mesh, e0, e1)
        d = _metric(mesh, lam, ex, ey, ez)
        U = ug[g]                                # interior entries are zero
        Y = H_apply(p, d, U)
        Z = np.zeros_like(U)
        Z[:, 1:-1, 1:-1, 1:-1] = HII_solve(p, d, _interior(Y))
        out = _zero_interior(Y - H_apply(p, d, Z))
        vg += np.bincount(g.ravel(), weights=out.ravel(), minlength=mesh.n_global)
    return np.where(mesh.skeleton_free, mesh.pack(vg), 0.0)


def condensed_rhs(mesh: Mesh, lam: float, f_full: np.ndarray) -> np.ndarray:
    """fhat = sum_e Rhat_e (F_B - H_BI H_II^-1 F_I) in nodal space."""
    p = mesh.p
    f_full = np.asarray(f_full, float).ravel()
    vg = np.zeros(mesh.n_global)
    for e0, e1 in _chunks(mesh):
        g, ex, ey, ez = _l2g(mesh, e0, e1)
        d = _metric(mesh, lam, ex, ey, ez)
        F = _local_rhs(mesh, f_full, g, ex, ey, ez)
        Z = np.zeros_like(F)
        Z[:, 1:-1, 1:-1, 1:-1] = HII_solve(p, d, _interior(F))
        out = _zero_interior(F - H_apply(p, d, Z))
        vg += np.bincount(g.ravel(), weights=out.ravel(), minlength=mesh.n_global)
    return np.where(mesh.skeleton_free, mesh.pack(vg), 0.0)


def recover_interior(mesh: Mesh, lam: float, f_full: np.ndarray, uB: np.ndarray) -> np.ndarray:
    """u_I = H_II^-1 (F_I - H_IB u_B) per element; full nodal field."""
    p = mesh.p
    f_full = np.asarray(f_full, float).ravel()
    u = mesh.unpack(np.where(mesh.skeleton_free, uB, 0.0))
    ug = u.copy()
    for e0, e1 in _chunks(mesh):
        g, ex, ey, ez = _l2g(mesh, e0, e1)
        d = _metric(mesh, lam, ex, ey, ez)
        F = _local_rhs(mesh, f_full, g, ex, ey, ez)
        Y = H_apply(p, d, ug[g])
        uI = HII_solve(p, d, _interior(F) - _interior(Y))
        u[_interior(g).ravel()] = uI.ravel()
    return u


def apply_full(mesh: Mesh, lam: float, u_full: np.ndarray) -> np.ndarray:
    """A u = sum_e R_e H_e R_e^T u for the uncondensed system (all nodes)."""
    p = mesh.p
    u_full = np.asarray(u_full, float).ravel()
    vg = np.zeros(mesh.n_global)
    for e0, e1 in _chunks(mesh):
        g, ex, ey, ez = _l2g(mesh, e0, e1)
        d = _metric(mesh, lam, ex, ey, ez)
        vg += np.bincount(g.ravel(), weights=H_apply(p, d, u_full[g]).ravel(),
                          minlength=mesh.n_global)
    return vg


def rhs_full(mesh: Mesh, f_full: np.ndarray) -> np.ndarray:
    f_full = np.asarray(f_full, float).ravel()
    vg = np.zeros(mesh.n_global)
    for e0, e1 in _chunks(mesh):
        g, ex, ey, ez = _l2g(mesh, e0, e1)
        vg += np.bincount(g.ravel(), weights=_local_rhs(mesh, f_full, g, ex, ey, ez).ravel(),
                          minlength=mesh.n_global)
    return vg


def transformed_diagonal(mesh: Mesh, lam: float, chunk_probes: int = 2048) -> np.ndarray:
    """Diagonal of the assembled transformed condensed operator T Ahat T^T.

    The diagonal of a sum is the sum of the element diagonals.  For an element
    and a boundary node b, the element entry is psi_b^T Hhat_e psi_b with
    psi_b = T_e^T e_b, which is supported on b's entity: an outer product of
    two eigenvectors on a face, one eigenvector on an edge, a unit value at a
    vertex.  Elements of equal widths share their diagonal, so each width
    class is probed once, then the class diagonals are scatter-added.
    """
    p, q = mesh.p, mesh.p + 1
    _, V = eigenbasis(p)
    S = np.eye(q)
    S[1:p, 1:p] = V.T                               # S = diag(1, S_II, 1)
    c, b, a = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    inner = ((a > 0) & (a < p) & (b > 0) & (b < p) & (c > 0) & (c < p)).ravel()
    bidx = np.flatnonzero(~inner)
    ab, bb, cb = a.ravel()[bidx], b.ravel()[bidx], c.ravel()[bidx]
    widths = mesh.elem_widths
    keys, inv = np.unique(widths, axis=0, return_inverse=True)
    inv = inv.ravel()
    dclass = np.zeros((len(keys), len(bidx)))
    for ci, h in enumerate(keys):
        d = metric(h[0], h[1], h[2], lam)[None, :]
        for s0 in range(0, len(bidx), chunk_probes):
            sel = slice(s0, min(len(bidx), s0 + chunk_probes))
            P = len(bidx[sel])
            # psi = (S^T (x) S^T (x) S^T) e_b: row b of S in every direction
            psi = (S[cb[sel]][:, :, None, None] * S[bb[sel]][:, None, :, None]
                   * S[ab[sel]][:, None, None, :])
            dd = np.repeat(d, P, axis=0)
            Y = H_apply(p, dd, psi)
            Z = np.zeros_like(psi)
            Z[:, 1:-1, 1:-1, 1:-1] = HII_solve(p, dd, _interior(Y))
            out = _zero_interior(Y - H_apply(p, dd, Z))
            dclass[ci, sel] = np.einsum("pcba,pcba->p", psi, out)
    diag = np.zeros(mesh.n_global)
    slot_vals = dclass[inv]                                   # (n_e, n_boundary)
    for e0, e1 in _chunks(mesh):
        g, _, _, _ = _l2g(mesh, e0, e1)
        gb = g.reshape(e1 - e0, -1)[:, bidx]
        diag += np.bincount(gb.ravel(), weights=slot_vals[e0:e1].ravel(), minlength=mesh.n_global)
    return np.where(mesh.skeleton_free, diag[mesh.pack_map], 0.0)
