"""The coordinate transform of Sec. 6 on the packed skeleton.

S = diag(1, S_II, 1) applied in all three directions turns H_e into
H~_e = (S(x)S(x)S) H_e (S(x)S(x)S)^T.  S_II comes from the generalised
eigenproblem of K_II and M_II (Eq. generalized_eigenvalues).  Reading of the
paper's convention: V holds M_II-orthonormal eigenvectors as columns,
K_II V = M_II V Lambda, V^T M_II V = I, and S_II := V^T; then
S_II M_II S_II^T = I and S_II K_II S_II^T = Lambda as the paper states.

Eigenvectors are unique up to sign.  Canonical choice used here: eigenvalues
ascending, each column scaled so that its first entry (the interior node next
to xi = -1) is positive.

Because S keeps the vertex indices 0 and p and acts on interior indices only,
S(x)S(x)S maps each skeleton entity onto itself: S_II(x)S_II on a face,
S_II on an edge, 1 on a vertex.  That entity-wise matrix T is the same for
every element touching the entity, so the assembled transformed condensed
operator is T Ahat T^T.  Vectors transform as u~ = T^-T u (solution-like,
Algorithm 4 first loop) and F~ = T F (load-like).

Test infrastructure only.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .gll import mass_stiffness
from .mesh import Mesh


@functools.lru_cache(maxsize=None)
def eigenbasis(p: int):
    """(Lambda, V): generalised eigenpairs of (K_II, M_II), canonical signs."""
    M, K = mass_stiffness(p)
    KII = K[1:p, 1:p]
    MII = M[1:p, 1:p]
    lam, V = sla.eigh(KII, MII)
    V = V * np.sign(V[0, :])[None, :]
    lam.setflags(write=False)
    V.setflags(write=False)
    return lam, V


def S_II(p: int) -> np.ndarray:
    return eigenbasis(p)[1].T.copy()


def _apply_entitywise(mesh: Mesh, vec, A):
    """Apply A(x)A to every face block, A to every edge block, 1 to vertices.

    Face values are stored [slow, fast] so A(x)A acting on them is A U A^T."""
    out = np.array(vec, dtype=np.float64, copy=True)
    n = mesh.n
    c = mesh.block_counts
    off = 0
    for kind in ("xface", "yface", "zface"):
        cnt = c[kind]
        blk = out[off:off + cnt * n * n].reshape(cnt, n, n)
        out[off:off + cnt * n * n] = np.einsum("ij,ejk,lk->eil", A, blk, A).ravel()
        off += cnt * n * n
    for kind in ("xedge", "yedge", "zedge"):
        cnt = c[kind]
        blk = out[off:off + cnt * n].reshape(cnt, n)
        out[off:off + cnt * n] = (blk @ A.T).ravel()
        off += cnt * n
    return out


def T_matrix(mesh: Mesh) -> sp.csr_matrix:
    """Sparse entity-wise transform T on the packed skeleton."""
    S = S_II(mesh.p)
    SS = np.kron(S, S)
    blocks = []
    for kind, idx in mesh.entity_blocks():
        if kind.endswith("face"):
            blocks.append(SS)
        elif kind.endswith("edge"):
            blocks.append(S)
        else:
            blocks.append(np.ones((1, 1)))
    return sp.block_diag(blocks, format="csr")


def solution_to_transformed(mesh: Mesh, uB):
    """u~ = T^-T u; per direction S_II^-T = V^-1 = V^T M_II."""
    lam, V = eigenbasis(mesh.p)
    M, _ = mass_stiffness(mesh.p)
    return _apply_entitywise(mesh, uB, V.T @ M[1:-1, 1:-1])


def solution_from_transformed(mesh: Mesh, ut):
    """u = T^T u~; per direction S_II^T = V."""
    _, V = eigenbasis(mesh.p)
    return _apply_entitywise(mesh, ut, V)


def load_to_transformed(mesh: Mesh, vB):
    """F~ = T F; per direction S_II = V^T."""
    _, V = eigenbasis(mesh.p)
    return _apply_entitywise(mesh, vB, V.T)

