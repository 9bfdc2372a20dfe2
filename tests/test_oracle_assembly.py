"""Pins for the oracle's assembled system, condensation, transform and PCG.

* The condensed solve with interior recovery (Algorithm 1) equals a brute-force
  direct solve of the uncondensed system.
* The element-local tier (mode products + fast diagonalisation) equals the
  dense Schur-complement tier.
* Spectral convergence to the manufactured solution.
* In the transformed system of Sec. 6, the interior block is the diagonal D of
  Eq. hii_diagonal, only faces couple to the interior, and the self-blocks of
  faces, edges and vertices of the assembled condensed operator are diagonal
  (Eq. east_east_primary_part_transformed and the block preconditioner of
  Sec. 8 being diagonal).
* PCG equals a direct solve; block-Jacobi in nodal space (BC) and the diagonal
  preconditioner in the transformed space (BT) take the same iterations (Sec. 8).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import sem_inputs as si
from oracle import dense, local, transform
from oracle.element import boundary_interior, element_operator
from oracle.gll import mass_stiffness
from oracle.mesh import Mesh
from oracle.pcg import pcg


def _mesh(p, m, ar=1.0):
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar)
    return Mesh(p, hx, hy, hz)


def test_layout_bijection_and_counts():
    for p, m in [(2, (1, 1, 1)), (3, (2, 3, 1)), (4, (4, 4, 4)), (5, (1, 2, 3))]:
        ms = _mesh(p, m)
        pm = ms.pack_map
        np.testing.assert_array_equal(np.sort(pm), np.flatnonzero(ms.skeleton_mask))
        if m[0] == m[1] == m[2]:
            mm, n = m[0], p - 1
            assert ms.n_skeleton == 3 * mm * mm * (mm + 1) * n * n + 3 * mm * (mm + 1) ** 2 * n + (mm + 1) ** 3
    ms = _mesh(4, (4, 4, 4))
    assert ms.n_skeleton == 3185 and int(ms.skeleton_free.sum()) == 1647
    assert int(ms.free_mask.sum()) == 15 ** 3


def test_graded_widths_hit_target():
    for m, ar in [(8, 17.0), (8, 128.0), (32, 128.0), (16, 16.0)]:
        hx, hy, hz, r = si.graded_widths(m, m, m, ar=ar)
        assert si.max_aspect_ratio(hx, hy, hz) == pytest.approx(ar, rel=1e-9)
        assert hx.sum() == pytest.approx(1.0) and r > 1.0


@pytest.mark.parametrize("p,m,lam,ar", [(2, (2, 2, 2), 1.0, 1.0), (3, (3, 2, 2), 0.0, 4.0),
                                        (4, (2, 3, 2), 5.0, 2.0), (5, (2, 2, 3), 0.0, 1.0)])
def test_condensed_solve_equals_direct(p, m, lam, ar):
    ms = _mesh(p, m, ar)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 3).reshape(X.shape)).ravel()
    uc, _ = dense.solve_condensed(ms, lam, f)
    uf = dense.solve_full(ms, lam, f)
    assert np.linalg.norm(uc - uf) <= 1e-12 * np.linalg.norm(uf)
    # the full residual vanishes on free nodes
    A = dense.assemble_full(ms, lam)
    F = dense.rhs_full(ms, f)
    r = (A @ uc - F)[ms.free_mask]
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(F)


@pytest.mark.parametrize("p,m,lam,ar", [(2, (3, 2, 2), 1.0, 3.0), (3, (2, 2, 2), 0.0, 1.0),
                                        (4, (3, 2, 2), 2.5, 5.0), (6, (2, 2, 1), 0.7, 2.0)])
def test_local_tier_equals_dense(p, m, lam, ar):
    ms = _mesh(p, m, ar)
    u = si.random_vector(ms.n_skeleton, 11)
    vd = dense.apply_condensed(ms, lam, u)
    vl = local.apply_condensed(ms, lam, u)
    assert np.linalg.norm(vl - vd) <= 1e-13 * np.linalg.norm(vd)
    X, Y, Z = ms.coords()
    f = si.node_noise(X.size, 12)
    fd = dense.condensed_rhs(ms, lam, f)
    fl = local.condensed_rhs(ms, lam, f)
    assert np.linalg.norm(fl - fd) <= 1e-13 * np.linalg.norm(fd)
    ud = dense.recover_interior(ms, lam, f, u)
    ul = local.recover_interior(ms, lam, f, u)
    assert np.linalg.norm(ul - ud) <= 1e-12 * np.linalg.norm(ud)
    # uncondensed action: A u from mode products vs assembled sparse matrix
    uu = si.random_vector(ms.n_global, 13)
    np.testing.assert_allclose(local.apply_full(ms, lam, uu), dense.assemble_full(ms, lam) @ uu,
                               rtol=0, atol=1e-12 * np.abs(uu).max() * 50)


def test_manufactured_spectral_convergence():
    """u = sin(pi x) sin(pi y) sin(pi z), f = (3 pi^2 + lambda) u on 2^3 elements:
    the max nodal error decays spectrally with p."""
    errs = []
    for p in (2, 4, 6, 8):
        ms = _mesh(p, (2, 2, 2))
        X, Y, Z = ms.coords()
        f = si.manufactured_f(X, Y, Z, 1.0).ravel()
        u, _ = dense.solve_condensed(ms, 1.0, f)
        errs.append(np.abs(u - si.manufactured_u(X, Y, Z).ravel()).max())
    assert all(b < 0.1 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6


def _S3(p):
    lam, V = transform.eigenbasis(p)
    S = np.eye(p + 1)
    S[1:p, 1:p] = V.T
    return np.kron(S, np.kron(S, S)), lam


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_transformed_element_structure(p):
    h = (0.3, 1.2, 0.5)
    lamh = 2.0
    H = element_operator(p, h, lamh)
    S3, lam = _S3(p)
    Ht = S3 @ H @ S3.T
    B, I = boundary_interior(p)
    # interior block = D = d0 + d1 Lambda_i + d2 Lambda_j + d3 Lambda_k
    from oracle.element import metric
    d = metric(*h, lamh)
    n = p - 1
    k, j, i = np.meshgrid(range(n), range(n), range(n), indexing="ij")
    D = (d[0] + d[1] * lam[i] + d[2] * lam[j] + d[3] * lam[k]).ravel()
    np.testing.assert_allclose(Ht[np.ix_(I, I)], np.diag(D), atol=1e-11 * D.max())
    # only face nodes couple to the interior
    q = p + 1
    c, b, a = np.unravel_index(B, (q, q, q))
    on_face = ((a == 0) | (a == p)).astype(int) + ((b == 0) | (b == p)) + ((c == 0) | (c == p)) == 1
    HBI = Ht[np.ix_(B, I)]
    assert np.abs(HBI[~on_face]).max() < 1e-12 * np.abs(Ht).max()
    # the transform maps boundary nodes to boundary nodes
    assert np.abs(S3[np.ix_(B, I)]).max() == 0.0


@pytest.mark.parametrize("p,m,ar", [(3, (2, 2, 2), 3.0), (4, (3, 2, 2), 1.0), (5, (2, 2, 2), 8.0)])
def test_transformed_self_blocks_diagonal(p, m, ar):
    ms = _mesh(p, m, ar)
    A = dense.assemble_condensed(ms, 0.0)
    T = transform.T_matrix(ms)
    At = (T @ A @ T.T).toarray()
    free = ms.skeleton_free
    scale = np.abs(At).max()
    for kind, idx in ms.entity_blocks():
        if not free[idx].all():
            continue
        blk = At[np.ix_(idx, idx)]
        assert np.abs(blk - np.diag(np.diag(blk))).max() < 1e-11 * scale, kind
    # the transform helpers reproduce T A T^T
    ut = si.random_vector(ms.n_skeleton, 21)
    v = transform.load_to_transformed(ms, A @ transform.solution_from_transformed(ms, ut))
    np.testing.assert_allclose(v, At @ ut, atol=1e-12 * np.abs(At @ ut).max())
    np.testing.assert_allclose(transform.solution_to_transformed(ms, transform.solution_from_transformed(ms, ut)),
                               ut, atol=1e-12 * np.abs(ut).max())


@pytest.mark.parametrize("p,m,lam,ar,grade", [(3, (3, 2, 2), 0.0, 8.0, "x"), (4, (2, 3, 2), 1.5, 4.0, "xy"),
                                              (6, (2, 2, 2), 0.3, 3.0, "x")])
def test_transformed_diagonal_equals_dense(p, m, lam, ar, grade):
    """local.transformed_diagonal (the BT preconditioner's diagonal, formed by
    probing each width class with rows of S = diag(1, S_II, 1)) equals the
    diagonal of T Ahat T^T from the dense Schur-complement assembly entry by
    entry, and is zero at Dirichlet entries."""
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar, grade=grade)
    ms = Mesh(p, hx, hy, hz)
    A = dense.assemble_condensed(ms, lam)
    T = transform.T_matrix(ms)
    dd = np.where(ms.skeleton_free, (T @ A @ T.T).diagonal(), 0.0)
    dl = local.transformed_diagonal(ms, lam)
    np.testing.assert_allclose(dl, dd, rtol=0, atol=1e-13 * np.abs(dd).max())


def test_pcg_equals_direct():
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((60, 60))
    A = Q @ Q.T + 60 * np.eye(60)
    b = rng.standard_normal(60)
    x, it, hist = pcg(lambda v: A @ v, b, 1.0 / np.diag(A), rtol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    assert hist[-1] <= 1e-13 and it <= 60


@pytest.mark.parametrize("p,m,ar", [(4, (3, 3, 3), 8.0), (5, (3, 3, 2), 1.0)])
def test_block_jacobi_nodal_equals_diagonal_transformed(p, m, ar):
    """BC (nodal block-Jacobi over faces/edges/vertices) and BT (diagonal in
    the transformed system) are congruent by T and give the same iterates."""
    ms = _mesh(p, m, ar)
    free = np.flatnonzero(ms.skeleton_free)
    A = dense.assemble_condensed(ms, 0.0).toarray()
    T = transform.T_matrix(ms).toarray()
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, 0.0) + si.node_noise(X.size, 5).reshape(X.shape)).ravel()
    fh = dense.condensed_rhs(ms, 0.0, f)
    # BC in nodal space
    Pbc = np.zeros_like(A)
    for kind, idx in ms.entity_blocks():
        idx = idx[ms.skeleton_free[idx]]
        if len(idx):
            Pbc[np.ix_(idx, idx)] = np.linalg.inv(A[np.ix_(idx, idx)])
    Af, Pf = A[np.ix_(free, free)], Pbc[np.ix_(free, free)]

    def pcg_matrix_prec(b, P, rtol):
        x = np.zeros_like(b); r = b.copy(); z = P @ r; pp = z.copy(); rho = r @ z
        r0 = np.linalg.norm(r)
        for it in range(1, 5000):
            q = Af @ pp
            al = rho / (pp @ q); x += al * pp; r -= al * q
            if np.linalg.norm(r) <= rtol * r0:
                return x, it
            z = P @ r; rn = r @ z; pp = z + rn / rho * pp; rho = rn
        raise AssertionError

    # BT in the transformed space: diagonal preconditioner of T A T^T
    At = T @ A @ T.T
    Atf = At[np.ix_(free, free)]
    fht = (T @ fh)[free]
    xt, it_bt, _ = pcg(lambda v: Atf @ v, fht, 1.0 / np.diag(Atf), rtol=1e-10)
    xn, it_bc = pcg_matrix_prec(fh[free], Pf, 1e-10)
    # same solution in nodal space
    xt_full = np.zeros(ms.n_skeleton); xt_full[free] = xt
    xn_full = np.zeros(ms.n_skeleton); xn_full[free] = xn
    np.testing.assert_allclose(T.T @ xt_full, xn_full, atol=1e-8 * np.abs(xn_full).max())
    assert abs(it_bt - it_bc) <= 2, (it_bt, it_bc)
