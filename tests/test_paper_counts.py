"""Table 2 and Table 3 of the paper, checked against the dense definition.

A loop-by-loop evaluation of the condensed part in the transformed system,
written from Table 2 (expansions d * K~_{I0} / K~_{Ip} from the six faces into
the interior eigenspace, scaling by D^-1, contractions back with K~_{0I} /
K~_{pI}), must reproduce H~_BI H~_II^-1 H~_IB on the faces, where
H~ = (S(x)S(x)S) H_e (S(x)S(x)S)^T comes from the dense oracle.  Counting its
multiplications reproduces the 13 n^3 leading term of Table 3 (TPT, condensed
part), with the metric factors folded into the faces at O(n^2) cost.
"""
import numpy as np
import pytest

from oracle.element import boundary_interior, element_operator, local_index, metric
from oracle.gll import mass_stiffness
from oracle.transform import eigenbasis


class Counter:
    def __init__(self):
        self.n = 0

    def mul(self, a, b):
        self.n += 1
        return a * b


def table2_condensed(p, d, lam, Kt0, Ktp, faces, cnt):
    """faces: dict w,e,s,n,b,t -> n x n arrays in (slow, fast) local order:
    w/e: [k][j], s/n: [k][i], b/t: [j][i].  Returns the six face outputs."""
    n = p - 1
    # fold metric factors into the faces: O(n^2)
    sc = {"w": d[1], "e": d[1], "s": d[2], "n": d[2], "b": d[3], "t": d[3]}
    f = {key: [[cnt.mul(sc[key], faces[key][r][c]) for c in range(n)] for r in range(n)]
         for key in faces}
    # expansion into the eigenspace: 6 n^3
    u = [[[0.0] * n for _ in range(n)] for _ in range(n)]      # u[k][j][i]
    for k in range(n):
        for j in range(n):
            for i in range(n):
                u[k][j][i] = (cnt.mul(Kt0[i], f["w"][k][j]) + cnt.mul(Ktp[i], f["e"][k][j])
                              + cnt.mul(Kt0[j], f["s"][k][i]) + cnt.mul(Ktp[j], f["n"][k][i])
                              + cnt.mul(Kt0[k], f["b"][j][i]) + cnt.mul(Ktp[k], f["t"][j][i]))
    # diagonal scaling by D^-1: n^3 (D^-1 precomputed, Sec. 5)
    Dinv = [[[1.0 / (d[0] + d[1] * lam[i] + d[2] * lam[j] + d[3] * lam[k]) for i in range(n)]
             for j in range(n)] for k in range(n)]
    v = [[[cnt.mul(Dinv[k][j][i], u[k][j][i]) for i in range(n)] for j in range(n)] for k in range(n)]
    # contraction back to the faces: 6 n^3
    out = {key: [[0.0] * n for _ in range(n)] for key in faces}
    for k in range(n):
        for j in range(n):
            for i in range(n):
                out["w"][k][j] += cnt.mul(Kt0[i], v[k][j][i])
                out["e"][k][j] += cnt.mul(Ktp[i], v[k][j][i])
                out["s"][k][i] += cnt.mul(Kt0[j], v[k][j][i])
                out["n"][k][i] += cnt.mul(Ktp[j], v[k][j][i])
                out["b"][j][i] += cnt.mul(Kt0[k], v[k][j][i])
                out["t"][j][i] += cnt.mul(Ktp[k], v[k][j][i])
    return {key: [[cnt.mul(sc[key], out[key][r][c]) for c in range(n)] for r in range(n)]
            for key in faces}


FACE_NODES = {  # (a, b, c) of local node from (row, col) of the face array
    "w": lambda r, c, p: (0, c + 1, r + 1), "e": lambda r, c, p: (p, c + 1, r + 1),
    "s": lambda r, c, p: (c + 1, 0, r + 1), "n": lambda r, c, p: (c + 1, p, r + 1),
    "b": lambda r, c, p: (c + 1, r + 1, 0), "t": lambda r, c, p: (c + 1, r + 1, p),
}


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_table2_matches_dense_and_counts_13n3(p):
    h = (0.7, 0.4, 1.3)
    lamh = 0.8
    n = p - 1
    d = metric(*h, lamh)
    H = element_operator(p, h, lamh)
    lam, V = eigenbasis(p)
    S = np.eye(p + 1)
    S[1:p, 1:p] = V.T
    S3 = np.kron(S, np.kron(S, S))
    Ht = S3 @ H @ S3.T
    B, I = boundary_interior(p)
    cond = Ht[np.ix_(B, I)] @ np.linalg.solve(Ht[np.ix_(I, I)], Ht[np.ix_(I, B)])
    _, K = mass_stiffness(p)
    Kt = S @ K @ S.T
    Kt0, Ktp = Kt[1:p, 0], Kt[1:p, p]
    rng = np.random.default_rng(p)
    faces = {key: rng.standard_normal((n, n)) for key in FACE_NODES}
    # same data as a boundary vector for the dense operator
    pos = {int(g): t for t, g in enumerate(B)}
    uB = np.zeros(len(B))
    for key, F in faces.items():
        for r in range(n):
            for c in range(n):
                uB[pos[int(local_index(p, *FACE_NODES[key](r, c, p)))]] = F[r, c]
    ref = cond @ uB
    cnt = Counter()
    out = table2_condensed(p, d, lam, Kt0, Ktp, faces, cnt)
    for key, F in out.items():
        for r in range(n):
            for c in range(n):
                g = pos[int(local_index(p, *FACE_NODES[key](r, c, p)))]
                assert F[r][c] == pytest.approx(ref[g], rel=1e-10, abs=1e-12 * np.abs(ref).max())
    # Table 3, TPT condensed part: 13 n^3 multiplications (+ 12 n^2 for the
    # metric factors folded into the faces)
    assert cnt.n == 13 * n ** 3 + 12 * n ** 2
