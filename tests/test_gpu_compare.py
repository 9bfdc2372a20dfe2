"""The paper's comparison variants (Sec. 5, Sec. 8) against the dense oracle.

TPC (Algorithm 3 with Table 1) and MMC (Algorithm 2) compute the same nodal
condensed operator as the transformed operator between skeleton transforms;
each is compared entry by entry with the dense Schur complement (1e-12).  The
nodal diagonal (the DC preconditioner) is compared with the diagonal of the
assembled dense operator.  The CG solves with every operator and
preconditioner (UC: none, DC: diagonal, BC: block-Jacobi over faces, edges
and vertices) reach the solve bar against a direct solve of the uncondensed
system; BC takes the iterations of the transformed diagonal preconditioner
(BT) - the two preconditioned systems are congruent (Sec. 8) - and DC at
least as many.
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import dense
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

CASES = [  # p, elements, lambda, aspect ratio
    (2, (3, 2, 2), 1.0, 2.0),
    (3, (2, 3, 2), 0.0, 4.0),
    (4, (3, 2, 3), 2.5, 1.0),
    (5, (2, 2, 2), 100.0, 8.0),
    (8, (3, 2, 2), 0.5, 2.0),
    (9, (2, 1, 2), 1.0, 1.0),
]


@pytest.mark.parametrize("p,m,lam,ar", CASES)
def test_operator_variants_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    u = si.random_vector(ms.n_skeleton, 2000 + p)
    ref = dense.apply_condensed(ms, lam, u)
    base = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(u), base, sem.SPACE_NODAL)
    for op in (sem.OP_TPT, sem.OP_TPC, sem.OP_MMC):
        v = torch.full((ctx.nb,), np.nan, dtype=torch.float64, device="cuda")
        sem.sem_apply_condensed_variant(ctx, op, dev(u), v)
        got = host(v)
        assert np.all(got[~ms.skeleton_free] == 0.0), op
        err = relerr(got, ref)
        print(f"p={p} op={op}: {err:.2e}")
        assert err <= 1e-12, op
    assert relerr(host(base), ref) <= 1e-12


@pytest.mark.parametrize("p,m,lam,ar", CASES[:4])
def test_nodal_diagonal_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    d = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_diag_nodal(ctx, d)
    ref = np.where(ms.skeleton_free, dense.assemble_condensed(ms, lam).diagonal(), 0.0)
    got = host(d)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    assert relerr(got, ref) <= 1e-12
    assert np.all(got[ms.skeleton_free] > 0.0)


@pytest.mark.parametrize("p,m,lam,ar", [(4, (3, 3, 2), 0.0, 8.0), (8, (2, 2, 3), 1.0, 2.0), (3, (4, 2, 2), 100.0, 1.0)])
def test_solvers_vs_direct(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar, opts=sem.default_opts(rtol=1e-12))
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 2100 + p).reshape(X.shape)).ravel()
    ref = dense.solve_full(ms, lam, f)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    bt = sem.sem_solve(ctx, dev(f), u)
    assert relerr(host(u), ref) <= 1e-9
    iters = {}
    for op in (sem.OP_TPT, sem.OP_TPC, sem.OP_MMC):
        for pc in (sem.PC_NONE, sem.PC_DIAG, sem.PC_BLOCK):
            u.fill_(np.nan)
            info = sem.sem_solve_variant(ctx, op, pc, dev(f), u)
            assert relerr(host(u), ref) <= 1e-9, (op, pc)
            assert info["rel_res"] <= 1e-12
            iters[(op, pc)] = info["iters"]
    print("BT", bt["iters"], iters)
    for op in (sem.OP_TPT, sem.OP_TPC, sem.OP_MMC):
        assert abs(iters[(op, sem.PC_BLOCK)] - bt["iters"]) <= 2, (op, iters, bt["iters"])
        assert iters[(op, sem.PC_DIAG)] >= iters[(op, sem.PC_BLOCK)] - 2
        assert iters[(op, sem.PC_NONE)] >= iters[(op, sem.PC_DIAG)] - 2


def test_variants_refused_past_their_degree():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(17, (1, 1, 2), 1.0)
    u = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda")
    v = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda")
    for op in (sem.OP_TPC, sem.OP_MMC):
        with pytest.raises(sem.SemError) as err:
            sem.sem_apply_condensed_variant(ctx, op, u, v)
        assert err.value.status == sem.SEM_ENOTSUP
    sem.sem_apply_condensed_variant(ctx, sem.OP_TPT, u, v)   # the transformed operator takes any degree
