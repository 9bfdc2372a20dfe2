"""The pencil kernel (SEM_KERNEL_PENCIL: a thread per x-pencil, then a thread
per cube column; FP32, 5 <= n <= 8) against the FP64 oracle.

It computes the transformed condensed operator of Sec. 6 / Table 2 like the
other variants; covered here: every degree it serves, rounds whose last
elements lie past the mesh (element counts not a multiple of 256 / n^2),
rows of one element, elements with all six faces on the Dirichlet boundary,
aspect ratio 128 entry by entry, mixed solves with it, and the p = 8
benchmark mesh against the FP64 operator.
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import local, transform
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _oracle_apply(ms, lam, ut):
    free = ms.skeleton_free
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    return transform.load_to_transformed(ms, np.where(free, local.apply_condensed(ms, lam, u_nodal), 0.0))


def _apply(ctx, ut):
    import torch
    from paper_1601_08179_gb300 import sem
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    return host(v)


def _pencil_ctx(p, m, lam, ar, opts=None):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar, opts=opts)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PENCIL)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_PENCIL
    return ctx, ms


PENCIL_CASES = [  # p (n = p - 1 in 5..8), elements, lambda, aspect ratio; E = 256 // n^2 per round
    (6, (3, 2, 2), 10.0, 1.0),     # n = 5: 10 elements per round, 12 elements (2 rounds, ragged)
    (7, (2, 2, 3), 0.5, 2.0),      # n = 6: 7 per round
    (8, (3, 3, 3), 0.0, 8.0),      # n = 7 (the benchmark degree): 5 per round, 27 elements
    (9, (2, 3, 2), 1.0, 1.5),      # n = 8: 4 per round
    (8, (7, 3, 2), 100.0, 16.0),   # 42 elements, graded, lambda = 1e2
    (8, (1, 3, 2), 1.0, 1.0),      # rows of one element
    (7, (5, 1, 1), 2.0, 4.0),      # one row
    (8, (1, 1, 1), 1.0, 1.0),      # one element: every face on the boundary
]


@pytest.mark.parametrize("p,m,lam,ar", PENCIL_CASES)
def test_pencil_kernel_vs_oracle(p, m, lam, ar):
    ctx, ms = _pencil_ctx(p, m, lam, ar)
    ut = si.random_vector(ms.n_skeleton, 1700 + p).astype(np.float32).astype(np.float64)
    got = _apply(ctx, ut)
    ref = _oracle_apply(ms, lam, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    if np.linalg.norm(ref) == 0.0:
        assert np.linalg.norm(got) == 0.0
        return
    err = relerr(got, ref)
    print(f"pencil p={p} m={m}: {err:.2e}")
    assert err <= F32_TOL


@pytest.mark.parametrize("p", [6, 8, 9])
def test_pencil_kernel_entrywise_high_aspect_ratio(p):
    """x-graded to aspect ratio 128, entry by entry (floor 1e-3 of the
    largest entry), the bar of the other FP32 kernels."""
    m = {6: (9, 2, 2), 8: (8, 2, 2), 9: (7, 2, 2)}[p]
    ctx, ms = _pencil_ctx(p, m, 0.0, 128.0)
    ut = si.random_vector(ms.n_skeleton, 1800 + p).astype(np.float32).astype(np.float64)
    got, ref = _apply(ctx, ut), _oracle_apply(ms, 0.0, ut)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    worst = float(np.max(np.abs(got - ref) / scale))
    print(f"pencil p={p}: worst entry-wise error {worst:.2e}")
    assert worst <= 1e-4


def test_pencil_kernel_refuses_other_degrees():
    from paper_1601_08179_gb300 import sem
    for p in (3, 5, 10):
        ctx, _ = make_pair(p, (2, 2, 2), 1.0, 1.0)
        with pytest.raises(sem.SemError):
            sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PENCIL)


@pytest.mark.parametrize("p,m,lam,ar", [(8, (5, 3, 3), 1.0, 8.0), (6, (6, 4, 3), 0.0, 16.0), (9, (3, 4, 2), 100.0, 1.0)])
def test_mixed_solve_with_the_pencil_kernel(p, m, lam, ar):
    import torch
    from oracle import dense
    from paper_1601_08179_gb300 import sem
    ctx, ms = _pencil_ctx(p, m, lam, ar, opts=sem.default_opts(precision=sem.PREC_MIXED))
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 1900 + p).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["rel_res"] <= 1e-10
    assert relerr(host(u), dense.solve_full(ms, lam, f)) <= 1e-9


def test_pencil_kernel_at_benchmark_size_matches_fp64_operator():
    """p = 8 on the graded 32^3 mesh (6554 rounds of 5 elements, the launch a
    mixed solve takes with this kernel) against the FP64 operator of the same
    context on the same FP32-representable input."""
    import torch
    from paper_1601_08179_gb300 import build, sem
    build.build()
    w = si.scale_workload(8)
    hx, hy, hz = w.widths()
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam, sem.default_opts(precision=sem.PREC_MIXED))
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PENCIL)
    x32 = torch.tensor(si.random_vector(ctx.nb, 2000), dtype=torch.float32, device="cuda")
    v64 = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, x32.double(), v64, sem.SPACE_TRANSFORMED)
    v32 = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, x32, v32)
    got, ref = host(v32), host(v64)
    assert relerr(got, ref) <= F32_TOL
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-3
