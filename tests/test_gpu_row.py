"""The row kernel (SEM_KERNEL_ROW: one CTA per x-row segment of up to 32
elements, bulk copies in, bulk reduce-adds out) against the FP64 oracle.

It computes the transformed condensed operator of Sec. 6 / Table 2 like every
other variant; what is particular to it, and covered here: rows longer than
32 elements (several segments per row, the x-faces, y- and z-edges and
vertices at segment ends shared between CTAs), rows of one element, ranges
that start or end on the Dirichlet boundary, skeleton ranges whose ends are
not 16-byte aligned (every degree, many meshes), input and output vectors
at different addresses modulo 16 bytes (the kernel then runs as the plane
kernel), the mixed-precision solve with it, and the full p = 8 benchmark
mesh against the FP64 operator.
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


def _row_ctx(p, m, lam, ar, grade="x"):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar, grade=grade)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ROW)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_ROW
    return ctx, ms


def _apply(ctx, ut):
    import torch
    from paper_1601_08179_gb300 import sem
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    return host(v)


ROW_CASES = [  # p (n = p - 1 in 2..8), elements, lambda, aspect ratio
    (3, (5, 3, 2), 1.0, 3.0),
    (4, (3, 3, 2), 0.0, 4.0),
    (5, (7, 2, 3), 2.5, 2.0),
    (6, (3, 2, 2), 10.0, 1.0),
    (7, (2, 2, 3), 0.5, 2.0),
    (8, (6, 3, 3), 0.0, 8.0),      # the benchmark degree
    (9, (3, 3, 2), 1.0, 1.5),      # n = 8: eight warps
    (8, (40, 2, 1), 1.0, 16.0),    # two segments of 20 per row
    (3, (70, 1, 2), 100.0, 4.0),   # three segments of 24, 23, 23
    (4, (33, 2, 2), 0.0, 128.0),   # two segments of 17 and 16, aspect ratio 128
]


@pytest.mark.parametrize("p,m,lam,ar", ROW_CASES)
def test_row_kernel_vs_oracle(p, m, lam, ar):
    ctx, ms = _row_ctx(p, m, lam, ar)
    ut = si.random_vector(ms.n_skeleton, 1000 + p).astype(np.float32).astype(np.float64)
    got = _apply(ctx, ut)
    ref = _oracle_apply(ms, lam, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    err = relerr(got, ref)
    print(f"row p={p} m={m}: {err:.2e}")
    assert err <= F32_TOL


@pytest.mark.parametrize("p,m", [(3, (1, 3, 4)), (8, (1, 2, 2)), (8, (9, 1, 1)), (5, (4, 1, 1)), (4, (1, 1, 1)),
                                 (9, (2, 1, 3))])
def test_row_kernel_thin_meshes(p, m):
    """Rows of one element (both x-faces on the Dirichlet boundary), single
    rows and columns of elements, one element."""
    ar = 1.0 if m[0] == 1 else 4.0
    ctx, ms = _row_ctx(p, m, 1.0, ar)
    ut = si.random_vector(ms.n_skeleton, 1100 + p).astype(np.float32).astype(np.float64)
    got = _apply(ctx, ut)
    ref = _oracle_apply(ms, 1.0, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    if np.linalg.norm(ref) == 0.0:
        assert np.linalg.norm(got) == 0.0
    else:
        assert relerr(got, ref) <= F32_TOL


@pytest.mark.parametrize("p", [3, 5, 8, 9])
def test_row_kernel_entrywise_high_aspect_ratio(p):
    """x-graded to aspect ratio 128, entry by entry (floor 1e-3 of the
    largest entry), the bar of the other FP32 kernels."""
    m = {3: (10, 3, 2), 5: (8, 2, 2), 8: (8, 2, 2), 9: (7, 2, 2)}[p]
    ctx, ms = _row_ctx(p, m, 0.0, 128.0)
    ut = si.random_vector(ms.n_skeleton, 1200 + p).astype(np.float32).astype(np.float64)
    got, ref = _apply(ctx, ut), _oracle_apply(ms, 0.0, ut)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    worst = float(np.max(np.abs(got - ref) / scale))
    print(f"row p={p}: worst entry-wise error {worst:.2e}")
    assert worst <= 1e-4


def test_row_kernel_vectors_misaligned_modulo_16():
    """Input and output 4 bytes apart modulo 16: the bulk engines cannot keep
    both alignments, so the launch runs the plane kernel; same result."""
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = _row_ctx(8, (5, 3, 2), 1.0, 4.0)
    ut = si.random_vector(ms.n_skeleton, 1300).astype(np.float32).astype(np.float64)
    buf = torch.zeros(ctx.nb + 4, dtype=torch.float32, device="cuda")
    x = buf[1:1 + ctx.nb]
    x.copy_(torch.tensor(ut, dtype=torch.float32, device="cuda"))
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    assert (x.data_ptr() - v.data_ptr()) % 16 != 0
    sem.sem_apply_condensed_f32(ctx, x, v)
    assert relerr(host(v), _oracle_apply(ms, 1.0, ut)) <= F32_TOL


@pytest.mark.parametrize("p,m,lam,ar", [(8, (5, 3, 3), 1.0, 8.0), (4, (40, 3, 2), 0.0, 16.0), (6, (3, 4, 2), 100.0, 1.0)])
def test_mixed_solve_with_the_row_kernel(p, m, lam, ar):
    import torch
    from oracle import dense
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar, opts=sem.default_opts(precision=sem.PREC_MIXED))
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ROW)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 1400 + p).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["rel_res"] <= 1e-10
    assert relerr(host(u), dense.solve_full(ms, lam, f)) <= 1e-9


def test_row_kernel_at_benchmark_size_matches_fp64_operator():
    """p = 8 on the graded 32^3 mesh (1024 segments of 32, the launch the
    bench times) against the FP64 operator of the same context on the same
    FP32-representable input: FP32 rounding in the 2-norm and entry by entry."""
    import torch
    from paper_1601_08179_gb300 import build, sem
    build.build()
    w = si.scale_workload(8)
    hx, hy, hz = w.widths()
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam, sem.default_opts(precision=sem.PREC_MIXED))
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ROW)
    x32 = torch.tensor(si.random_vector(ctx.nb, 1500), dtype=torch.float32, device="cuda")
    v64 = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, x32.double(), v64, sem.SPACE_TRANSFORMED)
    v32 = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, x32, v32)
    got, ref = host(v32), host(v64)
    assert relerr(got, ref) <= F32_TOL
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-3
