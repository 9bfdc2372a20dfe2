"""The parameter grid of the graded-mesh workloads on small meshes.

The full-size sweep runs degrees 2 ... 32 with elements graded along x to a
maximum aspect ratio of 1, 8 or 128 and lambda = 0 or 1e2.  Here every
(aspect ratio, lambda) pair of that grid, at degrees 2, 4 and 8, is checked
against the dense Schur-complement oracle on a small mesh of the same kind:
the FP64 operator (1e-12), the FP32 operator (FP32 rounding, 1e-5), and the
FP64 and mixed-precision solves against a direct solve of the uncondensed
system (1e-9).  The paper's solver tests use the same aspect-ratio series
(Sec. 8); lambda = 1e2 is the implicit-time-step regime where the mass term
dominates the metric terms on coarse elements.
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import dense, transform
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

MESH = {2: (6, 3, 2), 4: (5, 2, 2), 8: (4, 2, 2)}    # graded along x
CUBE = {2: (3, 3, 3), 4: (3, 3, 3), 8: (2, 2, 2)}    # aspect ratio 1: equal widths on every axis


def _mesh(p, ar):
    return CUBE[p] if ar == 1.0 else MESH[p]


GRID = [(p, ar, lam) for p in (2, 4, 8) for ar in (1.0, 8.0, 128.0) for lam in (0.0, 100.0)]


def _transformed_ref(ms, lam, ut):
    A = dense.assemble_condensed(ms, lam)
    free = ms.skeleton_free
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    return transform.load_to_transformed(ms, np.where(free, A @ np.where(free, u_nodal, 0.0), 0.0))


@pytest.mark.parametrize("p,ar,lam", GRID)
def test_operator_fp64_and_fp32(p, ar, lam):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, _mesh(p, ar), lam, ar)
    ut = si.random_vector(ms.n_skeleton, 700 + p).astype(np.float32).astype(np.float64)
    ref = _transformed_ref(ms, lam, ut)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    got = host(v)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    assert relerr(got, ref) <= 1e-12
    v32 = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v32)
    got32 = host(v32)
    assert np.all(got32[~ms.skeleton_free] == 0.0)
    assert relerr(got32, ref) <= 1e-5


@pytest.mark.parametrize("p,ar,lam", GRID)
def test_solve_fp64_and_mixed(p, ar, lam):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, _mesh(p, ar), lam, ar)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 800 + p).reshape(X.shape)).ravel()
    ref = dense.solve_full(ms, lam, f)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert relerr(host(u), ref) <= 1e-9
    assert info["rel_res"] <= 1e-10
    sem.sem_set_opts(ctx, sem.default_opts(precision=sem.PREC_MIXED))
    info = sem.sem_solve(ctx, dev(f), u)
    assert relerr(host(u), ref) <= 1e-9
    assert info["rel_res"] <= 1e-10
