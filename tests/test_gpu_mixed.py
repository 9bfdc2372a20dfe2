"""Mixed precision (FP32 inner CG inside FP64 iterative refinement) against
the FP64 oracle: solutions within 1e-9 relative, the FP64 residual history
of the refinement, and the error after each refinement step."""
import numpy as np
import pytest

import sem_inputs as si
from oracle import dense, local
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-9


def _mixed(**kw):
    from paper_1601_08179_gb300 import sem
    return sem.default_opts(precision=sem.PREC_MIXED, **kw)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("p,m,lam,ar", [(4, (4, 4, 4), 1.0, 1.0), (6, (3, 3, 3), 0.0, 8.0),
                                        (8, (3, 2, 2), 10.0, 16.0), (2, (5, 4, 3), 0.5, 4.0)])
def test_mixed_solve_vs_direct(p, m, lam, ar, scheme):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar, opts=_mixed(mixed_scheme=scheme))
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 21).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert relerr(host(u), dense.solve_full(ms, lam, f)) <= SOLVE_TOL
    hist = sem.sem_refine_history(ctx)
    assert hist[0] == pytest.approx(1.0) and hist[-1] <= 1e-10
    assert np.all(np.diff(hist) < 0)
    assert info["refinements"] == len(hist) - 1 >= 2
    assert info["rel_res"] == hist[-1]


@pytest.mark.parametrize("scheme", [0, 1])
def test_mixed_error_per_refinement_step(scheme):
    """Error against the FP64 oracle after k refinement steps (max_refine = k):
    it falls by orders of magnitude per step down to the 1e-9 bar."""
    import torch
    from paper_1601_08179_gb300 import sem
    p, m, lam, ar = 5, (4, 3, 3), 1.0, 16.0
    ctx, ms = make_pair(p, m, lam, ar, opts=_mixed())
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 22).reshape(X.shape)).ravel()
    ref = dense.solve_full(ms, lam, f)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    errs = []
    for k in range(1, 13):
        sem.sem_set_opts(ctx, _mixed(max_refine=k, mixed_scheme=scheme))
        info = sem.sem_solve(ctx, dev(f), u, check=False)
        errs.append(relerr(host(u), ref))
        if info["status"] == sem.SEM_OK:
            break
    print(f"scheme {scheme}: error vs oracle per refinement step:", ["%.2e" % e for e in errs])
    assert errs[-1] <= SOLVE_TOL
    assert all(b < 0.1 * a for a, b in zip(errs, errs[1:]))


def test_mixed_matches_fp64_path_and_oracle_residual_full_size():
    """p = 16 on 16^3 elements, lambda = 10, aspect ratio 16 (N ~ 1.7e7):
    the uncondensed residual of the recovered field (oracle A u - F) meets
    the solver tolerance."""
    import torch
    from paper_1601_08179_gb300 import sem
    w = si.MIXED
    ctx, ms = make_pair(w.p, w.m, w.lam, w.ar, opts=_mixed())
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, w.lam) + si.node_noise(X.size, w.seed).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    got = host(u)
    F = local.rhs_full(ms, f)
    r = (local.apply_full(ms, w.lam, got) - F)[ms.free_mask]
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(F[ms.free_mask])
    sem.sem_set_opts(ctx, sem.default_opts())
    u64 = torch.empty_like(u)
    sem.sem_solve(ctx, dev(f), u64)
    d = relerr(got, host(u64))
    print("mixed vs fp64 relative difference", d, "refinements", info["refinements"])
    assert d <= 1e-7
