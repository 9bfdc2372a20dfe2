"""Every operator kernel variant against the FP64 oracle, through the C ABI.

The variants (SEM_KERNEL_CTA_TILE, _WARP, _PLANE, _ELEMENT, _SLAB) compute the same
transformed condensed operator (Sec. 6, Table 2) with different work
mappings; each is selected explicitly with sem_set_operator_kernel and
compared with the oracle's element-local tier on every skeleton entry.
Meshes have element counts that are not multiples of the elements per warp
or CTA tile (ragged tails) and graded widths (several width classes).
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import local, transform
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5      # FP32 rounding of one application (relative, 2-norm)
F64_TOL = 1e-12


def _oracle_apply(ms, lam, ut):
    free = ms.skeleton_free
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    return transform.load_to_transformed(ms, np.where(free, local.apply_condensed(ms, lam, u_nodal), 0.0))


def _check_f32(ctx, ms, lam, seed):
    import torch
    from paper_1601_08179_gb300 import sem
    ut = si.random_vector(ms.n_skeleton, seed).astype(np.float32).astype(np.float64)
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    got = host(v)
    ref = _oracle_apply(ms, lam, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    return relerr(got, ref)


PLANE_CASES = [  # p (n = p - 1 in 2..8), elements, lambda, aspect ratio
    (3, (3, 2, 3), 1.0, 3.0),
    (4, (3, 3, 2), 0.0, 4.0),     # G = 4 lanes, 8 elements per warp, 18 elements
    (5, (2, 3, 3), 2.5, 2.0),
    (6, (3, 2, 2), 10.0, 1.0),    # G = 8 lanes, n = 5: three idle lanes per group
    (7, (2, 2, 3), 0.5, 2.0),
    (8, (3, 3, 3), 0.0, 8.0),     # the benchmark degree
    (9, (2, 3, 2), 1.0, 1.5),     # n = 8 fills the group
    (10, (3, 2, 2), 2.0, 4.0),    # two half-rows per plane from here on (9 <= n <= 15)
    (12, (2, 2, 3), 0.0, 2.0),
    (16, (3, 2, 1), 1.0, 8.0),    # n = 15, the mixed-precision workload's degree
]


@pytest.mark.parametrize("p,m,lam,ar", PLANE_CASES)
def test_plane_kernel_vs_oracle(p, m, lam, ar):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PLANE)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_PLANE
    err = _check_f32(ctx, ms, lam, 300 + p)
    print(f"plane p={p}: {err:.2e}")
    assert err <= F32_TOL


@pytest.mark.parametrize("p,m,lam,ar", [(16, (7, 1, 1), 1.0, 4.0), (12, (13, 12, 12), 2.0, 16.0)])
def test_plane2_kernel_uneven_warp_counts(p, m, lam, ar):
    """The two-half-row kernel with element counts that do not divide over
    the warps: 7 elements over 9 warps (two idle), and 1872 elements over the
    full grid (one or two elements per warp)."""
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PLANE)
    err = _check_f32(ctx, ms, lam, 900 + p)
    print(f"plane2 p={p} m={m}: {err:.2e}")
    assert err <= F32_TOL


def test_plane_kernel_many_warps_ragged():
    """p = 8 on 9 x 7 x 5 = 315 elements (79 element groups over many warps,
    the last group one element short), x-graded to aspect ratio 32."""
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(8, (9, 7, 5), 1.0, 32.0)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_PLANE)
    assert _check_f32(ctx, ms, 1.0, 17) <= F32_TOL


SLAB_CASES = [  # p (n = p - 1 in 16..31), elements, lambda, aspect ratio
    (17, (2, 2, 2), 1.0, 2.0),    # n = 16: two full slabs of 8 planes, half of each row idle
    (18, (3, 2, 2), 0.0, 4.0),    # n = 17: the third slab holds one plane
    (25, (2, 2, 3), 2.5, 8.0),    # n = 24: three full slabs
    (26, (2, 3, 2), 0.5, 3.0),    # n = 25: four slabs, the last with one plane
    (32, (2, 2, 2), 1.0, 8.0),    # n = 31, the highest degree: last slab 7 planes, one idle lane per row
    (32, (3, 2, 1), 10.0, 32.0),
]


@pytest.mark.parametrize("p,m,lam,ar", SLAB_CASES)
def test_slab_kernel_vs_oracle(p, m, lam, ar):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_SLAB)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_SLAB
    err = _check_f32(ctx, ms, lam, 700 + p)
    print(f"slab p={p}: {err:.2e}")
    assert err <= F32_TOL


ELEM_CASES = [  # p (n = p - 1 in 2, 3), elements, lambda, aspect ratio
    (3, (3, 2, 3), 1.0, 3.0),
    (3, (2, 2, 2), 10.0, 1.0),
    (4, (3, 3, 2), 0.0, 4.0),
    (4, (2, 3, 3), 2.5, 16.0),
    (4, (37, 5, 3), 1.0, 8.0),    # 555 elements: several per thread, ragged last warp
]


@pytest.mark.parametrize("p,m,lam,ar", ELEM_CASES)
def test_element_kernel_fp32_vs_oracle(p, m, lam, ar):
    """The FP32 thread-per-element kernel at n = 2, 3 (boundary values,
    eigenspace points and contractions of an element in one thread)."""
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ELEMENT)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_ELEMENT
    err = _check_f32(ctx, ms, lam, 800 + p)
    print(f"element p={p}: {err:.2e}")
    assert err <= F32_TOL


def test_mixed_solve_with_the_element_kernel():
    """Mixed-precision solve at p = 4 with the FP32 thread-per-element
    operator against the dense oracle."""
    import torch
    from oracle import dense
    from paper_1601_08179_gb300 import sem
    p, m, lam, ar = 4, (3, 2, 3), 1.0, 8.0
    ctx, ms = make_pair(p, m, lam, ar, opts=sem.default_opts(precision=sem.PREC_MIXED))
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ELEMENT)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 37).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["refinements"] >= 1
    assert relerr(host(u), dense.solve_full(ms, lam, f)) <= 1e-9


def test_slab_kernel_many_units_ragged():
    """p = 20 on 5 x 3 x 4 = 60 elements x 3 slabs = 180 work units, more than
    one unit per CTA on most CTAs and unequal unit counts, x-graded to aspect
    ratio 16."""
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(20, (5, 3, 4), 1.0, 16.0)
    assert _check_f32(ctx, ms, 1.0, 19) <= F32_TOL


@pytest.mark.parametrize("p,m,ar", [(32, (8, 8, 8), 128.0), (17, (33, 32, 32), 8.0)])
def test_slab_kernel_at_scale_matches_fp64_operator(p, m, ar):
    """The k-slab FP32 operator at the p = 32 benchmark size (2048 units, one
    per CTA, the launch the bench times) and past 65536 units (p = 17 on
    33 x 32 x 32 = 67584 units: CTAs take ranges of units), against the FP64
    operator of the same context on the same FP32-representable input (both
    checked against the oracle at small sizes): equal to FP32 rounding in the
    2-norm and entry by entry (floor 1e-3 of the largest entry)."""
    import torch
    from paper_1601_08179_gb300 import build, sem
    build.build()
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar, grade="x")
    ctx = sem.sem_setup(p, hx, hy, hz, 0.0, sem.default_opts(precision=sem.PREC_MIXED))
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_SLAB
    x32 = torch.tensor(si.random_vector(ctx.nb, 77 + p), dtype=torch.float32, device="cuda")
    v64 = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, x32.double(), v64, sem.SPACE_TRANSFORMED)
    v32 = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, x32, v32)
    got, ref = host(v32), host(v64)
    assert relerr(got, ref) <= F32_TOL
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-3


@pytest.mark.parametrize("p,m,lam,ar", [(4, (3, 2, 3), 1.0, 3.0), (6, (2, 3, 2), 0.0, 2.0),
                                        (8, (3, 2, 2), 2.0, 4.0)])
def test_warp_kernel_vs_oracle(p, m, lam, ar):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_WARP)
    assert _check_f32(ctx, ms, lam, 400 + p) <= F32_TOL


@pytest.mark.parametrize("p,m,epb,ks", [(3, (3, 2, 3), 5, 1), (8, (3, 2, 2), 3, 4), (8, (3, 2, 2), 1, 7),
                                        (12, (2, 2, 1), 2, 6), (2, (3, 2, 4), 7, 1)])
def test_cta_tile_fp32_vs_oracle(p, m, epb, ks):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, 1.0, 2.0)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_CTA_TILE, epb, ks)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED) == (sem.KERNEL_CTA_TILE, epb, ks)
    assert _check_f32(ctx, ms, 1.0, 500 + p) <= F32_TOL


@pytest.mark.parametrize("p,m,epb,ks", [(8, (3, 2, 2), 3, 3),    # n = 7: slabs start at k = 0, 3, 6
                                        (4, (3, 3, 2), 6, 1),    # n = 3: every slab one plane
                                        (6, (2, 3, 2), 2, 2),    # n = 5: degree not compiled in
                                        (9, (2, 2, 2), 2, 5),    # n = 8
                                        (3, (3, 2, 3), 4, 1),    # n = 2
                                        (10, (2, 2, 1), 1, 9)])  # n = 9
def test_cta_tile_fp64_shapes_vs_oracle(p, m, epb, ks):
    """FP64 CTA tiles of chosen shapes (elements per CTA, k-slab depth: the
    autotuner's search space) against the oracle at 1e-12, with k-slabs
    that start at odd planes and degrees served by the run-time-n kernel
    (Sec. 6 / Table 2)."""
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, 1.5, 8.0)
    sem.sem_set_operator_kernel(ctx, sem.PREC_FP64, sem.KERNEL_CTA_TILE, epb, ks)
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_FP64) == (sem.KERNEL_CTA_TILE, epb, ks)
    ut = si.random_vector(ms.n_skeleton, 650 + p)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    got, ref = host(v), _oracle_apply(ms, 1.5, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    err = relerr(got, ref)
    print(f"cta fp64 p={p} epb={epb} ks={ks}: {err:.2e}")
    assert err <= F64_TOL


@pytest.mark.parametrize("kind,epb,ks", [("cta", 1, 1), ("cta", 4, 1), ("element", 0, 0)])
def test_p2_variants_fp64_vs_oracle(kind, epb, ks):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(2, (5, 3, 4), 0.5, 4.0)
    k = sem.KERNEL_CTA_TILE if kind == "cta" else sem.KERNEL_ELEMENT
    sem.sem_set_operator_kernel(ctx, sem.PREC_FP64, k, epb, ks)
    ut = si.random_vector(ms.n_skeleton, 61)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    assert relerr(host(v), _oracle_apply(ms, 0.5, ut)) <= F64_TOL


def test_defaults_and_rejected_variants():
    from paper_1601_08179_gb300 import sem
    ctx8, _ = make_pair(8, (2, 2, 2), 1.0)
    assert sem.sem_get_operator_kernel(ctx8, sem.PREC_FP64)[0] == sem.KERNEL_CTA_TILE
    assert sem.sem_get_operator_kernel(ctx8, sem.PREC_MIXED)[0] == sem.KERNEL_PLANE
    ctx2, _ = make_pair(2, (2, 2, 2), 1.0)
    assert sem.sem_get_operator_kernel(ctx2, sem.PREC_FP64)[0] == sem.KERNEL_ELEMENT
    ctx3, _ = make_pair(3, (2, 2, 2), 1.0)
    assert sem.sem_get_operator_kernel(ctx3, sem.PREC_MIXED)[0] == sem.KERNEL_ELEMENT
    assert sem.sem_get_operator_kernel(ctx3, sem.PREC_FP64)[0] == sem.KERNEL_CTA_TILE
    ctx4, _ = make_pair(4, (2, 2, 2), 1.0)
    assert sem.sem_get_operator_kernel(ctx4, sem.PREC_MIXED)[0] == sem.KERNEL_PLANE
    ctx16, _ = make_pair(16, (1, 1, 1), 1.0)
    assert sem.sem_get_operator_kernel(ctx16, sem.PREC_MIXED)[0] == sem.KERNEL_PLANE
    ctx17, _ = make_pair(17, (1, 1, 1), 1.0)
    assert sem.sem_get_operator_kernel(ctx17, sem.PREC_MIXED)[0] == sem.KERNEL_SLAB
    assert sem.sem_get_operator_kernel(ctx17, sem.PREC_FP64)[0] == sem.KERNEL_CTA_TILE
    bad = [(ctx8, sem.PREC_FP64, sem.KERNEL_PLANE, 0, 0),     # FP32-only variants
           (ctx8, sem.PREC_FP64, sem.KERNEL_WARP, 0, 0),
           (ctx8, sem.PREC_MIXED, sem.KERNEL_ELEMENT, 0, 0),  # n <= 3 only
           (ctx3, sem.PREC_FP64, sem.KERNEL_ELEMENT, 0, 0),   # FP64: n = 1 only
           (ctx17, sem.PREC_MIXED, sem.KERNEL_PLANE, 0, 0),   # n = 16 > 15
           (ctx16, sem.PREC_MIXED, sem.KERNEL_WARP, 0, 0),    # n = 15 > 7
           (ctx16, sem.PREC_MIXED, sem.KERNEL_SLAB, 0, 0),    # n = 15 < 16
           (ctx17, sem.PREC_FP64, sem.KERNEL_SLAB, 0, 0),     # FP32 only
           (ctx2, sem.PREC_MIXED, sem.KERNEL_WARP, 0, 0),     # n = 1 < 3
           (ctx8, sem.PREC_FP64, sem.KERNEL_CTA_TILE, 0, 7),  # epb out of range
           (ctx8, sem.PREC_FP64, sem.KERNEL_CTA_TILE, 4, 8),  # ks > n
           (ctx8, sem.PREC_FP64, 9, 0, 0),                    # no such kind
           (ctx8, 5, sem.KERNEL_AUTO, 0, 0)]                  # no such precision
    for c, prec, kind, epb, ks in bad:
        with pytest.raises(sem.SemError) as ei:
            sem.sem_set_operator_kernel(c, prec, kind, epb, ks)
        assert ei.value.status == sem.SEM_EINVAL
    # a rejected call leaves the choice unchanged; AUTO restores the default
    sem.sem_set_operator_kernel(ctx8, sem.PREC_MIXED, sem.KERNEL_WARP)
    assert sem.sem_get_operator_kernel(ctx8, sem.PREC_MIXED)[0] == sem.KERNEL_WARP
    sem.sem_set_operator_kernel(ctx8, sem.PREC_MIXED, sem.KERNEL_AUTO)
    assert sem.sem_get_operator_kernel(ctx8, sem.PREC_MIXED)[0] == sem.KERNEL_PLANE


@pytest.mark.parametrize("kind", ["plane", "warp", "cta"])
def test_mixed_solve_with_each_fp32_kernel(kind):
    """The mixed-precision solve (FP32 inner CG, FP64 refinement) reaches the
    FP64 oracle's solution to the solve bar with each FP32 operator kernel."""
    import torch
    from oracle import dense
    from paper_1601_08179_gb300 import sem
    p, m, lam, ar = 6, (3, 2, 3), 1.0, 8.0
    ctx, ms = make_pair(p, m, lam, ar, opts=sem.default_opts(precision=sem.PREC_MIXED))
    k = {"plane": sem.KERNEL_PLANE, "warp": sem.KERNEL_WARP, "cta": sem.KERNEL_CTA_TILE}[kind]
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, k, 4 if kind == "cta" else 0, 5 if kind == "cta" else 0)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 23).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["refinements"] >= 1
    assert relerr(host(u), dense.solve_full(ms, lam, f)) <= 1e-9


def test_mixed_solve_with_the_slab_kernel():
    """Mixed-precision solve at p = 20 (n = 19, the k-slab FP32 kernel by
    default) against the oracle's factorized PCG at rtol 1e-13."""
    import torch
    from oracle import solve as osolve
    from paper_1601_08179_gb300 import sem
    p, m, lam, ar = 20, (2, 2, 2), 1.0, 4.0
    ctx, ms = make_pair(p, m, lam, ar, opts=sem.default_opts(precision=sem.PREC_MIXED))
    assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == sem.KERNEL_SLAB
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 29).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["refinements"] >= 1
    ref = osolve.bt_solve(ms, lam, f, rtol=1e-13)[0]
    assert relerr(host(u), ref) <= 1e-9


@pytest.mark.parametrize("p", [2, 3, 4, 5, 8, 12, 16, 24, 32])
def test_f32_apply_entrywise_high_aspect_ratio(p):
    """FP32 operator on an x-graded mesh of aspect ratio 128 (metric factors
    d_1 : d_2 up to ~1.6e4 within one element), entry by entry (floor 1e-3 of
    the largest entry), so a coefficient formed with cancellation in FP32 shows
    even where the 2-norm would hide it.  The bar grows with the degree: the
    primary and condensed parts cancel more at high n and aspect ratio
    (measured worst entries ~2e-5 at p <= 8, ~3e-4 at p = 12)."""
    import torch
    from paper_1601_08179_gb300 import sem
    m = {2: (12, 3, 2), 3: (10, 3, 2), 4: (9, 2, 2), 5: (8, 2, 2), 8: (8, 2, 2), 12: (6, 1, 1), 16: (5, 1, 1), 24: (4, 2, 1),
         32: (4, 1, 2)}[p]
    ctx, ms = make_pair(p, m, 0.0, 128.0)
    ut = si.random_vector(ms.n_skeleton, 600 + p).astype(np.float32).astype(np.float64)
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    got, ref = host(v), _oracle_apply(ms, 0.0, ut)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    worst = float(np.max(np.abs(got - ref) / scale))
    print(f"p={p}: worst entry-wise error {worst:.2e}")
    assert worst <= (1e-4 if p <= 9 else 1e-3)
    if p in (3, 4):   # the thread-per-element kernel as well
        sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, sem.KERNEL_ELEMENT)
        sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
        assert float(np.max(np.abs(host(v) - ref) / scale)) <= 1e-4


THIN_CASES = [  # kernel, p, elements: one element thick in x, or a single row or column of elements
    ("ELEMENT", 2, (1, 4, 3)), ("ELEMENT", 2, (7, 1, 1)), ("ELEMENT", 3, (1, 3, 4)), ("ELEMENT", 4, (1, 1, 9)),
    ("PLANE", 4, (1, 5, 3)), ("PLANE", 4, (11, 1, 2)), ("PLANE", 8, (1, 2, 3)), ("PLANE", 8, (9, 1, 1)),
    ("PLANE", 12, (1, 2, 2)), ("PLANE", 16, (1, 1, 3)), ("WARP", 6, (1, 2, 3)),
    ("SLAB", 20, (1, 2, 2)), ("SLAB", 20, (3, 1, 1)), ("SLAB", 32, (1, 1, 2)),
]


@pytest.mark.parametrize("kind,p,m", THIN_CASES)
def test_f32_kernels_on_thin_meshes(kind, p, m):
    """Meshes one element thick in x (both x-faces of every element on the
    Dirichlet boundary) and single rows or columns of elements: the x-fastest
    element order, the affine entity offsets and the boundary masks of every
    FP32 kernel, against the oracle (uniform widths where x has one element,
    else graded in x to aspect ratio 4)."""
    from paper_1601_08179_gb300 import sem
    ar = 1.0 if m[0] == 1 else 4.0
    ctx, ms = make_pair(p, m, 1.5, ar)
    sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, getattr(sem, "KERNEL_" + kind))
    err = _check_f32(ctx, ms, 1.5, 900 + p)
    print(f"{kind.lower()} p={p} m={m}: {err:.2e}")
    assert err <= F32_TOL


@pytest.mark.parametrize("p,m", [(2, (1, 3, 4)), (4, (1, 3, 2)), (8, (5, 1, 1)), (8, (1, 1, 4)), (20, (1, 2, 1))])
def test_f64_kernels_on_thin_meshes(p, m):
    """The FP64 operator (thread per element at p = 2, CTA tile above) on the
    same kinds of thin meshes, at the 1e-12 apply bar."""
    import torch
    from paper_1601_08179_gb300 import sem
    ar = 1.0 if m[0] == 1 else 4.0
    ctx, ms = make_pair(p, m, 0.5, ar)
    ut = si.random_vector(ms.n_skeleton, 950 + p)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    got, ref = host(v), _oracle_apply(ms, 0.5, ut)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    assert relerr(got, ref) <= 1e-12
