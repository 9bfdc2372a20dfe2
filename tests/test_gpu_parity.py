"""CUDA path vs the FP64 oracle, through the C ABI (include/sem.h).

Bars: one operator application within 1e-12 relative (2-norm over the
skeleton); solutions within 1e-9 relative; index/layout work bit-exact.
Small meshes compare against the dense Schur-complement oracle; full
benchmark sizes against the element-local oracle tier on every output.
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import dense, local, transform
from oracle.gll import gll
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-12
SOLVE_TOL = 1e-9

SMALL_CASES = [  # p, (mx, my, mz), lambda, aspect ratio
    (2, (2, 2, 2), 1.0, 1.0),
    (2, (3, 2, 4), 0.0, 3.0),
    (3, (2, 3, 2), 2.5, 2.0),
    (4, (4, 4, 4), 1.0, 1.0),
    (4, (3, 1, 2), 0.0, 4.0),
    (5, (2, 2, 3), 10.0, 1.0),
    (7, (2, 2, 2), 0.0, 8.0),
    (8, (3, 2, 2), 1.0, 2.0),
    (4, (1, 1, 1), 1.0, 1.0),
]


@pytest.mark.parametrize("p", [2, 3, 4, 8, 16, 31, 32])
def test_basis_matches_oracle(p):
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, (1, 1, 1), 1.0)
    gx, gw, lam, V = sem.sem_get_basis(ctx)
    x, w = gll(p)
    np.testing.assert_allclose(gx, x, atol=2e-15)
    np.testing.assert_allclose(gw, w, rtol=1e-13)
    lo, Vo = transform.eigenbasis(p)
    np.testing.assert_allclose(lam, lo, rtol=1e-12)
    np.testing.assert_allclose(V, Vo, atol=1e-11 * np.abs(Vo).max())
    # the FP32 plane kernel uses K~_{Ip}[c] = (-1)^c K~_{I0}[c] (a symmetric
    # basis with canonical signs): the library's basis has it, to rounding that
    # grows with p (the FP64 kernels keep both vectors)
    from oracle.gll import mass_stiffness
    _, K = mass_stiffness(p)
    k0, k1 = V.T @ K[1:p, 0], V.T @ K[1:p, p]
    sign = (-1.0) ** np.arange(p - 1)
    np.testing.assert_allclose(k1, sign * k0, rtol=0, atol=3e-11 * np.abs(k0).max())


@pytest.mark.parametrize("p,m", [(2, (2, 3, 2)), (3, (1, 2, 3)), (5, (2, 2, 2))])
def test_pack_unpack_exact(p, m):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, 1.0)
    u = si.random_vector(ms.n_global, 1)
    uB = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_pack_skeleton(ctx, dev(u), uB)
    np.testing.assert_array_equal(host(uB), ms.pack(u))
    full = dev(np.full(ms.n_global, 7.0))
    vB = si.random_vector(ms.n_skeleton, 2)
    sem.sem_unpack_skeleton(ctx, dev(vB), full)
    ref = np.full(ms.n_global, 7.0)
    ref[ms.pack_map] = vB
    np.testing.assert_array_equal(host(full), ref)


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES)
def test_apply_nodal_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    u = si.random_vector(ms.n_skeleton, 3)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(u), v, sem.SPACE_NODAL)
    ref = dense.apply_condensed(ms, lam, u)
    got = host(v)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    if np.linalg.norm(ref) == 0.0:
        assert np.linalg.norm(got) == 0.0
    else:
        assert relerr(got, ref) <= APPLY_TOL


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES[:6])
def test_apply_transformed_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    ut = si.random_vector(ms.n_skeleton, 4)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    A = dense.assemble_condensed(ms, lam)
    free = ms.skeleton_free
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    ref = transform.load_to_transformed(ms, np.where(free, A @ np.where(free, u_nodal, 0.0), 0.0))
    assert relerr(host(v), ref) <= APPLY_TOL


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES[:6])
def test_precond_diag_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    d = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_precond_diag(ctx, d)
    A = dense.assemble_condensed(ms, lam)
    T = transform.T_matrix(ms)
    ref = np.where(ms.skeleton_free, (T @ A @ T.T).diagonal(), 0.0)
    got = host(d)
    assert np.all(got[~ms.skeleton_free] == 0.0)
    assert relerr(got, ref) <= APPLY_TOL
    assert np.all(got[ms.skeleton_free] > 0)


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES)
def test_condense_rhs_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    f = si.node_noise(ms.n_global, 5)
    ref = dense.condensed_rhs(ms, lam, f)
    out = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_condense_rhs(ctx, dev(f), out, sem.SPACE_NODAL)
    got = host(out)
    if np.linalg.norm(ref) == 0:
        assert np.linalg.norm(got) == 0
    else:
        assert relerr(got, ref) <= APPLY_TOL
    sem.sem_condense_rhs(ctx, dev(f), out, sem.SPACE_TRANSFORMED)
    ref_t = transform.load_to_transformed(ms, ref)
    if np.linalg.norm(ref_t) > 0:
        assert relerr(host(out), ref_t) <= APPLY_TOL


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES)
def test_recover_interior_vs_dense(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    f = si.node_noise(ms.n_global, 6)
    uB = si.random_vector(ms.n_skeleton, 7)
    ref = dense.recover_interior(ms, lam, f, uB)
    u = torch.full((ctx.n_nodes,), 3.0, dtype=torch.float64, device="cuda")
    sem.sem_recover_interior(ctx, dev(f), dev(uB), u, sem.SPACE_NODAL)
    assert relerr(host(u), ref) <= APPLY_TOL
    # transformed-space input gives the same field
    ut = transform.solution_to_transformed(ms, np.where(ms.skeleton_free, uB, 0.0))
    sem.sem_recover_interior(ctx, dev(f), dev(ut), u, sem.SPACE_TRANSFORMED)
    assert relerr(host(u), ref) <= 1e-11


@pytest.mark.parametrize("p,m,lam,ar", SMALL_CASES)
def test_solve_vs_direct(p, m, lam, ar):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 8).reshape(X.shape)).ravel()
    ref = dense.solve_full(ms, lam, f)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert relerr(host(u), ref) <= SOLVE_TOL
    assert info["rel_res"] <= 1e-10


def test_small_workload_manufactured():
    """4^3 elements, p = 4, lambda = 1, manufactured right-hand side."""
    import torch
    from paper_1601_08179_gb300 import sem
    w = si.SMALL
    ctx, ms = make_pair(w.p, w.m, w.lam)
    X, Y, Z = ms.coords()
    f = si.manufactured_f(X, Y, Z, w.lam).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    got = host(u)
    uc, _ = dense.solve_condensed(ms, w.lam, f)
    assert relerr(got, uc) <= SOLVE_TOL
    err = np.abs(got - si.manufactured_u(X, Y, Z).ravel()).max()
    assert err < 2e-3
    assert 0 < info["iters"] < 200


def test_solve_single_element_has_no_skeleton_unknowns():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(6, (1, 1, 1), 2.0)
    f = si.node_noise(ms.n_global, 9)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    assert info["iters"] == 0
    assert relerr(host(u), dense.solve_full(ms, 2.0, f)) <= SOLVE_TOL


def test_warm_start_and_set_lambda():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(4, (3, 3, 2), 1.0, 2.0)
    f = si.node_noise(ms.n_global, 10)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    sem.sem_set_lambda(ctx, 5.0)
    info0 = sem.sem_solve(ctx, dev(f), u)
    ref = dense.solve_full(ms, 5.0, f)
    assert relerr(host(u), ref) <= SOLVE_TOL
    u0 = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_pack_skeleton(ctx, u, u0)
    info1 = sem.sem_solve(ctx, dev(f), u, u0=u0)
    assert info1["iters"] < info0["iters"]
    assert relerr(host(u), ref) <= SOLVE_TOL


@pytest.mark.parametrize("p", [2, 3, 4, 8, 17])
def test_set_lambda_refreshes_every_operator_table(p):
    """sem_set_lambda rebuilds the class tables of every operator kernel
    (per-class blocks, their transposed copies for the thread-per-element
    kernels, the plane and k-slab blocks): FP64 and FP32 applications at the
    new lambda against the oracle."""
    import torch
    from paper_1601_08179_gb300 import sem
    m = {2: (4, 3, 2), 3: (3, 2, 3), 4: (3, 2, 2), 8: (2, 3, 2), 17: (2, 2, 1)}[p]
    ctx, ms = make_pair(p, m, 1.0, 3.0, opts=sem.default_opts(precision=sem.PREC_MIXED))
    ut = si.random_vector(ms.n_skeleton, 95).astype(np.float32).astype(np.float64)
    v32 = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v32)   # tables at lambda = 1
    sem.sem_set_lambda(ctx, 40.0)
    free = ms.skeleton_free
    ref = transform.load_to_transformed(
        ms, np.where(free, local.apply_condensed(ms, 40.0, transform.solution_from_transformed(ms, np.where(free, ut, 0.0))), 0.0))
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    assert relerr(host(v), ref) <= APPLY_TOL
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v32)
    assert relerr(host(v32), ref) <= 1e-5


@pytest.mark.parametrize("mixed", [False, True])
def test_solve_host_buffers(mixed):
    """sem_solve_host (host load in, host solution out, copies inside): two
    calls with different loads (the second reuses the context's device
    fields), each equal to the device-buffer solve and within the solve bar
    of the dense oracle."""
    import torch
    from paper_1601_08179_gb300 import sem
    opts = sem.default_opts(precision=sem.PREC_MIXED) if mixed else None
    ctx, ms = make_pair(5, (3, 2, 2), 2.0, 3.0, opts=opts)
    for seed in (41, 42):
        f = si.node_noise(ms.n_global, seed)
        u_host = np.zeros(ctx.n_nodes)
        sem.sem_solve_host(ctx, np.ascontiguousarray(f), u_host)
        u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
        sem.sem_solve(ctx, dev(f), u)
        assert relerr(u_host, host(u)) <= 1e-10   # equal up to the order of atomic adds
        assert relerr(u_host, dense.solve_full(ms, 2.0, f)) <= SOLVE_TOL


def test_vector_arguments_are_checked_before_any_launch():
    """Every entry point checks each device vector as sem_check_vector does
    (device memory of the context's device, aligned to its entry size).  A
    host array, pinned host memory and misaligned or null addresses are
    refused; each is first shown to fail sem_check_vector (which launches
    nothing) before an entry point is given it, and the entry point then
    returns SEM_EINVAL with nothing launched."""
    import ctypes
    import torch
    from paper_1601_08179_gb300 import sem
    L = sem.lib()
    ctx, ms = make_pair(4, (2, 2, 2), 1.0)
    uB = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda")
    vB = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda")
    u32 = torch.zeros(ctx.nb, dtype=torch.float32, device="cuda")
    assert sem.sem_check_vector(ctx, uB.data_ptr(), 8) == sem.SEM_OK
    assert sem.sem_check_vector(ctx, u32.data_ptr(), 4) == sem.SEM_OK
    assert sem.sem_check_vector(ctx, uB.data_ptr() + 4, 4) == sem.SEM_OK   # a float at a 4-byte offset
    host_arr = np.zeros(ctx.nb)
    pinned = torch.zeros(ctx.nb, dtype=torch.float64).pin_memory()
    bad = {"host": host_arr.ctypes.data, "pinned": pinned.data_ptr(), "misaligned": uB.data_ptr() + 4, "null": 0}
    for name, ptr in bad.items():
        assert sem.sem_check_vector(ctx, ptr, 8) == sem.SEM_EINVAL, name
        assert L.sem_last_error().decode(), name
    assert sem.sem_check_vector(ctx, uB.data_ptr(), 3) == sem.SEM_EINVAL
    n0 = sem.sem_launch_count()
    for name, ptr in bad.items():
        P = ctypes.c_void_p(ptr)
        good = ctypes.c_void_p(vB.data_ptr())
        assert L.sem_apply_condensed(ctx.handle, P, good, sem.SPACE_TRANSFORMED, None) == sem.SEM_EINVAL, name
        assert L.sem_apply_condensed(ctx.handle, good, P, sem.SPACE_TRANSFORMED, None) == sem.SEM_EINVAL, name
        assert L.sem_pack_skeleton(ctx.handle, P, good, None) == sem.SEM_EINVAL, name
        assert L.sem_solve(ctx.handle, P, P, None, None, None) == sem.SEM_EINVAL, name
    assert sem.sem_launch_count() == n0
    # the checks pass the context's own vectors through: a normal call still works
    uB.copy_(torch.randn(ctx.nb, dtype=torch.float64, device="cuda"))
    sem.sem_apply_condensed(ctx, uB, vB)
    torch.cuda.synchronize()
    assert torch.isfinite(vB).all()


def test_entry_points_refuse_another_current_device():
    """An entry point that launches refuses to run while a device other than
    the context's is current (its kernels would launch there and read the
    context's tables across devices), with nothing launched.  Needs two
    visible GPUs; skipped otherwise."""
    import ctypes
    import torch
    from paper_1601_08179_gb300 import sem
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU visible")
    L = sem.lib()
    with torch.cuda.device(0):
        ctx, ms = make_pair(3, (2, 2, 2), 1.0)
        uB = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda:0")
        vB = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(1):
        n0 = sem.sem_launch_count()
        st = L.sem_apply_condensed(ctx.handle, ctypes.c_void_p(uB.data_ptr()), ctypes.c_void_p(vB.data_ptr()),
                                   sem.SPACE_TRANSFORMED, None)
        assert st == sem.SEM_EINVAL
        assert "current device" in L.sem_last_error().decode()
        assert sem.sem_launch_count() == n0
    with torch.cuda.device(0):
        sem.sem_apply_condensed(ctx, uB, vB)
        torch.cuda.synchronize()


def test_breakdown_on_nan_input():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(3, (2, 2, 2), 1.0)
    f = si.node_noise(ms.n_global, 11)
    f[ms.gid(3, 3, 3)] = np.nan
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u, check=False)
    assert info["status"] == sem.SEM_EBREAKDOWN


def test_maxit_reports_no_convergence():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(4, (4, 4, 4), 0.0, 8.0, opts=None)
    sem.sem_set_opts(ctx, sem.default_opts(maxit=3, check_every=2))
    f = si.node_noise(ms.n_global, 12)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u, check=False)
    assert info["status"] == sem.SEM_ENOCONV and info["iters"] == 3


FULL = [si.scale_workload(p) for p in si.SCALE_DEGREES]


@pytest.mark.parametrize("w", FULL, ids=[w.name for w in FULL])
def test_apply_full_size_vs_local_oracle(w):
    """Every output of one transformed-space application at the benchmark
    sizes (N ~ 1.68e7), against the element-local oracle in nodal space."""
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(w.p, w.m, w.lam, w.ar)
    uB = si.random_vector(ms.n_skeleton, 13)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(uB), v, sem.SPACE_NODAL)
    ref = local.apply_condensed(ms, w.lam, uB)
    assert relerr(host(v), ref) <= APPLY_TOL


def test_solve_full_size_residual():
    """p = 8 on 32^3 graded elements (AR 128, lambda = 0): the recovered field
    satisfies the uncondensed system to the solver tolerance (oracle A u)."""
    import torch
    from paper_1601_08179_gb300 import sem
    w = si.scale_workload(8)
    ctx, ms = make_pair(w.p, w.m, w.lam, w.ar)
    x, y, z = sem.sem_node_coords(ctx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = (si.manufactured_f(X, Y, Z, w.lam) + si.node_noise(X.size, w.seed).reshape(X.shape)).ravel()
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, dev(f), u)
    got = host(u)
    F = local.rhs_full(ms, f)
    r = (local.apply_full(ms, w.lam, got) - F)[ms.free_mask]
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(F[ms.free_mask])
    assert info["rel_res"] <= 1e-10


@pytest.mark.parametrize("p,m,lam,ar", [(2, (3, 2, 4), 0.5, 3.0), (3, (2, 3, 2), 2.5, 2.0), (4, (3, 2, 3), 1.0, 4.0),
                                        (6, (2, 3, 2), 0.0, 2.0), (7, (2, 2, 2), 3.0, 1.0), (8, (3, 2, 2), 1.0, 2.0),
                                        (12, (2, 2, 1), 1.0, 1.0), (16, (2, 1, 1), 2.0, 1.0)])
def test_apply_f32_vs_oracle(p, m, lam, ar):
    """The FP32 operator of the mixed-precision solver against the FP64
    oracle: FP32 rounding only (relative error well below 1e-5)."""
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, lam, ar)
    ut = si.random_vector(ms.n_skeleton, 91)
    free = ms.skeleton_free
    v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
    sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut.astype(np.float32).astype(np.float64), 0.0))
    ref = transform.load_to_transformed(ms, np.where(free, local.apply_condensed(ms, lam, u_nodal), 0.0))
    got = host(v)
    assert np.all(got[~free] == 0.0)
    assert relerr(got, ref) <= 1e-5
