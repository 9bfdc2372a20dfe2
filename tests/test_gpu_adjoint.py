"""Differentiable solve (torch.autograd.Function around the C ABI) against the
oracle's dense adjoint gradient and against central finite differences of the
GPU solve itself, for J = 1/2 ||u - u_t||^2."""
import numpy as np
import pytest

import sem_inputs as si
from oracle.adjoint import solve_and_gradient
from oracle.mesh import Mesh

pytestmark = pytest.mark.gpu


def _grad_gpu(p, hx, hy, hz, lam, f, ut, opts):
    import torch
    from paper_1601_08179_gb300.autograd import helmholtz_solve
    fd = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
    lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    hxt = torch.tensor(hx, dtype=torch.float64, requires_grad=True)
    hyt = torch.tensor(hy, dtype=torch.float64, requires_grad=True)
    hzt = torch.tensor(hz, dtype=torch.float64, requires_grad=True)
    u = helmholtz_solve(fd, lt, hxt, hyt, hzt, p, opts)
    J = 0.5 * ((u - torch.tensor(ut, device="cuda")) ** 2).sum()
    J.backward()
    return (float(J), fd.grad.cpu().numpy(), float(lt.grad), hxt.grad.numpy(), hyt.grad.numpy(),
            hzt.grad.numpy())


@pytest.mark.parametrize("p,m,lam,ar", [(4, (3, 2, 2), 1.0, 3.0), (3, (2, 3, 2), 0.0, 1.0)])
def test_gradient_vs_oracle(p, m, lam, ar):
    from paper_1601_08179_gb300 import sem
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar)
    ms = Mesh(p, hx, hy, hz)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 51).reshape(X.shape)).ravel()
    ut = si.smooth_target(X, Y, Z, 52).ravel()
    J0, u0, df0, dl0, dh0 = solve_and_gradient(ms, lam, f, ut)
    J, df, dl, dhx, dhy, dhz = _grad_gpu(p, hx, hy, hz, lam, f, ut, sem.default_opts(rtol=1e-13))
    assert J == pytest.approx(J0, rel=1e-9)
    assert np.linalg.norm(df - df0) <= 1e-6 * np.linalg.norm(df0)
    assert dl == pytest.approx(dl0, rel=1e-6, abs=1e-12)
    for got, want in zip((dhx, dhy, dhz), dh0):
        np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


def test_gradient_vs_finite_differences_full_size():
    """p = 8 on 16^3 elements, lambda = 1: directional derivatives in f, lambda
    and one width of each axis against central differences of the GPU
    objective.  J is exactly quadratic in f, so the f-step (1e-2) adds no
    truncation error while keeping the solution change far above the 1e-13
    solve tolerance; lambda and h use relative steps of 1e-4 (truncation
    O(1e-8)).  The 1e-6-step check of the same formulas is the oracle pin in
    tests/test_oracle_adjoint.py."""
    import torch
    from paper_1601_08179_gb300 import sem
    from paper_1601_08179_gb300.autograd import context_for
    w = si.ADJOINT
    hx, hy, hz = w.widths()
    opts = sem.default_opts(rtol=1e-13)
    ctx = context_for(w.p, hx, hy, hz, w.lam, opts)
    x, y, z = sem.sem_node_coords(ctx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = si.manufactured_f(X, Y, Z, w.lam).ravel()
    ut = si.smooth_target(X, Y, Z, w.seed).ravel()
    J, df, dl, dhx, dhy, dhz = _grad_gpu(w.p, hx, hy, hz, w.lam, f, ut, opts)
    utd = torch.tensor(ut, device="cuda")

    def sol(ff, lam, hx_, hy_, hz_):
        c = context_for(w.p, hx_, hy_, hz_, lam, opts)
        fd = torch.tensor(ff, device="cuda")
        u = torch.empty_like(fd)
        sem.sem_solve(c, fd, u)
        return u

    def dJ(a, b):
        # J(a) - J(b) = 1/2 sum (u_a - u_b)(u_a + u_b - 2 u_t), without the
        # cancellation of two O(1e6) objectives
        return 0.5 * float(((a - b) * (a + b - 2.0 * utd)).sum())

    eps = 1e-2
    d = si.random_vector(f.size, 53)
    fdv = dJ(sol(f + eps * d, w.lam, hx, hy, hz), sol(f - eps * d, w.lam, hx, hy, hz)) / (2 * eps)
    assert float(df @ d) == pytest.approx(fdv, rel=1e-6)
    eps = 1e-4 * w.lam
    fdv = dJ(sol(f, w.lam + eps, hx, hy, hz), sol(f, w.lam - eps, hx, hy, hz)) / (2 * eps)
    assert dl == pytest.approx(fdv, rel=1e-6)
    for axis, (arr, g) in enumerate(((hx, dhx), (hy, dhy), (hz, dhz))):
        i = 5
        eps = 1e-4 * arr[i]
        hp = [hx.copy(), hy.copy(), hz.copy()]
        hm = [hx.copy(), hy.copy(), hz.copy()]
        hp[axis][i] += eps
        hm[axis][i] -= eps
        fdv = dJ(sol(f, w.lam, *hp), sol(f, w.lam, *hm)) / (2 * eps)
        assert g[i] == pytest.approx(fdv, rel=1e-6), axis


def test_lambda_as_number_and_as_cuda_tensor():
    """lambda passed as a plain number gets no gradient (None) and leaves the
    other gradients unchanged; passed as a CUDA 0-d tensor its gradient lands
    on that device and equals the one returned for a CPU tensor."""
    import torch
    from paper_1601_08179_gb300 import sem
    from paper_1601_08179_gb300.autograd import helmholtz_solve
    p, m, lam = 3, (2, 2, 3), 2.0
    hx, hy, hz, _ = si.graded_widths(*m, ar=2.0)
    ms = Mesh(p, hx, hy, hz)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 54).reshape(X.shape)).ravel()
    ut = torch.tensor(si.smooth_target(X, Y, Z, 55).ravel(), device="cuda")
    opts = sem.default_opts(rtol=1e-13)

    def run(lam_arg):
        fd = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
        hs = [torch.tensor(h, dtype=torch.float64, requires_grad=True) for h in (hx, hy, hz)]
        u = helmholtz_solve(fd, lam_arg, *hs, p, opts)
        (0.5 * ((u - ut) ** 2).sum()).backward()
        return fd.grad.cpu().numpy(), [h.grad.numpy() for h in hs]

    l_cpu = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    df_cpu, dh_cpu = run(l_cpu)
    l_cuda = torch.tensor(lam, dtype=torch.float64, device="cuda", requires_grad=True)
    df_cuda, dh_cuda = run(l_cuda)
    assert l_cuda.grad is not None and l_cuda.grad.is_cuda
    # the runs repeat the same solves; atomics in arrival order make them equal
    # to rounding, so they are compared at the solve bar
    assert float(l_cuda.grad) == pytest.approx(float(l_cpu.grad), rel=1e-9)
    df_num, dh_num = run(lam)
    for got in (df_cuda, df_num):
        assert np.linalg.norm(got - df_cpu) <= 1e-9 * np.linalg.norm(df_cpu)
    for dh in (dh_cuda, dh_num):
        for got, want in zip(dh, dh_cpu):
            np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
