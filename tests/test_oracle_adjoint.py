"""Pins for the oracle's adjoint gradient (oracle/adjoint.py): central finite
differences of the oracle objective J = 1/2 ||u - u_t||^2, with every solve a
sparse direct solve (exact to rounding), in f, lambda and every element width."""
import numpy as np
import pytest

import sem_inputs as si
from oracle.adjoint import objective, solve_and_gradient
from oracle.mesh import Mesh


@pytest.mark.parametrize("p,m,lam,ar", [(3, (3, 2, 2), 1.5, 3.0), (4, (2, 2, 3), 0.0, 1.0)])
def test_oracle_gradient_matches_finite_differences(p, m, lam, ar):
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar)
    ms = Mesh(p, hx, hy, hz)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, lam) + si.node_noise(X.size, 41).reshape(X.shape)).ravel()
    ut = si.smooth_target(X, Y, Z, 42).ravel()
    J, u, df, dlam, dh = solve_and_gradient(ms, lam, f, ut)
    eps = 1e-6
    d = si.random_vector(f.size, 43)
    fd = (objective(ms, lam, f + eps * d, ut) - objective(ms, lam, f - eps * d, ut)) / (2 * eps)
    assert float(df @ d) == pytest.approx(fd, rel=1e-6)
    fd = (objective(ms, lam + eps, f, ut) - objective(ms, lam - eps, f, ut)) / (2 * eps)
    assert dlam == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(J))
    for axis, arr in enumerate((hx, hy, hz)):
        for i in range(len(arr)):
            hp = [np.array(hx), np.array(hy), np.array(hz)]
            hm = [np.array(hx), np.array(hy), np.array(hz)]
            hp[axis][i] += eps
            hm[axis][i] -= eps
            # f is held fixed at its nodal values
            fd = (objective(Mesh(p, *hp), lam, f, ut) - objective(Mesh(p, *hm), lam, f, ut)) / (2 * eps)
            assert dh[axis][i] == pytest.approx(fd, rel=1e-5, abs=1e-8 * abs(J)), (axis, i)
