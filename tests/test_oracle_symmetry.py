"""A property of the 1D basis that the FP32 operator kernels use: the GLL
points and the interior generalised eigenproblem of (K_II, M_II) are
symmetric under x -> -x, so eigenvector c is even or odd with c (the
eigenvalues ascending, the first component positive), and the transformed
border vectors satisfy K~_{Ip}[c] = (-1)^c K~_{I0}[c].  Checked on the
oracle's own basis for every degree.  In floating point the two sides of the
relation differ by rounding that grows with the degree (3e-14 of the
largest entry at p = 8, 6e-13 at p = 16, 1e-11 at p = 32): far below FP32
resolution, where the FP32 kernels use it, but not below the 1e-12 bar of
the FP64 operator, which keeps both vectors."""
import numpy as np
import pytest

from oracle import transform
from oracle.gll import mass_stiffness


@pytest.mark.parametrize("p", list(range(2, 33)))
def test_border_vectors_are_even_and_odd(p):
    _, V = transform.eigenbasis(p)
    _, K = mass_stiffness(p)
    k0, k1 = V.T @ K[1:p, 0], V.T @ K[1:p, p]
    sign = (-1.0) ** np.arange(p - 1)
    np.testing.assert_allclose(k1, sign * k0, rtol=0, atol=3e-11 * np.abs(k0).max())
    if p <= 9:   # the degrees of the FP32 plane kernel that uses the relation
        np.testing.assert_allclose(k1, sign * k0, rtol=0, atol=1e-13 * np.abs(k0).max())
    # and each eigenvector is even or odd under reversal of the interior nodes
    np.testing.assert_allclose(V[::-1, :], V * sign[None, :], rtol=0, atol=1e-9 * np.abs(V).max())
