"""Preconditioned conjugate gradients (Hestenes-Stiefel), as used in Sec. 8.

Plain textbook iteration with x0 given (default 0), a diagonal preconditioner
and the stopping rule ||r_k||_2 <= rtol ||r_0||_2.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def pcg(apply, b, pdiag=None, rtol=1e-10, maxit=100000, x0=None, callback=None):
    """Solve A x = b.  ``apply(v)`` returns A v; ``pdiag`` is the diagonal of
    the preconditioner P ~ A^-1 (None: unpreconditioned).

    Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply(x) if x0 is not None else b.copy()
    z = r * pdiag if pdiag is not None else r.copy()
    p = z.copy()
    rho = float(r @ z)
    r0 = float(np.linalg.norm(r))
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    it = 0
    while it < maxit:
        q = apply(p)
        pq = float(p @ q)
        if not pq > 0.0:
            raise FloatingPointError("breakdown: p^T A p <= 0")
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / r0
        hist.append(rel)
        if callback is not None:
            callback(it, rel)
        if rel <= rtol:
            break
        z = r * pdiag if pdiag is not None else r
        rho_new = float(r @ z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, hist
