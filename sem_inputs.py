"""Seeded synthetic inputs for the condensed spectral-element Helmholtz solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds none of the method's arithmetic: no quadrature, no basis, no operator.
It only produces

* element widths of Cartesian meshes on the unit cube, uniform or
  geometrically graded to a target maximum aspect ratio;
* the manufactured solution u = sin(pi x) sin(pi y) sin(pi z) and its
  right-hand side f = (3 pi^2 + lambda) u, as plain functions of coordinates;
* seeded uniform noise (NumPy PCG64) to add to nodal right-hand sides;
* the named workloads (degree, mesh, lambda, aspect ratio, seed).

The paper grades its meshes by a constant expansion factor alpha and quotes
the resulting maximum aspect ratios 1, ~17 and 128 for an 8^3 mesh (Sec. 8).
Here the default grading is along x only: h_x,i = L r^i / sum_j r^j with
h_y = h_z = L/m, and r >= 1 chosen by bisection so that the largest element
aspect ratio max(h)/min(h) hits the target.  ``grade="xy"`` gives the paper's
own variant, where x and y widths grow by r = AR^(1/(m-1)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1601


def _geometric(m: int, r: float, L: float) -> np.ndarray:
    w = r ** np.arange(m, dtype=np.float64)
    return L * w / w.sum()


def max_aspect_ratio(hx, hy, hz) -> float:
    """Largest max(h)/min(h) over the elements of the tensor mesh hx x hy x hz."""
    hx = np.asarray(hx, float)
    hy = np.asarray(hy, float)
    hz = np.asarray(hz, float)
    # the extreme ratio is reached at an extreme width of each axis
    best = 1.0
    for a in (hx.min(), hx.max()):
        for b in (hy.min(), hy.max()):
            for c in (hz.min(), hz.max()):
                best = max(best, max(a, b, c) / min(a, b, c))
    return float(best)


def graded_widths(mx: int, my: int, mz: int, ar: float = 1.0, L: float = 1.0,
                  grade: str = "x"):
    """Element widths (hx, hy, hz) on [0, L]^3 with maximum aspect ratio ``ar``.

    grade="x": only x is graded, r found by bisection (monotone in r >= 1).
    grade="xy": x and y widths both scale by r = ar^(1/(m-1)) (paper's meshes).
    Returns (hx, hy, hz, r).
    """
    if ar < 1.0:
        raise ValueError("aspect ratio must be >= 1")
    hy = np.full(my, L / my)
    hz = np.full(mz, L / mz)
    if ar == 1.0 or (grade == "x" and mx == 1):
        if mx == 1 and ar != 1.0 and grade == "x":
            raise ValueError("cannot grade a single element")
        return np.full(mx, L / mx), hy, hz, 1.0
    if grade == "xy":
        r = ar ** (1.0 / max(mx - 1, 1))
        return _geometric(mx, r, L), _geometric(my, r, L), hz, r
    if grade != "x":
        raise ValueError("grade must be 'x' or 'xy'")
    lo, hi = 1.0, 2.0
    while max_aspect_ratio(_geometric(mx, hi, L), hy, hz) < ar:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if max_aspect_ratio(_geometric(mx, mid, L), hy, hz) < ar:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    return _geometric(mx, r, L), hy, hz, r


def manufactured_u(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def manufactured_f(x, y, z, lam: float):
    """Right-hand side of lambda u - Laplace u = f for the manufactured u."""
    return (3.0 * np.pi ** 2 + lam) * manufactured_u(x, y, z)


def node_noise(num: int, seed: int) -> np.ndarray:
    """U[-1, 1] i.i.d. values, one per global node, from PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, size=num)


def random_vector(num: int, seed: int) -> np.ndarray:
    """Standard-normal test vector (operator inputs), from PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(num)


@dataclass(frozen=True)
class Workload:
    name: str
    p: int
    m: tuple
    lam: float
    ar: float = 1.0
    noise: bool = False
    seed: int = SEED_BASE
    grade: str = "x"
    rtol: float = 1e-10

    def widths(self):
        hx, hy, hz, _ = graded_widths(*self.m, ar=self.ar, grade=self.grade)
        return hx, hy, hz

    @property
    def n_elements(self) -> int:
        return self.m[0] * self.m[1] * self.m[2]

    @property
    def dofs(self) -> int:
        """N = n_e p^3, the paper's count of unknowns."""
        return self.n_elements * self.p ** 3

    @property
    def grid_shape(self):
        """(Nz, Ny, Nx) of the global nodal grid, x fastest in memory."""
        mx, my, mz = self.m
        return (mz * self.p + 1, my * self.p + 1, mx * self.p + 1)


# Small correctness workload: 4^3 uniform elements, p = 4, lambda = 1,
# manufactured right-hand side, FP64, relative residual 1e-10.
SMALL = Workload("uniform_p4_m4_lam1", p=4, m=(4, 4, 4), lam=1.0, seed=SEED_BASE + 0)


def scale_workload(p: int, ar: float = 128.0, lam: float = 0.0) -> Workload:
    """Degree sweep at N ~ 1.68e7: m p = 256, x-graded to aspect ratio ``ar``,
    manufactured right-hand side plus U[-1,1] nodal noise."""
    m = {2: 128, 4: 64, 8: 32, 16: 16, 32: 8}[p]
    return Workload(f"graded_p{p}_m{m}_ar{int(ar)}_lam{lam:g}", p=p, m=(m, m, m),
                    lam=lam, ar=ar, noise=True, seed=SEED_BASE + 1)


SCALE_DEGREES = (2, 4, 8, 16, 32)

# Mixed-precision workload: p = 16 on 16^3 elements, lambda = 10, aspect ratio 16.
MIXED = Workload("graded_p16_m16_ar16_lam10", p=16, m=(16, 16, 16), lam=10.0,
                 ar=16.0, noise=True, seed=SEED_BASE + 2)


def batched_problems(count: int = 64, seed: int = SEED_BASE + 3):
    """Heterogeneous batch: m in {4,8,12,16,24}, p in {4,6,8,12,16},
    lambda log-uniform in [1e-2, 1e4], aspect ratio U[1, 64]."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        m = int(g.choice([4, 8, 12, 16, 24]))
        p = int(g.choice([4, 6, 8, 12, 16]))
        lam = float(10.0 ** g.uniform(-2.0, 4.0))
        ar = float(g.uniform(1.0, 64.0))
        out.append(Workload(f"batch{b}_p{p}_m{m}", p=p, m=(m, m, m), lam=lam, ar=ar,
                            noise=True, seed=SEED_BASE * 100 + b))
    return out


def smooth_target(x, y, z, seed: int, terms: int = 8):
    """Seeded smooth field: a sum of `terms` products of low-wavenumber sines
    with random amplitudes and phases (the target of the differentiable solve)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros(np.broadcast(x, y, z).shape)
    for _ in range(terms):
        a = g.uniform(-1.0, 1.0)
        k = g.integers(1, 4, size=3)
        ph = g.uniform(0.0, 2.0 * np.pi, size=3)
        out += a * np.sin(k[0] * np.pi * x + ph[0]) * np.sin(k[1] * np.pi * y + ph[1]) * np.sin(k[2] * np.pi * z + ph[2])
    return out


# Differentiable-solve workload: p = 8 on 16^3 elements, lambda = 1, FP64,
# J = 1/2 ||u - u_target||^2 with a smooth seeded target.
ADJOINT = Workload("uniform_p8_m16_lam1_adjoint", p=8, m=(16, 16, 16), lam=1.0, seed=SEED_BASE + 4)
