"""Helpers shared by the GPU parity tests: build one library context and the
matching oracle mesh from the same seeded inputs."""
import numpy as np

import sem_inputs as si
from oracle.mesh import Mesh


def make_pair(p, m, lam, ar=1.0, grade="x", opts=None):
    import torch
    from paper_1601_08179_gb300 import build, sem
    build.build()
    hx, hy, hz, _ = si.graded_widths(*m, ar=ar, grade=grade)
    ctx = sem.sem_setup(p, hx, hy, hz, lam, opts)
    ms = Mesh(p, hx, hy, hz)
    assert ctx.nb == ms.n_skeleton and ctx.n_nodes == ms.n_global
    return ctx, ms


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
