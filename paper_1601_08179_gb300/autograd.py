"""Differentiable Helmholtz solve: a torch.autograd.Function around the C ABI.

u = solve(f; lambda, hx, hy, hz) is the recovered nodal solution of
lambda u - Laplace u = f (sem_solve).  The backward pass runs one adjoint
solve w = A^-1 (dJ/du) with the same condensed solver (no CG iterate is
stored: the adjoint is recomputed from scratch) and the gradient kernels of
sem_gradients for dJ/df, dJ/dlambda and dJ/dh.  All arithmetic runs in the
CUDA library; this module only marshals tensors.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from . import sem

_CACHE: "OrderedDict[tuple, sem.SemContext]" = OrderedDict()
_CACHE_SIZE = 4


def context_for(p, hx, hy, hz, lam, opts=None, device=None):
    """Library context for (p, widths, lambda) on a CUDA device (index or
    torch.device; default: the current one), cached (LRU of 4)."""
    hx = np.ascontiguousarray(np.asarray(hx, dtype=np.float64))
    hy = np.ascontiguousarray(np.asarray(hy, dtype=np.float64))
    hz = np.ascontiguousarray(np.asarray(hz, dtype=np.float64))
    d = None if device is None else (torch.device("cuda", device) if isinstance(device, int)
                                     else torch.device(device))
    dev = torch.cuda.current_device() if d is None or d.index is None else d.index
    key = (dev, int(p), hx.tobytes(), hy.tobytes(), hz.tobytes(), float(lam),
           None if opts is None else bytes(opts))
    ctx = _CACHE.pop(key, None)
    if ctx is None:
        with torch.cuda.device(dev):        # a context lives on the device current at setup
            ctx = sem.sem_setup(p, hx, hy, hz, float(lam), opts)
    _CACHE[key] = ctx
    while len(_CACHE) > _CACHE_SIZE:
        _CACHE.popitem(last=False)
    return ctx


class HelmholtzSolve(torch.autograd.Function):
    """u = HelmholtzSolve.apply(f, lam, hx, hy, hz, p, opts).

    f: CUDA float64 full nodal field (x fastest); lam: 0-d float64 tensor
    (its gradient is returned on its device) or a number (no gradient);
    hx, hy, hz: 1-D float64 tensors of element widths; p: degree; opts:
    sem.sem_opts or None.  Gradients flow to f, lam, hx, hy, hz."""

    @staticmethod
    def forward(ctx, f, lam, hx, hy, hz, p, opts=None):
        sctx = context_for(p, hx.detach().cpu().numpy(), hy.detach().cpu().numpy(),
                           hz.detach().cpu().numpy(), float(lam), opts, device=f.device)
        f = f.detach().contiguous()
        u = torch.empty_like(f)
        with torch.cuda.device(f.device):   # the library runs on the context's (f's) device
            sem.sem_solve(sctx, f, u)
        ctx.sctx = sctx
        # lambda may be a tensor (on any device) or a plain number (no gradient)
        ctx.lam_device = lam.device if torch.is_tensor(lam) else None
        ctx.save_for_backward(f, u, hx, hy, hz)
        return u

    @staticmethod
    def backward(ctx, gu):
        f, u, hx, hy, hz = ctx.saved_tensors
        sctx = ctx.sctx
        w = torch.empty_like(u)
        df = torch.empty_like(u)
        with torch.cuda.device(u.device):
            sem.sem_solve_adjoint(sctx, gu.detach().contiguous(), w)
            dl, dhx, dhy, dhz = sem.sem_gradients(sctx, w, u, f, df)
        as_t = lambda a, like: torch.as_tensor(a, dtype=torch.float64, device=like.device)
        dlam = None if ctx.lam_device is None else torch.tensor(dl, dtype=torch.float64, device=ctx.lam_device)
        return (df, dlam, as_t(dhx, hx), as_t(dhy, hy), as_t(dhz, hz), None, None)


def helmholtz_solve(f, lam, hx, hy, hz, p, opts=None):
    return HelmholtzSolve.apply(f, lam, hx, hy, hz, p, opts)
