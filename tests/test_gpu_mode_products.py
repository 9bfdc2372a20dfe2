"""The O(n^4) mode products of load condensation and recovery (S (x) S (x) S
on every interior cube, Algorithm 4), computed in double-float arithmetic on
the FP32 pipe, against the element-local FP64 oracle.

Covered: degrees up to 32 (contraction length 31), loads scaled over 60
orders of magnitude (the double-float parts must stay normal floats, else
the split falls back to the FP64 conversion), loads with exact zeros and
with entries below 2^-74 next to entries of order 1, and the recovery that
writes the interior of the nodal field.  Bar: 1e-12 relative (2-norm), the
FP64 operator's bar.
"""
import numpy as np
import pytest

import sem_inputs as si
from oracle import local
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _condense(ctx, f):
    import torch
    from paper_1601_08179_gb300 import sem
    out = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_condense_rhs(ctx, dev(f), out, sem.SPACE_NODAL)
    return host(out)


@pytest.mark.parametrize("p,m", [(32, (2, 1, 1)), (17, (2, 2, 1)), (9, (3, 2, 2))])
@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e30])
def test_condensed_load_high_degree_and_scale(p, m, scale):
    ctx, ms = make_pair(p, m, 2.0, 6.0)
    f = scale * si.node_noise(ms.n_global, 900 + p)
    ref = local.condensed_rhs(ms, 2.0, f)
    got = _condense(ctx, f)
    err = relerr(got, ref)
    print(f"p={p} scale={scale:.0e}: {err:.2e}")
    assert err <= TOL


def test_condensed_load_with_zeros_and_tiny_entries():
    """Half the nodes zero, a quarter at 1e-25 (below 2^-74: the FP64
    conversion path of the split), the rest of order 1."""
    p, m = 16, (2, 2, 1)
    ctx, ms = make_pair(p, m, 0.5, 4.0)
    f = si.node_noise(ms.n_global, 950)
    idx = np.arange(ms.n_global)
    f[idx % 2 == 0] = 0.0
    f[idx % 4 == 1] *= 1e-25
    ref = local.condensed_rhs(ms, 0.5, f)
    assert relerr(_condense(ctx, f), ref) <= TOL
    # and the tiny entries alone, where they carry the whole result
    g = np.where(idx % 4 == 1, f, 0.0)
    ref = local.condensed_rhs(ms, 0.5, g)
    assert relerr(_condense(ctx, g), ref) <= TOL


@pytest.mark.parametrize("p,m", [(32, (2, 1, 1)), (12, (2, 2, 2))])
def test_recovery_high_degree(p, m):
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(p, m, 1.0, 8.0)
    f = si.node_noise(ms.n_global, 960 + p)
    uB = si.random_vector(ms.n_skeleton, 961 + p)
    ref = local.recover_interior(ms, 1.0, f, np.where(ms.skeleton_free, uB, 0.0))
    u = torch.full((ctx.n_nodes,), 3.0, dtype=torch.float64, device="cuda")
    sem.sem_recover_interior(ctx, dev(f), dev(uB), u, sem.SPACE_NODAL)
    err = relerr(host(u), ref)
    print(f"recovery p={p}: {err:.2e}")
    assert err <= TOL
