"""sem_condense_rhs_noalloc: the condensed load for callers that cannot
allocate device memory during the call (an application whose own pool holds
the device memory, or a loop that must not take the device-wide
synchronisation of cudaFree / cudaMalloc).

It must give the same result as the allocating entry point sem_condense_rhs,
on consecutive calls that reuse the library's fixed scratch array, and must
reject meshes larger than that array with an error.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import sem_inputs as si
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the operator-level tolerance of the parity tests


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(4, (4, 3, 5), 1.0, 2.0)
    fs = [dev(si.node_noise(ms.n_global, seed)) for seed in (31, 32)]
    for space in (sem.SPACE_TRANSFORMED, sem.SPACE_NODAL):
        outs = []
        for f in fs:       # two calls in a row through the C ABI
            o = torch.full((ctx.nb,), np.nan, dtype=torch.float64, device="cuda")
            sem.sem_condense_rhs_noalloc(ctx, f, o, space)
            outs.append(o)
        for f, o in zip(fs, outs):
            ref = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
            sem.sem_condense_rhs(ctx, f, ref, space)
            got, want = host(o), host(ref)
            assert np.all(np.isfinite(got))
            assert relerr(got, want) <= TOL


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(8, (12, 12, 12), 1.0)      # 1728 * 7^3 > 2^19
    f = torch.zeros(ctx.n_nodes, dtype=torch.float64, device="cuda")
    out = torch.zeros(ctx.nb, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as err:
        sem.sem_condense_rhs_noalloc(ctx, f, out)
    assert err.value.status == sem.SEM_EINVAL
    assert "too large" in str(err.value)
