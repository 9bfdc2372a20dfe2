"""The debug build (SEM_DEBUG): every kernel checks the skeleton entity
offsets and class indices it forms before any access.  Over the operator
kernels of both precisions, load condensation, preconditioner, solves
(FP64, mixed, batched) and recovery on regular and thin meshes, the record
stays empty and the results meet the same bars as the release build; with the
checked bound lowered below the vertex block, the offsets past it are caught
(and skipped) while every access stays inside the real vectors.  The
one-pass CG step's grid barrier, made never to complete, gives up after its
bounded wait and stops the CG, and the context solves normally afterwards.
The work runs in a child process that loads the debug library (SEM_LIB)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import sem_inputs as si
from oracle import dense, local, transform
from paper_1601_08179_gb300 import sem
from tests.gpu_util import dev, host, make_pair, relerr

def oracle_apply(ms, lam, ut):
    free = ms.skeleton_free
    u = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    return transform.load_to_transformed(ms, np.where(free, local.apply_condensed(ms, lam, u), 0.0))

out = {"applies": [], "solves": []}
K = {"AUTO": sem.KERNEL_AUTO, "WARP": sem.KERNEL_WARP, "PLANE": sem.KERNEL_PLANE,
     "ELEMENT": sem.KERNEL_ELEMENT, "SLAB": sem.KERNEL_SLAB, "ROW": sem.KERNEL_ROW, "PENCIL": sem.KERNEL_PENCIL}
# FP64: the built-in kernel (thread per element at p = 2, CTA tile above)
cases = [(2, (3, 2, 2), ["AUTO"], ["ELEMENT"]), (3, (1, 3, 2), ["AUTO"], ["ELEMENT", "PLANE", "ROW"]),
         (4, (3, 2, 2), ["AUTO"], ["PLANE", "ELEMENT", "WARP", "ROW"]),
         (8, (2, 2, 3), ["AUTO"], ["PLANE", "WARP", "ROW", "PENCIL"]),
         (12, (2, 1, 2), ["AUTO"], ["PLANE"]), (20, (2, 2, 1), ["AUTO"], ["SLAB"])]
for p, m, k64, k32 in cases:
    ar = 1.0 if m[0] == 1 else 4.0
    ctx, ms = make_pair(p, m, 1.0, ar)
    ut = si.random_vector(ms.n_skeleton, 70 + p)
    ref = oracle_apply(ms, 1.0, ut)
    for k in k64:
        sem.sem_set_operator_kernel(ctx, sem.PREC_FP64, K[k])
        v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
        sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
        out["applies"].append(["f64", k, p, relerr(host(v), ref)])
    u32 = ut.astype(np.float32).astype(np.float64)
    ref32 = oracle_apply(ms, 1.0, u32)
    for k in k32:
        sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, K[k])
        v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
        sem.sem_apply_condensed_f32(ctx, torch.tensor(u32, dtype=torch.float32, device="cuda"), v)
        out["applies"].append(["f32", k, p, relerr(host(v), ref32)])
for p, m, prec in [(4, (2, 2, 3), sem.PREC_FP64), (8, (2, 2, 2), sem.PREC_MIXED), (3, (1, 2, 2), sem.PREC_MIXED)]:
    ctx, ms = make_pair(p, m, 2.0, 1.0, opts=sem.default_opts(precision=prec))
    f = si.node_noise(ms.n_global, 5)
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    sem.sem_solve(ctx, dev(f), u)
    out["solves"].append([p, prec, relerr(host(u), dense.solve_full(ms, 2.0, f))])
ctxs, fs, us, refs = [], [], [], []
for p, m in [(4, (2, 2, 2)), (6, (2, 1, 2))]:
    ctx, ms = make_pair(p, m, 1.0, 2.0)
    f = si.node_noise(ms.n_global, 9)
    ctxs.append(ctx); fs.append(dev(f)); us.append(torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda"))
    refs.append(dense.solve_full(ms, 1.0, f))
sem.SemBatch(ctxs, fs, us).solve()
out["batch"] = [relerr(host(u), r) for u, r in zip(us, refs)]
st, n, first = sem.sem_debug_oob()
out["clean"] = [st, n, first]

# lower the checked bound to the start of the vertex block: the free vertices
# of a 2 x 2 x 2 mesh (one) are caught in every operator kernel and skipped
ctx, ms = make_pair(4, (2, 2, 2), 1.0)
bound = ctx.nb - 27
ut = si.random_vector(ms.n_skeleton, 3)
caught = []
for prec, kind in [(sem.PREC_FP64, sem.KERNEL_AUTO), (sem.PREC_MIXED, sem.KERNEL_PLANE),
                   (sem.PREC_MIXED, sem.KERNEL_ELEMENT), (sem.PREC_MIXED, sem.KERNEL_WARP),
                   (sem.PREC_MIXED, sem.KERNEL_ROW)]:
    assert sem.sem_debug_limit_skeleton(ctx, bound) == sem.SEM_OK
    sem.sem_set_operator_kernel(ctx, prec, kind)
    if prec == sem.PREC_FP64:
        v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
        sem.sem_apply_condensed(ctx, dev(ut), v, sem.SPACE_TRANSFORMED)
    else:
        v = torch.empty(ctx.nb, dtype=torch.float32, device="cuda")
        sem.sem_apply_condensed_f32(ctx, torch.tensor(ut, dtype=torch.float32, device="cuda"), v)
    st, n, first = sem.sem_debug_oob()
    finite = bool(torch.isfinite(v).all())
    assert sem.sem_debug_limit_skeleton(ctx, ctx.nb) == sem.SEM_OK
    caught.append([prec, kind, st, n, first, finite])
out["caught"] = caught
out["bound"] = bound
out["limit_out_of_range"] = sem.sem_debug_limit_skeleton(ctx, ctx.nb + 1)
st, n, first = sem.sem_debug_oob()
out["after"] = [st, n, first]

# the one-pass CG step's grid barrier with its arrival count preset so that
# it never completes: every CTA's bounded wait runs out, the CG stops as a
# breakdown, and the context solves normally afterwards
ctx, ms = make_pair(6, (3, 2, 2), 1.0, 2.0, opts=sem.default_opts(precision=sem.PREC_MIXED))
f = si.node_noise(ms.n_global, 11)
u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
sem.sem_solve(ctx, dev(f), u)
st, bar_fail, done = sem.sem_debug_cg_step_timeout(ctx)
info = sem.sem_solve(ctx, dev(f), u)
out["barrier"] = [st, bar_fail, done, info["rel_res"], relerr(host(u), dense.solve_full(ms, 1.0, f))]
print("RESULT " + json.dumps(out))
"""


def test_debug_build_bounds_record():
    from paper_1601_08179_gb300 import build, sem
    lib = build.build(debug=True)
    env = dict(os.environ, SEM_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT), 1)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    for prec, kind, p, err in out["applies"]:
        print(prec, kind, p, f"{err:.2e}")
        assert err <= (1e-12 if prec == "f64" else 1e-5), (prec, kind, p, err)
    for p, prec, err in out["solves"]:
        assert err <= 1e-9, (p, prec, err)
    assert max(out["batch"]) <= 1e-9
    assert out["clean"] == [sem.SEM_OK, 0, -1]
    for prec, kind, st, n, first, finite in out["caught"]:
        assert st == sem.SEM_OK and n >= 1 and first >= out["bound"] and finite, (prec, kind, st, n, first)
    assert out["limit_out_of_range"] == sem.SEM_EINVAL
    assert out["after"] == [sem.SEM_OK, 0, -1]
    st, bar_fail, done, rel_res, err = out["barrier"]
    assert st == sem.SEM_OK and bar_fail == 1 and done == 2, out["barrier"]
    assert rel_res <= 1e-10 and err <= 1e-9, out["barrier"]
