"""Batched solves (one captured CUDA graph with a device-side while loop over
many independent problems) and the operator autotuner, against the dense
oracle and against one-at-a-time solves."""
import numpy as np
import pytest

import sem_inputs as si
from oracle import dense, local
from oracle.mesh import Mesh
from tests.gpu_util import dev, host, make_pair, relerr

pytestmark = pytest.mark.gpu


def _small_batch(count=12, seed=71):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        p = int(g.choice([2, 3, 4, 6, 8]))
        m = tuple(int(v) for v in g.integers(1, 4, size=3))
        lam = float(10.0 ** g.uniform(-2.0, 4.0))
        ar = float(g.uniform(1.0, 8.0)) if m[0] > 1 else 1.0
        out.append((p, m, lam, ar, seed * 100 + b))
    return out


def test_batch_matches_oracle_and_single_solves():
    import torch
    from paper_1601_08179_gb300 import sem
    probs = _small_batch()
    ctxs, meshes, fs, us, refs = [], [], [], [], []
    for p, m, lam, ar, seed in probs:
        ctx, ms = make_pair(p, m, lam, ar)
        f = si.node_noise(ms.n_global, seed)
        ctxs.append(ctx)
        meshes.append(ms)
        fs.append(dev(f))
        us.append(torch.full((ctx.n_nodes,), np.nan, dtype=torch.float64, device="cuda"))
        refs.append(dense.solve_full(ms, lam, f))
    batch = sem.SemBatch(ctxs, fs, us)
    for rep in range(2):                      # the same graph, launched twice
        st, infos = batch.solve()
        for k, (u, ref) in enumerate(zip(us, refs)):
            assert relerr(host(u), ref) <= 1e-9, k
    # FP64 solves sum every shared skeleton entry in a fixed order (faces onto
    # zero, edges and vertices through per-element shares, the condensed load
    # per face): a batched solve gives the single solve's bits
    for k, (ctx, f) in enumerate(zip(ctxs, fs)):
        u1 = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
        info = sem.sem_solve(ctx, f, u1)
        assert info["iters"] == infos[k]["iters"], k
        assert info["rel_res"] == infos[k]["rel_res"], k
        assert np.array_equal(host(us[k]), host(u1)), k


def test_batched_workload_heterogeneous_64():
    """64 problems: m in {4,8,12,16,24}^3, p in {4,6,8,12,16}, lambda
    log-uniform in [1e-2, 1e4], aspect ratio U[1, 64], seeded uniform loads:
    every solution meets the oracle's uncondensed residual (checked on the
    smaller problems) and equals its one-at-a-time solve."""
    import torch
    from paper_1601_08179_gb300 import sem
    work = si.batched_problems()
    ctxs, fs, us = [], [], []
    for w in work:
        hx, hy, hz = w.widths()
        c = sem.sem_setup(w.p, hx, hy, hz, w.lam)
        ctxs.append(c)
        fs.append(dev(si.node_noise(c.n_nodes, w.seed)))
        us.append(torch.empty(c.n_nodes, dtype=torch.float64, device="cuda"))
    batch = sem.SemBatch(ctxs, fs, us)
    st, infos = batch.solve()
    assert all(i["rel_res"] <= 1e-10 for i in infos)
    order = sorted(range(len(work)), key=lambda k: work[k].dofs)
    for k in order[:3]:
        w = work[k]
        ms = Mesh(w.p, *w.widths())
        f = host(fs[k])
        F = local.rhs_full(ms, f)
        r = (local.apply_full(ms, w.lam, host(us[k])) - F)[ms.free_mask]
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(F[ms.free_mask]), k
    for k in order[::8]:
        u1 = torch.empty_like(us[k])
        info = sem.sem_solve(ctxs[k], fs[k], u1)
        assert info["iters"] == infos[k]["iters"], k
        assert np.array_equal(host(us[k]), host(u1)), k


@pytest.mark.parametrize("p,m,lam,ar", [(2, (5, 4, 3), 1.0, 4.0), (4, (4, 3, 5), 0.0, 16.0), (8, (3, 4, 2), 100.0, 2.0),
                                        (6, (1, 3, 4), 3.0, 1.0), (16, (2, 2, 3), 0.5, 8.0), (12, (3, 1, 2), 1.0, 1.0)])
def test_fixed_order_operator_is_reproducible_and_matches_atomics(p, m, lam, ar):
    """The FP64 operator with fixed-order edge and vertex sums (the default)
    gives the same bits on every application, agrees with the atomic form to
    rounding, and both match the oracle."""
    import torch
    from paper_1601_08179_gb300 import sem
    from oracle import transform
    ctx, ms = make_pair(p, m, lam, ar)
    assert sem.default_opts().deterministic == 1
    ut = si.random_vector(ms.n_skeleton, 2100 + p)
    x = dev(ut)
    outs = []
    for _ in range(3):
        v = torch.full_like(x, np.nan)
        sem.sem_apply_condensed(ctx, x, v, sem.SPACE_TRANSFORMED)
        outs.append(host(v))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    sem.sem_set_opts(ctx, sem.default_opts(deterministic=0))
    va = torch.full_like(x, np.nan)
    sem.sem_apply_condensed(ctx, x, va, sem.SPACE_TRANSFORMED)
    assert relerr(host(va), outs[0]) <= 1e-14
    free = ms.skeleton_free
    u_nodal = transform.solution_from_transformed(ms, np.where(free, ut, 0.0))
    ref = transform.load_to_transformed(ms, np.where(free, local.apply_condensed(ms, lam, u_nodal), 0.0))
    assert relerr(outs[0], ref) <= 1e-12
    assert np.all(outs[0][~free] == 0.0)


def test_fixed_order_solves_repeat_bit_for_bit():
    """Repeated FP64 solves of one context, and the same problem set up in a
    second context, return identical solutions and iteration counts; the
    option switched off still solves to the tolerance."""
    import torch
    from paper_1601_08179_gb300 import sem
    p, m, lam, ar = 6, (4, 3, 5), 2.0, 8.0
    ctx, ms = make_pair(p, m, lam, ar)
    ctx2, _ = make_pair(p, m, lam, ar)
    f = dev(si.node_noise(ms.n_global, 2200))
    sols, iters = [], []
    for c in (ctx, ctx, ctx2):
        u = torch.empty(c.n_nodes, dtype=torch.float64, device="cuda")
        info = sem.sem_solve(c, f, u)
        sols.append(host(u))
        iters.append(info["iters"])
    assert iters[0] == iters[1] == iters[2]
    assert np.array_equal(sols[0], sols[1]), "repeat on one context"
    assert np.array_equal(sols[0], sols[2]), "a second context"
    sem.sem_set_opts(ctx, sem.default_opts(deterministic=0))
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    info = sem.sem_solve(ctx, f, u)
    assert info["rel_res"] <= 1e-10 and abs(info["iters"] - iters[0]) <= 2
    assert relerr(host(u), sols[0]) <= 1e-10


@pytest.mark.parametrize("p,m,mixed", [(8, (6, 5, 4), False), (4, (8, 6, 6), False), (8, (6, 5, 4), True),
                                      (20, (3, 2, 2), True)])
def test_autotune_keeps_results(p, m, mixed):
    import torch
    from paper_1601_08179_gb300 import sem
    opts = sem.default_opts(precision=sem.PREC_MIXED) if mixed else None
    ctx, ms = make_pair(p, m, 2.0, 4.0, opts=opts)
    ms_def, ms_best = sem.sem_autotune(ctx)
    assert 0 < ms_best <= ms_def
    u = si.random_vector(ms.n_skeleton, 81)
    v = torch.empty(ctx.nb, dtype=torch.float64, device="cuda")
    sem.sem_apply_condensed(ctx, dev(u), v, sem.SPACE_NODAL)
    assert relerr(host(v), local.apply_condensed(ms, 2.0, u)) <= 1e-12
    f = si.node_noise(ms.n_global, 82)
    w = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    sem.sem_solve(ctx, dev(f), w)
    F = local.rhs_full(ms, f)
    r = (local.apply_full(ms, 2.0, host(w)) - F)[ms.free_mask]
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(F[ms.free_mask])


def _mixed():
    from paper_1601_08179_gb300 import sem
    return sem.default_opts(precision=sem.PREC_MIXED)


def test_mixed_batch_matches_oracle_and_single_solves():
    """Mixed-precision problems (FP32 CG, reliable updates, FP64 refinement
    decided on the device) and FP64 problems in one graph: every solution
    within the solve bar of the dense oracle; the relative FP64 residual of
    each refinement step (sem_refine_history) ends below rtol."""
    import torch
    from paper_1601_08179_gb300 import sem
    probs = _small_batch(count=10, seed=73)
    ctxs, fs, us, refs, mixed = [], [], [], [], []
    for k, (p, m, lam, ar, seed) in enumerate(probs):
        mx = k % 4 != 3                       # every fourth problem stays FP64
        ctx, ms = make_pair(p, m, lam, ar, opts=_mixed() if mx else None)
        f = si.node_noise(ms.n_global, seed)
        ctxs.append(ctx)
        fs.append(dev(f))
        us.append(torch.full((ctx.n_nodes,), np.nan, dtype=torch.float64, device="cuda"))
        refs.append(dense.solve_full(ms, lam, f))
        mixed.append(mx)
    batch = sem.SemBatch(ctxs, fs, us)
    for rep in range(2):
        st, infos = batch.solve()
        for k, (u, ref) in enumerate(zip(us, refs)):
            assert relerr(host(u), ref) <= 1e-9, k
            assert infos[k]["rel_res"] <= 1e-10, k
            assert (infos[k]["refinements"] >= 1) == mixed[k], k
    for k, c in enumerate(ctxs):
        if not mixed[k]:
            continue
        hist = sem.sem_refine_history(c)
        assert len(hist) == infos[k]["refinements"] + 1 and abs(hist[0] - 1.0) < 1e-5
        assert hist[-1] <= 1e-10 and all(b < a for a, b in zip(hist, hist[1:])), hist
        u1 = torch.empty_like(us[k])
        sem.sem_solve(c, fs[k], u1)           # the single (host-looped) mixed solve of the same problem
        assert relerr(host(us[k]), host(u1)) <= 1e-9, k


def test_mixed_batch_high_degree_slab_kernel():
    """Mixed-precision problems whose FP32 operator is the k-slab kernel
    (p = 17, 20, 24: two and three slabs per element) and a low-degree one in
    one graph: every solution against the oracle's factorized PCG (rtol 1e-13)
    within the solve bar, and equal to the single solve of the same problem."""
    import torch
    from oracle import solve as osolve
    from paper_1601_08179_gb300 import sem
    probs = [(17, (2, 1, 2), 1.0, 2.0, 91), (20, (1, 2, 2), 10.0, 1.0, 92), (24, (2, 2, 1), 0.5, 4.0, 93),
             (6, (2, 2, 2), 1.0, 2.0, 94)]
    ctxs, fs, us, refs = [], [], [], []
    for p, m, lam, ar, seed in probs:
        ctx, ms = make_pair(p, m, lam, ar, opts=_mixed())
        assert sem.sem_get_operator_kernel(ctx, sem.PREC_MIXED)[0] == (sem.KERNEL_SLAB if p > 16 else sem.KERNEL_PLANE)
        f = si.node_noise(ms.n_global, seed)
        ctxs.append(ctx)
        fs.append(dev(f))
        us.append(torch.full((ctx.n_nodes,), np.nan, dtype=torch.float64, device="cuda"))
        refs.append(osolve.bt_solve(ms, lam, f, rtol=1e-13)[0])
    st, infos = sem.SemBatch(ctxs, fs, us).solve()
    for k, (u, ref) in enumerate(zip(us, refs)):
        assert relerr(host(u), ref) <= 1e-9, k
        assert infos[k]["rel_res"] <= 1e-10 and infos[k]["refinements"] >= 1, k
        u1 = torch.empty_like(u)
        sem.sem_solve(ctxs[k], fs[k], u1)
        assert relerr(host(u), host(u1)) <= 1e-9, k


def test_mixed_batch_heterogeneous_64_beats_fp64():
    """The 64-problem workload in mixed precision: every problem converges to
    rtol in FP64 terms, agrees with the FP64 batch to the solve bar, and the
    mixed batch takes less time than the FP64 batch."""
    import torch
    from paper_1601_08179_gb300 import sem
    work = si.batched_problems()
    batches, outs, times = {}, {}, {}
    for form in ("fp64", "mixed"):
        ctxs, fs, us = [], [], []
        for w in work:
            hx, hy, hz = w.widths()
            c = sem.sem_setup(w.p, hx, hy, hz, w.lam, _mixed() if form == "mixed" else None)
            ctxs.append(c)
            fs.append(dev(si.node_noise(c.n_nodes, w.seed)))
            us.append(torch.empty(c.n_nodes, dtype=torch.float64, device="cuda"))
        b = sem.SemBatch(ctxs, fs, us)
        b.solve()                             # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, infos = b.solve()
        e1.record()
        torch.cuda.synchronize()
        times[form] = e0.elapsed_time(e1)
        assert all(i["rel_res"] <= 1e-10 for i in infos), form
        batches[form], outs[form] = (b, ctxs, fs), us
    print("batch ms: fp64 %.1f, mixed %.1f" % (times["fp64"], times["mixed"]))
    for k in range(len(work)):
        assert relerr(host(outs["mixed"][k]), host(outs["fp64"][k])) <= 1e-8, k
    assert times["mixed"] < times["fp64"]


def test_mixed_batch_rejects_restarted_scheme():
    import torch
    from paper_1601_08179_gb300 import sem
    ctx, ms = make_pair(4, (2, 2, 2), 1.0, opts=sem.default_opts(precision=sem.PREC_MIXED, mixed_scheme=0))
    f = dev(si.node_noise(ms.n_global, 5))
    u = torch.empty(ctx.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as ei:
        sem.SemBatch([ctx], [f], [u])
    assert ei.value.status == sem.SEM_ENOTSUP
