#!/usr/bin/env python3
"""Benchmark of the condensed spectral-element Helmholtz solver on GB300.

One step = one full solve (Algorithm 4 of the paper): transformed condensed
load, CG with the BT preconditioner to a relative residual of 1e-10, interior
recovery, on the graded-mesh workload N = n_e p^3 ~ 1.68e7 (default p = 8 on
32^3 elements, aspect ratio 128, lambda = 0, manufactured right-hand side plus
seeded U[-1,1] noise).  Inputs are synthetic; f is resident in HBM when the
timed region starts.

Prints one JSON line (rank 0).  `value` is solve time per unknown (s/DOF,
lower is better) over all ranks; every rank solves its own replica of the
workload (weak scaling, no collective on the data path).  On one GPU the
default line also carries, measured after the timed region: the other
points of the graded grid (`sweep`), the paper's operator and solver
comparisons, the 64-problem batch (`batched64`) and the differentiable solve
(`adjoint`), each with its own CUDA-event timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--p 8] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sem_inputs as si  # noqa: E402

METRIC = "condensed-operator GDOF/s; PCG s/DOF to 1e-10, chosen form vs plain FP64 on GB300"
UNIT = "s/DOF"
# FP64 ceiling of the GB300: 152 SMs x 2 DFMA/clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 ceiling: 152 SMs x 128 FMA/clock x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_hbm(path: str = os.path.join(ROOT, "MEASURED_PEAKS.json")):
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth of this
    machine's GPUs, else the fallback figure of a GB300 copy, saying which."""
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback: 6.8 TB/s, an earlier GB300 copy (no measured peak)"


HBM_GBS, HBM_SOURCE = measured_hbm()
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--p", type=int, default=8, choices=list(si.SCALE_DEGREES))
    ap.add_argument("--ar", type=float, default=128.0)
    ap.add_argument("--lam", type=float, default=0.0)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the solves that measure the error against the oracle's recorded solve")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the other points of the graded grid (degree sweep, aspect ratio 1 and 8, "
                         "lambda = 1e2, the mixed-precision workload) measured after the headline")
    ap.add_argument("--workload", default="scale", choices=["scale", "mixed16", "batched", "adjoint"],
                    help="scale: graded N~1.68e7 workload of degree --p (default); mixed16: p = 16 on 16^3, "
                         "lambda = 10, AR 16; batched: 64 heterogeneous problems in one graph launch; "
                         "adjoint: forward + backward of the differentiable solve (p = 8 on 16^3)")
    ap.add_argument("--oracle-one-core", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--one-core-iters", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--one-core-target", type=float, default=8.0, help=argparse.SUPPRESS)
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="'both': time the plain FP64 solve and the mixed-precision solve (the headline)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_seed(w: si.Workload, rank: int) -> int:
    """Seed of rank `rank`'s replica: every rank solves its own right-hand side."""
    return w.seed + 1000 * rank


def whole_job_value(step_s_max: float, dofs_per_rank: int, world: int) -> float:
    """s/DOF of the whole job: the slowest rank's step time over all unknowns
    the ranks solved together."""
    return step_s_max / (dofs_per_rank * world)


def skeleton_size(p: int, m) -> int:
    """Length N_B of the packed skeleton vector of an m[0] x m[1] x m[2] mesh of
    degree p: n^2 values per face, n per edge, one per vertex (n = p - 1),
    Dirichlet entities included."""
    n = p - 1
    mx, my, mz = m
    faces = (mx + 1) * my * mz + mx * (my + 1) * mz + mx * my * (mz + 1)
    edges = mx * (my + 1) * (mz + 1) + (mx + 1) * my * (mz + 1) + (mx + 1) * (my + 1) * mz
    return faces * n * n + edges * n + (mx + 1) * (my + 1) * (mz + 1)


def workload_config(w: si.Workload, world: int) -> dict:
    """The `config` of a solve bench line; both arms print this same dict."""
    return {"workload": w.name, "p": w.p, "elements": list(w.m), "dofs_per_gpu": w.dofs,
            "skeleton_unknowns": skeleton_size(w.p, w.m), "lambda": w.lam, "aspect_ratio": w.ar,
            "rtol": 1e-10, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (solve working set > 129 MB)"}


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        busy = [x for x in sm if smax is None or x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def node_field(x, y, z, w: si.Workload, seed: int):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = si.manufactured_f(X, Y, Z, w.lam)
    if w.noise:
        f = f + si.node_noise(X.size, seed).reshape(X.shape)
    return np.ascontiguousarray(f.ravel())


# DRAM bytes (read + written) of one operator launch, from one ncu capture of
# the kernel as committed (the kernel summaries under profiles/; the FP64
# figures include the per-element edge/vertex shares of the fixed-order sums);
# a kernel or workload with no capture reports null.
TRAFFIC_BYTES = {
    ("k_tpt_apply_plane<7>", "graded_p8_m32_ar128_lam0"): 43244032 + 0,
    ("k_tpt_apply<double, 7> (epb 5, ks 7)", "graded_p8_m32_ar128_lam0"): 82519552 + 17870336,
    ("k_tpt_apply_slab", "graded_p32_m8_ar128_lam0"): 10740992 + 0,
    ("k_tpt_apply_p2<float>", "graded_p2_m128_ar128_lam0"): 117042176 + 14091520,
    ("k_tpt_apply_p2<double>", "graded_p2_m128_ar128_lam0"): 178927360 + 321355008,
    ("k_tpt_apply<double, 31> (epb 1, ks 8)", "graded_p32_m8_ar128_lam0"): 23401472 + 0,
    ("k_tpt_apply_plane<3>", "graded_p4_m64_ar128_lam0"): 77063680 + 213504,
    ("k_tpt_apply<double, 3> (epb 28, ks 3)", "graded_p4_m64_ar128_lam0"): 189429504 + 122293760,
    ("k_tpt_apply_plane2<15>", "graded_p16_m16_ar128_lam0"): 22298624 + 0,
    ("k_tpt_apply<double, 15> (epb 1, ks 15)", "graded_p16_m16_ar128_lam0"): 43648000 + 66304,
    ("k_tpt_apply_plane2<15>", "graded_p16_m16_ar16_lam10"): 22293760 + 0,
}


def kernel_name(sem, ctx, precision: int, p: int) -> str:
    """Name of the operator kernel in use for one precision."""
    kind, epb, ks = sem.sem_get_operator_kernel(ctx, precision)
    n = p - 1
    t = "float" if precision == sem.PREC_MIXED else "double"
    if kind == sem.KERNEL_PLANE:
        return f"k_tpt_apply_plane<{n}>" if n <= 8 else f"k_tpt_apply_plane2<{n}>"
    if kind == sem.KERNEL_SLAB:
        return "k_tpt_apply_slab"
    if kind == sem.KERNEL_ROW:
        return f"k_tpt_apply_row<{n}>"
    if kind == sem.KERNEL_PENCIL:
        return f"k_tpt_apply_pencil<{n}>"
    if kind == sem.KERNEL_WARP:
        return f"k_tpt_apply_warp<{t}, {n}>"
    if kind == sem.KERNEL_ELEMENT:
        return f"k_tpt_apply_p2<{t}>" if n == 1 else f"k_tpt_apply_elem<{n}>"
    return f"k_tpt_apply<{t}, {n if n in (1, 3, 7, 15, 31) else 0}> (epb {epb}, ks {ks})"


def roofline(sem, ctx, w: si.Workload, apply_s: float, precision: str) -> dict:
    """Roofline record of one operator launch of `precision` ("fp64" or
    "mixed", whose operator is FP32) taking `apply_s` seconds."""
    flops = apply_flops(w)
    nb = ctx.nb
    if precision == "fp64":
        name = kernel_name(sem, ctx, sem.PREC_FP64, w.p)
        achieved = flops / apply_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES.get((name, w.name)),
                "peak_source": "FP64 FMA units x SM clock (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                "flops_per_launch": flops}
    # FP32 operator: flops and bytes both near their ridge; report the bound
    # whose floor is larger
    name = kernel_name(sem, ctx, sem.PREC_MIXED, w.p)
    t_alu = flops / (FP32_PEAK_TFLOPS * 1e12)
    t_hbm = 8.0 * nb / (HBM_GBS * 1e9)
    if t_alu >= t_hbm:
        achieved = flops / apply_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES.get((name, w.name)),
                "peak_source": "FP32 FMA units x SM clock (152 SMs x 128 FMA/clk x 2.07 GHz)",
                "flops_per_launch": flops}
    achieved = 8.0 * nb / apply_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": HBM_GBS, "unit": "GB/s",
            "frac": achieved / HBM_GBS, "traffic": TRAFFIC_BYTES.get((name, w.name)), "peak_source": HBM_SOURCE,
            "bytes_per_launch": 8.0 * nb}


def sweep_workloads():
    """The other points of the graded-mesh grid, measured beside the headline:
    the degree sweep at aspect ratio 128 and lambda = 0, the p = 8 mesh at
    aspect ratio 1 and 8 and at lambda = 1e2, and the mixed-precision
    workload (p = 16 on 16^3 elements, lambda = 10, aspect ratio 16)."""
    out = [si.scale_workload(p) for p in (2, 4, 16, 32)]
    out += [si.scale_workload(8, ar=1.0), si.scale_workload(8, ar=8.0), si.scale_workload(8, lam=100.0)]
    return out + [si.MIXED]


def sweep_point(sem, w: si.Workload, seed: int, steps: int = 2) -> dict:
    """FP64 and mixed-precision solve time, iterations and operator time of
    one workload (CUDA events; one untimed warm-up solve per form)."""
    import torch
    hx, hy, hz = w.widths()
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam)
    x, y, z = sem.sem_node_coords(ctx)
    f = torch.from_numpy(node_field(x, y, z, w, seed)).cuda()
    u = torch.empty_like(f)
    rec = {"workload": w.name, "p": w.p, "elements": list(w.m), "aspect_ratio": w.ar, "lambda": w.lam,
           "dofs": w.dofs}
    for form, opts in (("fp64", sem.default_opts()), ("mixed", sem.default_opts(precision=sem.PREC_MIXED))):
        sem.sem_set_opts(ctx, opts)
        sem.sem_profile_enable(ctx, False)
        sem.sem_solve(ctx, f, u)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            info = sem.sem_solve(ctx, f, u)
        ev1.record()
        torch.cuda.synchronize()
        step_s = ev0.elapsed_time(ev1) / 1e3 / steps
        sem.sem_profile_enable(ctx, True)
        sem.sem_profile_read(ctx, reset=True)
        sem.sem_solve(ctx, f, u)
        apply_ms, apply_n = sem.sem_profile_read(ctx, reset=True)
        sem.sem_profile_enable(ctx, False)
        apply_s = apply_ms / 1e3 / max(apply_n, 1)
        roof = roofline(sem, ctx, w, apply_s, form)
        rec[form] = {"solve_ms": step_s * 1e3, "s_per_dof": step_s / w.dofs, "iters": info["iters"],
                     "refinements": info["refinements"], "rel_res": info["rel_res"],
                     "operator_us": apply_s * 1e6, "operator_kernel": roof["kernel"],
                     "operator_bound": roof["bound"], "operator_frac": roof["frac"]}
    rec["speedup_mixed_vs_fp64"] = rec["fp64"]["solve_ms"] / rec["mixed"]["solve_ms"]
    del ctx, f, u
    torch.cuda.empty_cache()
    return rec


# The paper's solver timings (Table 5: one Xeon E5-2690 core, 8^3 elements,
# expansion factor 2, i.e. aspect ratio 128, lambda = 0, residual reduced by
# 1e12): iteration time per DOF (ns) and solve time per DOF (us).  Context for
# the solver comparison below, measured on other hardware.
PAPER_TABLE5 = {8: {"BT": (25.6, 4.25), "UC": (52.3, 154.0), "DC": (56.2, 15.3), "BC": (75.7, 12.6)},
                16: {"BT": (17.7, 3.47)}}


def _event_time(fn, reps: int) -> float:
    """Seconds per call of fn (CUDA events, after one untimed call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def operator_variants(sem, w: si.Workload, reps: int = 10) -> dict:
    """One application of the condensed operator on the workload's mesh in
    FP64 by each of the paper's variants (Sec. 5): TPT in the transformed
    space (the operator of the BT solver), TPT between the nodal skeleton
    transforms, TPC (Algorithm 3 with Table 1) and MMC (Algorithm 2, its
    dense face matrices built first, timed separately)."""
    import torch
    hx, hy, hz = w.widths()
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam)
    x = torch.tensor(si.random_vector(ctx.nb, 3000), device="cuda")
    y = torch.empty_like(x)
    out = {"workload": w.name, "unit": "us per application, FP64"}
    out["tpt_transformed"] = _event_time(lambda: sem.sem_apply_condensed(ctx, x, y, sem.SPACE_TRANSFORMED), reps) * 1e6
    t0 = time.perf_counter()
    sem.sem_apply_condensed_variant(ctx, sem.OP_MMC, x, y)
    torch.cuda.synchronize()
    out["mmc_setup_s"] = time.perf_counter() - t0
    for name, op in (("tpt_nodal", sem.OP_TPT), ("tpc", sem.OP_TPC), ("mmc", sem.OP_MMC)):
        out[name] = _event_time(lambda: sem.sem_apply_condensed_variant(ctx, op, x, y), reps) * 1e6
    del ctx, x, y
    torch.cuda.empty_cache()
    return out


def paper_solvers(sem, p: int) -> dict:
    """The solver comparison of Sec. 8 / Table 5 on the paper's own mesh: 8^3
    elements graded in x and y to aspect ratio 128, lambda = 0, residual
    reduced by 1e12 (seeded load, homogeneous Dirichlet data).  BT is this
    library's solve (TPT operator, diagonal of the transformed operator);
    UC, DC, BC use the TPC operator with no, the nodal diagonal and the
    block-Jacobi preconditioner, FP64 throughout."""
    import torch
    hx, hy, hz, _ = si.graded_widths(8, 8, 8, ar=128.0, grade="xy")
    ctx = sem.sem_setup(p, hx, hy, hz, 0.0, sem.default_opts(rtol=1e-12))
    x, y, z = sem.sem_node_coords(ctx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = torch.tensor((si.manufactured_f(X, Y, Z, 0.0) + si.node_noise(X.size, 3100 + p).reshape(X.shape)).ravel(),
                     device="cuda")
    u = torch.empty_like(f)
    dofs = 512 * p ** 3
    out = {"workload": f"paper_table5_p{p}_m8_xy128_lam0", "dofs": dofs, "rtol": 1e-12}
    runs = {"BT": lambda: sem.sem_solve(ctx, f, u)}
    for name, pc in (("UC", sem.PC_NONE), ("DC", sem.PC_DIAG), ("BC", sem.PC_BLOCK)):
        runs[name] = (lambda pc=pc: sem.sem_solve_variant(ctx, sem.OP_TPC, pc, f, u))
    for name, fn in runs.items():
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = fn()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        rec = {"iters": info["iters"], "solve_ms": t * 1e3, "solve_us_per_dof": t / dofs * 1e6,
               "iteration_ns_per_dof": t / max(info["iters"], 1) / dofs * 1e9}
        if p in PAPER_TABLE5 and name in PAPER_TABLE5[p]:
            rec["paper_xeon_core"] = {"iteration_ns_per_dof": PAPER_TABLE5[p][name][0],
                                      "solve_us_per_dof": PAPER_TABLE5[p][name][1]}
        out[name] = rec
    del ctx
    torch.cuda.empty_cache()
    return out


def apply_flops(w: si.Workload) -> float:
    """Algorithmic FP64 flops of one condensed-operator application: the
    multiplication counts of Table 3 (TPT: 13 n^3 + 68 n^2 per element), each
    with its addition."""
    n = w.p - 1
    return 2.0 * (13 * n ** 3 + 68 * n ** 2) * w.n_elements


# --------------------------------------------------------------------------
# CPU oracle sample (the baseline; test infrastructure timed as it stands)
# --------------------------------------------------------------------------
def oracle_sample(w: si.Workload, iterations: int, target_s: float = 12.0):
    """Times the oracle on a slab of the workload's mesh: condensed load, one
    CG iteration (operator application + vector updates) and the interior
    recovery, then scales to the full element count and `iterations`."""
    from oracle import local
    from oracle.mesh import Mesh
    hx, hy, hz = w.widths()
    mz_s = 1
    t_est = None
    while True:
        ms = Mesh(w.p, hx, hy, hz[:mz_s])
        X, Y, Z = ms.coords()
        f = si.manufactured_f(X, Y, Z, w.lam).ravel()
        uB = si.random_vector(ms.n_skeleton, 1)
        c0 = time.process_time()
        t0 = time.perf_counter()
        fh = local.condensed_rhs(ms, w.lam, f)
        t1 = time.perf_counter()
        v = local.apply_condensed(ms, w.lam, uB)
        r = fh - 0.5 * v                      # CG vector work of one iteration
        z = r * 1.0
        _ = float(r @ z) + float(uB @ v)
        uB2 = uB + 0.5 * z
        t2 = time.perf_counter()
        local.recover_interior(ms, w.lam, f, uB2)
        t3 = time.perf_counter()
        cpu_s = time.process_time() - c0
        t_est = (t1 - t0, t2 - t1, t3 - t2)
        total = sum(t_est)
        if total * 2 > target_s or mz_s >= w.m[2]:
            break
        mz_s = min(w.m[2], max(mz_s + 1, int(mz_s * min(4.0, target_s / max(total, 1e-3) / 2))))
    scale = w.m[2] / mz_s
    t_full = scale * (t_est[0] + t_est[2] + iterations * t_est[1])
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # threads the sample kept busy on average: process CPU time (all threads) over wall time
    threads = cpu_s / max(sum(t_est), 1e-9)
    return {"value": t_full / w.dofs, "unit": UNIT, "cores": cores, "threads": round(threads, 2), "kind": "oracle",
            "sample": (f"NumPy FP64 oracle (element-local tier) on the {w.m[0]}x{w.m[1]}x{mz_s} slab of the "
                       f"{w.m[0]}x{w.m[1]}x{w.m[2]} mesh: condensed load {t_est[0]:.2f}s, one CG iteration "
                       f"{t_est[1]:.2f}s, recovery {t_est[2]:.2f}s; scaled x{scale:g} to the full mesh and to "
                       f"{iterations} CG iterations"),
            "sample_s": sum(t_est)}


BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def oracle_sample_one_core(w: si.Workload, iterations: int, target_s: float = 8.0):
    """oracle_sample in a child process pinned to one host core with one BLAS
    thread (the like-for-like figure for the paper's single-core timings).
    The BLAS thread counts are set in the child's environment, so they hold
    from the moment NumPy loads; None if the child fails."""
    env = dict(os.environ)
    env.update({k: "1" for k in BLAS_THREAD_VARS})
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-one-core", "--p", str(w.p), "--ar", repr(w.ar),
           "--lam", repr(w.lam), "--one-core-iters", str(iterations), "--one-core-target", repr(target_s)]
    try:
        res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
        return json.loads(lines[-1]) if res.returncode == 0 and lines else None
    except (OSError, ValueError, subprocess.TimeoutExpired):
        return None


def one_core_child(args):
    """Body of the one-core child: pins itself to one core of its affinity
    set, then prints oracle_sample's result as JSON."""
    if hasattr(os, "sched_setaffinity"):
        os.sched_setaffinity(0, {min(os.sched_getaffinity(0))})
    w = si.scale_workload(args.p, ar=args.ar, lam=args.lam)
    out = oracle_sample(w, args.one_core_iters, target_s=args.one_core_target)
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def time_solves(sem, ctx, f, u, steps, warmup, world, local_rank):
    """Times `steps` solves after `warmup`, CUDA events on the caller's stream,
    clocks sampled during the timed region; then the operator's own launch
    time inside `steps` more solves, measured by event nodes in the solve
    graphs (kept out of the timed region: they cost about 1 % of a solve per
    hundred iterations).  Returns a dict."""
    import torch
    sem.sem_profile_enable(ctx, False)
    for _ in range(warmup):
        sem.sem_solve(ctx, f, u)
    torch.cuda.synchronize()
    barrier(world)
    launches0 = sem.sem_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            infos.append(sem.sem_solve(ctx, f, u))
        ev1.record()
        torch.cuda.synchronize()
    barrier(world)
    launches = sem.sem_launch_count() - launches0
    step_s = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / steps, world)
    sem.sem_profile_enable(ctx, True)
    sem.sem_profile_read(ctx, reset=True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record()
    for _ in range(steps):
        sem.sem_solve(ctx, f, u)
    ev3.record()
    torch.cuda.synchronize()
    apply_ms, apply_n = sem.sem_profile_read(ctx, reset=True)
    sem.sem_profile_enable(ctx, False)
    return {"step_s": step_s, "info": infos[-1], "apply_s": apply_ms / 1e3 / max(apply_n, 1),
            "apply_n": apply_n, "launches": launches, "clocks": clk.summary(),
            "profiled_step_s": ev2.elapsed_time(ev3) / 1e3 / steps}


def our_arm(args, rank, world, local_rank):
    import torch

    from paper_1601_08179_gb300 import build, sem

    build.build()
    torch.cuda.set_device(local_rank)
    w = si.MIXED if args.workload == "mixed16" else si.scale_workload(args.p, ar=args.ar, lam=args.lam)
    seed = replica_seed(w, rank)
    hx, hy, hz = w.widths()
    t0 = time.perf_counter()
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam)
    setup_s = time.perf_counter() - t0
    x, y, z = sem.sem_node_coords(ctx)
    f_host = node_field(x, y, z, w, seed)
    f = torch.from_numpy(f_host).cuda()
    u = torch.empty_like(f)

    forms = {"fp64": sem.default_opts(), "mixed": sem.default_opts(precision=sem.PREC_MIXED)}
    order = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {}
    for form in order:
        sem.sem_set_opts(ctx, forms[form])
        res[form] = time_solves(sem, ctx, f, u, args.steps, args.warmup, world, local_rank)
        if form == "mixed":
            res[form]["refine_hist"] = [float(v) for v in sem.sem_refine_history(ctx)]
    head = order[-1]          # the chosen form: mixed unless only fp64 was asked for
    r = res[head]
    sem.sem_set_opts(ctx, forms[head])

    # end to end through the host-buffer entry point: H2D f, solve, D2H u
    e2e_steps = args.steps if args.e2e_steps is None else args.e2e_steps
    e2e_s = None
    if e2e_steps > 0:
        f_pin = torch.from_numpy(f_host).pin_memory().numpy()
        u_pin = torch.empty(f_host.size, dtype=torch.float64).pin_memory().numpy()
        sem.sem_solve_host(ctx, f_pin, u_pin)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            sem.sem_solve_host(ctx, f_pin, u_pin)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)

    flops = apply_flops(w)
    nb = ctx.nb
    assert nb == skeleton_size(w.p, w.m), (nb, w.p, w.m)
    roof = roofline(sem, ctx, w, r["apply_s"], head)
    out = {
        "metric": METRIC,
        "value": whole_job_value(r["step_s"], w.dofs, world),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["step_s"] * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32+f64",
        "data": "synthetic",
        "precision": head,
        "config": workload_config(w, world),
        "solve": {"iters": r["info"]["iters"], "refinements": r["info"]["refinements"],
                  "rel_res": r["info"]["rel_res"], "setup_s": setup_s},
        "operator": {"gdof_s": w.dofs / r["apply_s"] / 1e9, "apply_ms": r["apply_s"] * 1e3,
                     "timed_launches": r["apply_n"], "dtype": "f64" if head == "fp64" else "f32",
                     "measured_in": "event nodes around each operator launch in the solve graphs, in solves "
                                    "repeated after the timed region (%.2f ms per solve with the events)"
                                    % (r["profiled_step_s"] * 1e3)},
        "roofline": roof,
        "e2e": {"value": whole_job_value(e2e_s, w.dofs, world) if e2e_s else None, "unit": UNIT,
                "h2d_bytes_per_step": f_host.nbytes, "d2h_bytes_per_step": f_host.nbytes},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    if "mixed" in res:
        out["solve"]["refine_hist"] = res["mixed"]["refine_hist"]
    if "fp64" in res and head != "fp64":
        p64 = res["fp64"]
        out["fp64"] = {"value": whole_job_value(p64["step_s"], w.dofs, world), "ms_per_step": p64["step_s"] * 1e3,
                       "iters": p64["info"]["iters"], "operator_gdof_s": w.dofs / p64["apply_s"] / 1e9,
                       "operator_ms": p64["apply_s"] * 1e3,
                       "operator_frac_fp64_peak": flops / p64["apply_s"] / 1e12 / FP64_PEAK_TFLOPS,
                       "clocks": p64["clocks"]}
        out["speedup_vs_fp64"] = p64["step_s"] / r["step_s"]
    rec = oracle_record(w) if rank == 0 and not args.no_oracle_error else None
    if rec is not None and "mixed" in res:
        out["error_vs_oracle"] = errors_vs_oracle(sem, ctx, f, u, rec, int(res["mixed"]["info"]["refinements"]),
                                                  forms[head])
    if world == 1 and args.workload == "scale" and not args.no_sweep:
        # every other point of the graded grid, measured in this run after the timed region
        out["sweep"] = [sweep_point(sem, sw, replica_seed(sw, rank)) for sw in sweep_workloads()]
        # the paper's comparison operators (Sec. 5) and solvers (Sec. 8, Table 5)
        if w.p <= 16:
            out["operator_variants"] = operator_variants(sem, w)
        out["paper_solvers"] = [paper_solvers(sem, pp) for pp in (8, 16)]
        # the batched and differentiable workloads, also after the timed region
        out["batched64"] = measure_batched(2, 1, rank, world, local_rank, ["fp64", "mixed"])
        out["adjoint"] = measure_adjoint(3, 2, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref_iters = reference_iterations(w)
        iters = res["fp64"]["info"]["iters"] if "fp64" in res else r["info"]["iters"]
        cb_iters = ref_iters if ref_iters is not None else iters
        out["cpu_baseline"] = oracle_sample(w, cb_iters, target_s=8.0)
        if ref_iters is None:
            out["cpu_baseline"]["sample"] += " (iteration count of this GPU FP64 solve; no oracle solve recorded)"
        one = oracle_sample_one_core(w, cb_iters) if args.workload == "scale" else None
        out["cpu_baseline"]["one_core"] = (
            {"value": one["value"], "unit": UNIT, "cores": 1, "threads": one["threads"], "sample": one["sample"]}
            if one else None)
    if rank == 0:
        print(json.dumps(out), flush=True)


def batched_arm(args, rank, world, local_rank):
    """64 heterogeneous problems solved by one graph launch per step: the
    plain FP64 batch and the mixed-precision batch (FP32 CG with reliable
    updates, FP64 refinement decided on the device), the latter the headline."""
    import torch
    from paper_1601_08179_gb300 import build
    build.build()
    torch.cuda.set_device(local_rank)
    forms = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    out = measure_batched(args.steps, args.warmup, rank, world, local_rank, forms)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_batched(steps, warmup, rank, world, local_rank, forms):
    """The batched64 line (see batched_arm)."""
    import torch

    from paper_1601_08179_gb300 import sem
    work = si.batched_problems()
    dofs = sum(w.dofs for w in work)
    res = {}
    for form in forms:
        opts = sem.default_opts(precision=sem.PREC_MIXED) if form == "mixed" else None
        ctxs, fs, us = [], [], []
        for w in work:
            hx, hy, hz = w.widths()
            c = sem.sem_setup(w.p, hx, hy, hz, w.lam, opts)
            sem.sem_autotune(c)
            ctxs.append(c)
            fs.append(torch.from_numpy(si.node_noise(c.n_nodes, replica_seed(w, rank))).cuda())
            us.append(torch.empty(c.n_nodes, dtype=torch.float64, device="cuda"))
        batch = sem.SemBatch(ctxs, fs, us)
        for _ in range(warmup):
            batch.solve()
        torch.cuda.synchronize()
        barrier(world)
        l0 = sem.sem_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            ev0.record()
            for _ in range(steps):
                st, infos = batch.solve()
            ev1.record()
            torch.cuda.synchronize()
        barrier(world)
        res[form] = {"step_s": max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / steps, world), "infos": infos,
                     "launches": sem.sem_launch_count() - l0, "clocks": clk.summary()}
        del batch, ctxs, fs, us
        torch.cuda.empty_cache()
    head = forms[-1]
    r = res[head]
    out = {"metric": METRIC + " (batched problems)", "value": whole_job_value(r["step_s"], dofs, world), "unit": UNIT,
           "n_gpus": world, "steps": steps, "warmup": warmup, "ms_per_step": r["step_s"] * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": "batched64", "problems": len(work), "dofs_total": dofs,
                      "degrees": sorted(set(w.p for w in work)), "rtol": 1e-10,
                      "parallelism": f"replicas{world}"},
           "precision": head,
           "iters_max": max(i["iters"] for i in r["infos"]), "iters_sum": sum(i["iters"] for i in r["infos"]),
           "rel_res_max": max(i["rel_res"] for i in r["infos"]),
           "gpu_launches": r["launches"], "clocks": r["clocks"]}
    if head == "mixed":
        out["refinements_max"] = max(i["refinements"] for i in r["infos"])
    if "fp64" in res and head != "fp64":
        p64 = res["fp64"]
        out["fp64"] = {"value": whole_job_value(p64["step_s"], dofs, world), "ms_per_step": p64["step_s"] * 1e3,
                       "iters_max": max(i["iters"] for i in p64["infos"]), "clocks": p64["clocks"]}
        out["speedup_vs_fp64"] = p64["step_s"] / r["step_s"]
    return out


def adjoint_arm(args, rank, world, local_rank):
    """Forward solve + backward (adjoint solve and gradient kernels) of the
    differentiable solve, J = 1/2 ||u - u_target||^2."""
    import torch
    from paper_1601_08179_gb300 import build
    build.build()
    torch.cuda.set_device(local_rank)
    out = measure_adjoint(args.steps, args.warmup, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_adjoint(steps, warmup, rank, world, local_rank):
    """The adjoint line (see adjoint_arm)."""
    import torch

    from paper_1601_08179_gb300 import sem
    from paper_1601_08179_gb300.autograd import context_for, helmholtz_solve
    w = si.ADJOINT
    hx, hy, hz = w.widths()
    ctx = context_for(w.p, hx, hy, hz, w.lam)
    x, y, z = sem.sem_node_coords(ctx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f0 = torch.tensor(si.manufactured_f(X, Y, Z, w.lam).ravel(), device="cuda")
    ut = torch.tensor(si.smooth_target(X, Y, Z, w.seed).ravel(), device="cuda")
    lam = torch.tensor(w.lam, dtype=torch.float64, requires_grad=True)
    hs = [torch.tensor(h, dtype=torch.float64, requires_grad=True) for h in (hx, hy, hz)]

    def step():
        f = f0.clone().requires_grad_(True)
        u = helmholtz_solve(f, lam, *hs, w.p)
        J = 0.5 * ((u - ut) ** 2).sum()
        J.backward()
        return float(J)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record()
        for _ in range(steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    barrier(world)
    step_s = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / steps, world)
    return {"metric": METRIC + " (forward + adjoint gradient)", "value": whole_job_value(step_s, w.dofs, world),
            "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "p": w.p, "elements": list(w.m), "lambda": w.lam},
            "clocks": clk.summary()}


def oracle_record(w: si.Workload):
    """The oracle's full-size solve of this workload, as recorded in
    tests/golden by `python -m oracle.reference_solve` (None if not recorded)."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


def errors_vs_oracle(sem, ctx, f, u, rec, refinements: int, form_opts):
    """Relative error, over the recorded sample nodes, against the oracle's
    solve (rtol 1e-12) of the FP64 solution and of the mixed-precision
    solution after each FP64 refinement step (the mixed solve re-run with
    max_refine = 1, 2, ...).  Outside the timed region."""
    import torch
    idx = torch.as_tensor(np.asarray(rec["u_samples"]["index"], dtype=np.int64), device=u.device)
    want = np.asarray(rec["u_samples"]["value"])

    def err():
        got = u[idx].cpu().numpy()
        return float(np.linalg.norm(got - want) / np.linalg.norm(want))

    out = {"samples": int(want.size), "reference": "oracle Algorithm 4 solve of this workload, rtol %g" % rec["rtol"]}
    sem.sem_set_opts(ctx, sem.default_opts())
    sem.sem_solve(ctx, f, u)
    out["fp64"] = err()
    steps = []
    for k in range(1, refinements + 1):
        sem.sem_set_opts(ctx, sem.default_opts(precision=sem.PREC_MIXED, max_refine=k))
        sem.sem_solve(ctx, f, u, check=False)
        steps.append(err())
    out["mixed_per_refinement_step"] = steps
    sem.sem_set_opts(ctx, form_opts)
    return out


def reference_iterations(w: si.Workload):
    """CG iterations to 1e-10 of the oracle's own solve of this workload, as
    recorded by `python -m oracle.reference_solve` (None if not recorded)."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return int(json.load(fh)["iterations_to_1e-10"])


def reference_arm(args, rank, world):
    """The oracle, timed as it stands on the host cores, per step one bounded
    sample of the same workload, scaled by the iteration count of the
    oracle's own full solve of this workload (tests/golden)."""
    if rank != 0:
        return
    w = si.scale_workload(args.p, ar=args.ar, lam=args.lam)
    iters = reference_iterations(w)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle solve recorded for {w.name}; "
                          f"run python -m oracle.reference_solve {w.p}"}), flush=True)
        return
    samples = []
    for i in range(args.warmup + args.steps):
        s = oracle_sample(w, iters, target_s=6.0)
        if i >= args.warmup:
            samples.append(s)
    v = statistics.median(s["value"] for s in samples)
    last = samples[-1]
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.median(s["sample_s"] for s in samples) * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "precision": "fp64", "config": workload_config(w, world),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "threads": last["threads"],
                            "kind": "oracle", "sample": last["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.oracle_one_core:
        one_core_child(args)
        return
    rank, world, local_rank = dist_setup()
    try:
        if args.impl == "reference":
            reference_arm(args, rank, world)
        elif args.workload == "batched":
            batched_arm(args, rank, world, local_rank)
        elif args.workload == "adjoint":
            adjoint_arm(args, rank, world, local_rank)
        else:
            our_arm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
