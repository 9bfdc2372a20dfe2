"""Applies one operator variant a few times on a graded workload: the launch
that kernel profiles capture.

    python -m paper_1601_08179_gb300.apply_loop --op plane --p 8 --reps 4

--op names the FP32 mapping of the transformed condensed operator (plane,
pencil, row, slab, elem, warp, cta, auto) or an FP64 form (tpt64, tpc, mmc), --p the degree
of the graded workload (the elements per direction follow the degree, as in
bench.py).  The input is a seeded random vector; nothing is checked.  It
prints the mean time of one application (CUDA events around the loop, after
one untimed application).  --atomic selects the FP64 operator's atomic edge
and vertex scatter instead of the fixed-order sums.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import sem_inputs as si  # noqa: E402


def main(argv=None) -> None:
    import torch
    from paper_1601_08179_gb300 import build, sem
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--op", default="plane",
                    choices=["plane", "pencil", "row", "slab", "elem", "warp", "cta", "auto", "tpt64", "tpc", "mmc"])
    ap.add_argument("--p", type=int, default=8, choices=list(si.SCALE_DEGREES))
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--atomic", action="store_true")
    a = ap.parse_args(argv)
    build.build()
    w = si.scale_workload(a.p)
    hx, hy, hz = w.widths()
    f32 = a.op in ("plane", "pencil", "row", "slab", "elem", "warp", "cta", "auto")
    opts = sem.default_opts(precision=sem.PREC_MIXED if f32 else sem.PREC_FP64, deterministic=0 if a.atomic else 1)
    ctx = sem.sem_setup(w.p, hx, hy, hz, w.lam, opts)
    gen = torch.Generator(device="cuda").manual_seed(1234)
    if f32:
        kern = {"plane": sem.KERNEL_PLANE, "pencil": sem.KERNEL_PENCIL, "row": sem.KERNEL_ROW, "slab": sem.KERNEL_SLAB, "elem": sem.KERNEL_ELEMENT,
                "warp": sem.KERNEL_WARP, "cta": sem.KERNEL_CTA_TILE, "auto": sem.KERNEL_AUTO}[a.op]
        sem.sem_set_operator_kernel(ctx, sem.PREC_MIXED, kern)
        x = torch.randn(ctx.nb, dtype=torch.float32, device="cuda", generator=gen)
        y = torch.zeros_like(x)

        def apply():
            sem.sem_apply_condensed_f32(ctx, x, y)
    else:
        x = torch.randn(ctx.nb, dtype=torch.float64, device="cuda", generator=gen)
        y = torch.zeros_like(x)

        def apply():
            if a.op == "tpt64":
                sem.sem_apply_condensed(ctx, x, y, sem.SPACE_TRANSFORMED)
            else:
                sem.sem_apply_condensed_variant(ctx, sem.OP_TPC if a.op == "tpc" else sem.OP_MMC, x, y)
    apply()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        apply()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.reps, 1)
    print(f"{a.op} p={a.p}{' atomic' if a.atomic else ''}: {a.reps} applications of {ctx.nb} skeleton unknowns, "
          f"{ms * 1e3:.1f} us each (host calls included)")


if __name__ == "__main__":
    main()
