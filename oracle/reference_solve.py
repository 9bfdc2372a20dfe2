"""Writes the oracle's full-size reference record of a benchmark workload.

    python -m oracle.reference_solve [p | mixed16] [--ar 128] [--lam 0] [--rtol 1e-12]

Runs the oracle's Algorithm 4 (oracle.solve.bt_solve) on the graded workload
of degree p (N ~ 1.68e7; x-graded to aspect ratio --ar, Helmholtz parameter
--lam), or on the mixed-precision workload (p = 16 on 16^3 elements,
lambda = 10, aspect ratio 16), with the right-hand side built from
the oracle's own node coordinates, and stores in
tests/golden/oracle_<workload>.json:
  * the CG iteration count at which ||r|| <= 1e-10 ||b|| (used to scale CPU
    timing samples of the oracle) and the full residual history endpoints;
  * seeded samples of the solution, of the transformed diagonal and of the
    nodal condensed load, for full-size parity tests.
Only oracle/ and sem_inputs are used.  Takes about an hour on 8 cores.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sem_inputs as si  # noqa: E402
from oracle import local, solve  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402

SAMPLES = 2000


def golden_path(w: si.Workload) -> str:
    return os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")


def main():
    arg = sys.argv[1] if len(sys.argv) > 1 and not sys.argv[1].startswith("-") else "8"
    def opt(name, default):
        return float(sys.argv[sys.argv.index(name) + 1]) if name in sys.argv else default

    rtol = opt("--rtol", 1e-12)
    w = si.MIXED if arg == "mixed16" else si.scale_workload(int(arg), ar=opt("--ar", 128.0), lam=opt("--lam", 0.0))
    hx, hy, hz = w.widths()
    ms = Mesh(w.p, hx, hy, hz)
    X, Y, Z = ms.coords()
    f = (si.manufactured_f(X, Y, Z, w.lam) + si.node_noise(X.size, w.seed).reshape(X.shape)).ravel()
    t0 = time.time()
    diag = local.transformed_diagonal(ms, w.lam)
    print(f"diagonal {time.time() - t0:.1f}s", flush=True)
    fhat = local.condensed_rhs(ms, w.lam, f)

    def cb(it, rel):
        if it % 50 == 0:
            print(f"it {it} rel {rel:.3e} t {time.time() - t0:.0f}s", flush=True)

    u, ut, it, hist = solve.bt_solve(ms, w.lam, f, rtol=rtol, diag=diag, callback=cb)
    it10 = next(i for i, h in enumerate(hist) if h <= 1e-10)
    g = np.random.Generator(np.random.PCG64(w.seed + 77))
    node_idx = np.sort(g.choice(ms.n_global, SAMPLES, replace=False))
    free_slots = np.flatnonzero(ms.skeleton_free)
    skel_idx = np.sort(g.choice(free_slots, SAMPLES, replace=False))
    rec = {
        "workload": w.name, "p": w.p, "m": list(w.m), "lambda": w.lam, "aspect_ratio": w.ar, "seed": w.seed,
        "rhs": "manufactured_f at the oracle's node coordinates + node_noise(seed)",
        "solver": "oracle.solve.bt_solve (Algorithm 4, CG with the transformed diagonal)",
        "iterations_to_1e-10": int(it10), "iterations": int(it), "rtol": rtol, "final_rel_res": hist[-1],
        "u_norm2": float(np.linalg.norm(u)), "u_absmax": float(np.abs(u).max()),
        "u_samples": {"index": node_idx.tolist(), "value": u[node_idx].tolist()},
        "diag_samples": {"index": skel_idx.tolist(), "value": diag[skel_idx].tolist()},
        "fhat_nodal_samples": {"index": skel_idx.tolist(), "value": fhat[skel_idx].tolist()},
        "fhat_nodal_norm2": float(np.linalg.norm(fhat)),
        "seconds": time.time() - t0,
    }
    with open(golden_path(w), "w") as fh:
        json.dump(rec, fh)
    print(f"wrote {golden_path(w)}: {it10} iterations to 1e-10, {it} to {rtol:g}", flush=True)


if __name__ == "__main__":
    main()
