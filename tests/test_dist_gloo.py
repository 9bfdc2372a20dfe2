"""The N > 1 host path of bench.py on CPU: two gloo ranks.

The solver shards by replica only (every rank solves its own seeded copy of
the workload, no collective on the data path), so what runs across ranks is
host logic: rendezvous, the barriers around the timed region, the max over
ranks of the step time, the per-rank seeds, the whole-job value, and rank 0
alone printing (for the reference arm, rank 0 alone working)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import sem_inputs as si
    r, wsz, local = bench.dist_setup()
    try:
        assert (r, wsz, local) == (rank, world, rank)
        assert dist.get_backend() == "gloo"
        bench.barrier(wsz)
        step_max = bench.max_over_ranks(0.25 * (rank + 1), wsz)
        w = si.scale_workload(8)
        q.put({"rank": r, "max": step_max, "seed": bench.replica_seed(w, r),
               "value": bench.whole_job_value(step_max, w.dofs, wsz)})
        bench.barrier(wsz)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_replica_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import sem_inputs as si
    dofs = si.scale_workload(8).dofs
    # every rank sees the slowest rank's time, and the value counts both replicas
    assert [d["max"] for d in out] == [0.5, 0.5]
    assert all(d["value"] == pytest.approx(0.5 / (2 * dofs), rel=1e-15) for d in out)
    # the replicas solve different right-hand sides
    assert out[0]["seed"] != out[1]["seed"]


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` under torchrun with two ranks: rank 0 alone
    times the oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["unit"] == "s/DOF" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"] == {"value": d["value"], "unit": "s/DOF", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same workload config as the arm that runs the library, the oracle's precision beside it
    sys.path.insert(0, ROOT)
    import bench
    import sem_inputs as si
    assert d["config"] == bench.workload_config(si.scale_workload(8), 2)
    assert d["precision"] == "fp64" and d["dtype"] == "f64"
