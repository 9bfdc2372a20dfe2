"""Host logic of bench.py that needs no GPU: the packed skeleton length the
oracle arm reports (against the oracle mesh's own count) and the workload
config both arms print.  CPU only."""
import numpy as np
import pytest

import bench
import sem_inputs as si
from oracle.mesh import Mesh


@pytest.mark.parametrize("p,m", [(2, (1, 1, 1)), (3, (2, 1, 3)), (4, (3, 3, 2)), (8, (1, 4, 2)), (17, (2, 2, 1))])
def test_skeleton_size_matches_oracle_mesh(p, m):
    hx, hy, hz, _ = si.graded_widths(*m)
    assert bench.skeleton_size(p, m) == Mesh(p, hx, hy, hz).n_skeleton


def test_workload_config_of_the_degree_sweep():
    for p in si.SCALE_DEGREES:
        w = si.scale_workload(p)
        c = bench.workload_config(w, 1)
        assert c["workload"] == w.name and c["p"] == p and c["parallelism"] == "replicas1"
        assert c["dofs_per_gpu"] == w.dofs == int(np.prod(w.m)) * p ** 3
        assert c["skeleton_unknowns"] == bench.skeleton_size(p, w.m)
    assert bench.workload_config(si.scale_workload(8), 1)["skeleton_unknowns"] == 5735169


def test_whole_job_value_counts_every_rank():
    assert bench.whole_job_value(0.5, 1000, 4) == pytest.approx(0.5 / 4000)


def test_hbm_peak_names_its_source(tmp_path):
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 7001.5}')
    assert bench.measured_hbm(str(f)) == (7001.5, "MEASURED_PEAKS.json hbm_gbs (copy)")
    gbs, src = bench.measured_hbm(str(tmp_path / "missing.json"))
    assert gbs == 6800.0 and src.startswith("fallback")
