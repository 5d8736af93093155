"""The checked build (libmpm_b300_checked.so, MPM_CHECKED=1).

Every indirect index of the hot kernels is tested against its buffer there:
- block ranks from the work list, the sort keys and the neighbour table;
- particle indices from the sort permutation;
- table slots from the particle codes;
- scatter positions.

An index out of range raises a map error instead of touching memory. This
build runs the same steps as the normal one in a separate process, since a
process loads one build. It must give the same bits in deterministic mode and
raise no error in either mode. The cases cover the sparse and dense grids, the
hash and the scan, Neo-Hookean and Drucker-Prager, and an ensemble."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

RUN = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[3])
from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import small_blob

case, out = sys.argv[1], sys.argv[2]
if case == "cube_det":
    wl = W.elastic_cube(steps=1)
    wl.v = np.tile(np.array([[0.4, -0.2, 0.1]], np.float32), (wl.n, 1))
    sim, n = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC), 20
elif case == "cube_dense_det":
    wl = W.elastic_cube(steps=1)
    sim, n = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mpm.DENSE_GRID), 20
elif case == "blob_dp_scan_det":
    wl, Cm, F = small_blob(n=4000, seed=19, material=W.DRUCKER_PRAGER, E=1e6)
    cfg = mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC | mpm.SCAN_COMPACTION)
    sim, n = mpm.Simulation(cfg, wl.x, wl.v, Cm, F), 20
elif case == "ensemble_det":
    wl = W.column_ensemble(n_scenarios=4, n_min=5000, n_max=40000)
    sim, n = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC), 15
elif case == "column_fast":
    wl = W.column_collapse(cells_xy=16, cells_z=64)
    sim, n = mpm.Simulation.from_workload(wl), 30
else:
    raise SystemExit("unknown case " + case)
sim.step(n)
st = sim.read_particles()
np.savez(out, blocks=np.int64(sim.stats()["n_active_blocks"]), **st)
"""


def _run(case, lib, out):
    env = dict(os.environ, MPM_B300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", RUN, case, out, ROOT], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


@pytest.fixture(scope="module")
def libs():
    from paper_2605_28525_b300 import build
    if not os.path.exists(build.CHECKED_LIB):
        build.build_checked()
    return build.LIB, build.CHECKED_LIB


@pytest.mark.parametrize("case", ["cube_det", "cube_dense_det", "blob_dp_scan_det", "ensemble_det"])
def test_checked_build_same_bits(libs, tmp_path, case):
    a = _run(case, libs[0], str(tmp_path / "a.npz"))
    b = _run(case, libs[1], str(tmp_path / "b.npz"))
    assert int(a["blocks"]) == int(b["blocks"])
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (case, k)


def test_checked_build_fast_mode_runs_clean(libs, tmp_path):
    a = _run("column_fast", libs[0], str(tmp_path / "a.npz"))
    b = _run("column_fast", libs[1], str(tmp_path / "b.npz"))
    assert int(a["blocks"]) == int(b["blocks"])
    assert np.abs(a["x"] - b["x"]).max() <= 1e-5
