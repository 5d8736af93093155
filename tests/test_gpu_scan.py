"""MPM_SCAN_COMPACTION: the paper's scan realisation of the active set
(Sec. 4.2, Alg. 2-4: mark a bit per block, scan, Phi = rank) on the GPU in
place of the hash (Sec. 4.3).  Both realisations must give the same active
set, the same Phi and therefore the same bits."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import eq_keys, oracle_for, small_blob
from tests.test_gpu_batch import _explosion

pytestmark = pytest.mark.gpu

SCAN = mpm.SCAN_COMPACTION


def _bits(sim):
    p = sim.read_particles()
    return {k: p[k].view(np.uint32).copy() for k in ("x", "v", "C", "F")}


@pytest.mark.parametrize("B", [1, 4])
@pytest.mark.parametrize("seed", [3, 8])
def test_scan_active_set_bit_exact(oracle_mod, B, seed):
    wl, Cm, F = small_blob(n=5000, seed=seed, block_size=B)
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=SCAN), wl.x, wl.v, Cm, F)
    sim.rebuild_active()
    assert np.array_equal(sim.read_active(), eq_keys(oracle_for(wl).active_blocks(wl.x)))
    assert sim.stats()["hash_capacity"] == 0


def test_scan_equals_hash_bitwise(oracle_mod):
    wl = W.column_collapse(cells_xy=8, cells_z=16, steps=30)
    out = []
    for flags in (mpm.DETERMINISTIC, mpm.DETERMINISTIC | SCAN, mpm.DETERMINISTIC | SCAN | mpm.SYNC_STEPS):
        sim = mpm.Simulation.from_workload(wl, flags=flags)
        sim.step(wl.steps)
        out.append(_bits(sim))
    for o in out[1:]:
        for k in o:
            assert np.array_equal(o[k], out[0][k]), k


def test_scan_batch_regrowth(oracle_mod):
    wl = _explosion(seed=13)
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | SCAN)
    a.step(1)
    a.step(79)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    b.step(80)
    assert a.stats()["rebuild_rounds"] >= 1
    for k, v in _bits(a).items():
        assert np.array_equal(v, _bits(b)[k]), k


def test_scan_ensemble_matches_hash_ensemble(oracle_mod):
    ens = W.column_ensemble(n_scenarios=4, seed=5, n_min=2_000, n_max=20_000, steps=10)
    a = mpm.Simulation.from_workload(ens, flags=mpm.DETERMINISTIC | SCAN)
    b = mpm.Simulation.from_workload(ens, flags=mpm.DETERMINISTIC)
    a.step(ens.steps)
    b.step(ens.steps)
    for k, v in _bits(a).items():
        assert np.array_equal(v, _bits(b)[k]), k
    a.rebuild_active()
    b.rebuild_active()
    assert np.array_equal(a.read_active(), b.read_active())


def test_scan_rejects_dense(oracle_mod):
    wl, Cm, F = small_blob(n=100)
    with pytest.raises(mpm.MpmError) as e:
        mpm.Simulation(mpm.config_from_workload(wl, flags=SCAN | mpm.DENSE_GRID), wl.x, wl.v, Cm, F)
    assert e.value.status == mpm.ERR_INVALID_ARG
