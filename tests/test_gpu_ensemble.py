"""Ensembles: independent scenarios in one context (mpm_create_ensemble),
every launch covering all of them.  Each scenario is held to the same
scenario run alone: bit for bit in deterministic mode (queued steps, graphs
or plain launches), closely in the fast mode, and its active blocks are the
oracle's for that scenario's particles, shifted by the scenario's offset."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import eq_keys, oracle_for

pytestmark = pytest.mark.gpu


def _small_ensemble():
    return W.column_ensemble(n_scenarios=5, seed=9, n_min=2_000, n_max=40_000, steps=40)


def _slices(ens):
    c = np.concatenate([[0], np.cumsum(ens.scenario_counts)])
    return [slice(int(c[s]), int(c[s + 1])) for s in range(len(ens.scenario_counts))]


@pytest.mark.parametrize("mode", [0, mpm.NO_GRAPHS])
def test_ensemble_equals_single_runs_bitwise(oracle_mod, mode):
    ens = _small_ensemble()
    e = mpm.Simulation.from_workload(ens, flags=mpm.DETERMINISTIC | mode)
    assert e.stats()["n_scenarios"] == 5
    e.step(1)
    e.step(ens.steps - 1)
    got = e.read_particles()
    for s, sl in enumerate(_slices(ens)):
        m = W.ensemble_member(ens, s)
        one = mpm.Simulation.from_workload(m, flags=mpm.DETERMINISTIC)
        one.step(ens.steps)
        want = one.read_particles()
        for k in ("x", "v", "C", "F"):
            assert np.array_equal(got[k][sl].view(np.uint32), want[k].view(np.uint32)), (s, k)
        one.close()


def test_ensemble_fast_mode_close_to_single_runs(oracle_mod):
    ens = _small_ensemble()
    e = mpm.Simulation.from_workload(ens)
    e.step(ens.steps)
    got = e.read_particles()["x"]
    for s, sl in enumerate(_slices(ens)):
        one = mpm.Simulation.from_workload(W.ensemble_member(ens, s))
        one.step(ens.steps)
        assert np.abs(got[sl] - one.read_particles()["x"]).max() <= 1e-5
        one.close()


def test_ensemble_active_set_is_the_shifted_union(oracle_mod):
    ens = _small_ensemble()
    e = mpm.Simulation.from_workload(ens)
    e.step(3)
    x = e.read_particles()["x"]
    e.rebuild_active()
    got = e.read_active()
    pitch = (ens.hi[0] // 4) - (ens.lo[0] // 4) + 1          # blocks of one box along x
    want = []
    for s, sl in enumerate(_slices(ens)):
        b = oracle_for(W.ensemble_member(ens, s)).active_blocks(x[sl].astype(np.float64))
        b = np.asarray(b, np.int64).copy()
        b[:, 0] += s * pitch
        want.append(eq_keys(b))
    want = np.sort(np.concatenate(want))
    assert np.array_equal(got, want)


def test_ensemble_rejects_bad_arguments(oracle_mod):
    ens = _small_ensemble()
    cfg = mpm.config_from_workload(ens, flags=mpm.DENSE_GRID)
    with pytest.raises(mpm.MpmError) as e:
        mpm.Simulation(cfg, ens.x, scenario_counts=ens.scenario_counts)
    assert e.value.status == mpm.ERR_INVALID_ARG
    cfg = mpm.config_from_workload(ens)
    bad = ens.scenario_counts.copy()
    bad[1] = 0
    bad[0] += ens.scenario_counts[1]
    with pytest.raises(mpm.MpmError) as e:
        mpm.Simulation(cfg, ens.x, scenario_counts=bad)
    assert e.value.status == mpm.ERR_INVALID_ARG
    # 5,000 boxes of 65 blocks side by side leave the 2^20 node range of Eq. (key)
    n = 5000
    x = np.tile(ens.x[:1], (n, 1))
    with pytest.raises(mpm.MpmError) as e:
        mpm.Simulation(cfg, x, scenario_counts=np.ones(n, np.int64))
    assert e.value.status == mpm.ERR_INVALID_ARG
