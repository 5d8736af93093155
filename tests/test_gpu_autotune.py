"""mpm_autotune / mpm_set_tuning: launch shapes change timing, never results."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W

pytestmark = pytest.mark.gpu


def _bits(sim):
    p = sim.read_particles()
    return {k: p[k].view(np.uint32).copy() for k in ("x", "v", "C", "F")}


def test_autotune_keeps_state_and_results(oracle_mod):
    wl = W.column_collapse(cells_xy=16, cells_z=32, steps=12)
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    a.step(2)
    b.step(2)
    before = _bits(a)
    t = a.autotune(repeats=3)
    assert 1 <= t["p2g_ctas_per_sm"] <= 4 and t["g2p_threads"] in (128, 256) and (t["g2p_threads"], t["g2p_regs"]) in ((128, 72), (128, 80), (128, 96), (128, 128), (256, 80), (256, 128))
    assert t["p2g_ms"] > 0 and t["g2p_ms"] > 0
    assert a.tuning()["g2p_threads"] == t["g2p_threads"]
    after = _bits(a)
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert a.stats()["steps"] == 2
    a.step(10)
    b.step(10)
    for k, v in _bits(a).items():
        assert np.array_equal(v, _bits(b)[k]), k


@pytest.mark.parametrize("shape", [(1, 128, 128), (2, 256, 128), (3, 128, 80), (4, 256, 80), (4, 128, 72), (2, 128, 96)])
def test_every_shape_gives_the_same_bits(oracle_mod, shape):
    wl = W.elastic_cube(steps=8)
    wl.v = np.tile(np.array([[0.4, -0.2, 0.1]], np.float32), (wl.n, 1))
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    a.set_tuning(*shape)
    a.step(wl.steps)
    b.step(wl.steps)
    for k, v in _bits(a).items():
        assert np.array_equal(v, _bits(b)[k]), k


def test_set_tuning_rejects_out_of_range(oracle_mod):
    wl = W.elastic_cube(steps=1)
    a = mpm.Simulation.from_workload(wl)
    for bad in [(0, 128, 80), (9, 128, 80), (4, 512, 80), (4, 128, 64), (4, 256, 72), (4, 256, 96)]:
        with pytest.raises(mpm.MpmError) as e:
            a.set_tuning(*bad)
        assert e.value.status == mpm.ERR_INVALID_ARG
