"""mpm_step queues its steps without host synchronisation (CUDA graphs, or
plain launches with MPM_NO_GRAPHS) and stops on the device at the first
failure.  These tests hold the queued path to the synchronous one
(MPM_SYNC_STEPS: a status read after every insert, the host sizing every
array from the exact block count): in deterministic mode the two give the
same bits, the same status and the same number of completed steps, including
when a step outgrows the capacities (Alg. 7 regrowth inside a batch) and when
the state blows up part-way through a batch."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import eq_keys, oracle_for

pytestmark = pytest.mark.gpu

MODES = [0, mpm.NO_GRAPHS, mpm.SYNC_STEPS]


def _bits(sim):
    p = sim.read_particles()
    return {k: p[k].view(np.uint32).copy() for k in ("x", "v", "C", "F")}


def _same(a, b):
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(a[k], b[k]), k


def _explosion(n=6000, seed=11, s=20.0):
    """A ball of particles whose velocity points away from its centre
    (v = s (x - c)), nearly stress-free (E = 1 Pa): it expands to about three
    times its radius within 100 steps and its active set grows ten-fold."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 0.1 * rng.random(n) ** (1.0 / 3.0)
    c = np.array([0.5, 0.5, 0.5])
    x = (c + d * r[:, None]).astype(np.float32)
    v = (s * (x - c)).astype(np.float32)
    return W.Workload("explosion", (0, 0, 0), (64, 64, 64), 1.0 / 64, 1e-3, (0.0, 0.0, 0.0), W.NEOHOOKEAN, 1.0,
                      0.3, 1000.0, 30.0, 8.0, W.FLOOR_NONE, 0.0, 0.0, x, v=v)


@pytest.mark.parametrize("dense", [False, True])
def test_batch_equals_sync_bitwise(oracle_mod, dense):
    wl = W.elastic_cube(steps=40)
    wl.v = np.tile(np.array([[0.6, -0.4, 0.2]], np.float32), (wl.n, 1))
    base = mpm.DETERMINISTIC | (mpm.DENSE_GRID if dense else 0)
    out = []
    for mode in MODES:
        sim = mpm.Simulation.from_workload(wl, flags=base | mode)
        sim.step(1)
        sim.step(wl.steps - 1)
        out.append(_bits(sim))
        assert sim.stats()["steps"] == wl.steps
    _same(out[0], out[2])
    _same(out[1], out[2])


def test_batch_dp_column_equals_sync(oracle_mod):
    wl = W.column_collapse(cells_xy=8, cells_z=16, steps=30)
    out = []
    for mode in MODES:
        sim = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mode)
        sim.step(wl.steps)
        out.append(_bits(sim))
    _same(out[0], out[2])
    _same(out[1], out[2])


@pytest.mark.parametrize("mode", [0, mpm.NO_GRAPHS])
def test_batch_regrowth_inside_batch(oracle_mod, mode):
    """The active set grows beyond the batch's headroom: the queue stops on the
    device, the host enlarges the capacities and reruns the remaining steps
    from the last completed one; the result is the synchronous one."""
    wl = _explosion()
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mode)
    a.step(1)
    n1 = a.stats()["n_active_blocks"]
    a.step(99)
    sa = a.stats()
    assert sa["steps"] == 100
    assert sa["n_active_blocks"] > 3 * n1 + 64      # grew past the first batch's capacities
    assert sa["rebuild_rounds"] >= 1
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mpm.SYNC_STEPS)
    b.step(100)
    _same(_bits(a), _bits(b))
    # and the active set after the batch is the oracle's for the final positions
    x = a.read_particles()["x"]
    a.rebuild_active()
    assert np.array_equal(a.read_active(), eq_keys(oracle_for(wl).active_blocks(x)))


def test_batch_fast_mode_active_set_and_closeness(oracle_mod):
    wl = _explosion(seed=12)
    a = mpm.Simulation.from_workload(wl)
    a.step(60)
    b = mpm.Simulation.from_workload(wl, flags=mpm.SYNC_STEPS)
    b.step(60)
    xa, xb = a.read_particles()["x"], b.read_particles()["x"]
    assert np.abs(xa - xb).max() <= 1e-5
    a.rebuild_active()
    assert np.array_equal(a.read_active(), eq_keys(oracle_for(wl).active_blocks(xa)))


def _unstable():
    """Neo-Hookean cube at twice the CFL limit (c = sqrt(E/rho) = 316 m/s,
    dx/c = 4.9e-5 s, dt = 1e-4 s) with a slightly perturbed F: the unstable
    modes grow every step until the state fails part-way through a batch."""
    wl = W.elastic_cube(steps=1)
    wl.E = 1e8
    wl.dt = 1e-4
    rng = np.random.default_rng(3)
    F = (np.eye(3)[None] + 1e-4 * rng.standard_normal((wl.n, 3, 3))).astype(np.float32).reshape(-1, 9)
    return wl, F


@pytest.mark.parametrize("mode", [0, mpm.NO_GRAPHS])
def test_batch_stops_where_sync_stops(oracle_mod, mode):
    wl, F = _unstable()
    res = []
    for flags in (mpm.DETERMINISTIC | mpm.SYNC_STEPS, mpm.DETERMINISTIC | mode):
        sim = mpm.Simulation(mpm.config_from_workload(wl, flags=flags), wl.x, wl.v, None, F)
        status = mpm.OK
        if flags & mpm.SYNC_STEPS:
            for _ in range(200):
                try:
                    sim.step(1)
                except mpm.MpmError as e:
                    status = e.status
                    break
        else:
            sim.step(1)
            try:
                sim.step(199)
            except mpm.MpmError as e:
                status = e.status
        res.append((status, sim.stats()["steps"], _bits(sim)))
    (s0, n0, b0), (s1, n1, b1) = res
    assert s0 in (mpm.ERR_NUMERIC, mpm.ERR_OUT_OF_DOMAIN), "the unstable setup did not fail"
    assert 1 < n0 < 200
    assert (s1, n1) == (s0, n0)
    _same(b0, b1)


def test_batch_after_phase_calls(oracle_mod):
    """A partial phase sequence, then mpm_step: the first step runs
    synchronously and the rest queued; same bits as the synchronous loop."""
    wl = W.elastic_cube(steps=12)
    wl.v = np.tile(np.array([[0.2, 0.1, -0.3]], np.float32), (wl.n, 1))
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    a.step(3)
    a.rebuild_active()
    a.p2g()
    a.step(9)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mpm.SYNC_STEPS)
    b.step(12)
    _same(_bits(a), _bits(b))
    assert a.stats()["steps"] == 12


def test_batch_launch_count(oracle_mod):
    """kernel_launches counts the kernels of replayed graphs too."""
    wl = W.elastic_cube(steps=1)
    a = mpm.Simulation.from_workload(wl)
    b = mpm.Simulation.from_workload(wl, flags=mpm.NO_GRAPHS)
    for s in (a, b):
        s.step(1)
    la, lb = a.stats()["kernel_launches"], b.stats()["kernel_launches"]
    for s in (a, b):
        s.step(10)
    assert a.stats()["kernel_launches"] - la == b.stats()["kernel_launches"] - lb > 10 * 10
