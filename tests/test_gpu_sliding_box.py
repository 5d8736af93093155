"""The paper's Coulomb sliding box (Sec. 2.2.1) as a GPU workload: an elastic
block on a frictional floor under gravity tilted by theta, mu = tan 15 deg.
For tan(theta) > mu the block slides with constant acceleration
g (sin theta - mu cos theta); at 14 deg it sticks.  The GPU path is checked
against that closed form (the same bars as the oracle's pin), against the
FP64 oracle's trajectory, and sparse against dense bit for bit."""
import json
import math
import os

import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import oracle_for

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
MU = math.tan(math.radians(15.0))


def _acc(theta):
    return 9.81 * (math.sin(math.radians(theta)) - MU * math.cos(math.radians(theta)))


@pytest.mark.parametrize("theta", GOLDEN["sliding_box_angles_deg"]["value"])
def test_sliding_box_closed_form(oracle_mod, theta):
    wl = W.sliding_block(theta, mu=MU, E=1e7, dt=6e-5, steps=2000)
    sim = mpm.Simulation.from_workload(wl)
    x0 = wl.x.astype(np.float64)
    half = wl.steps // 2
    sim.step(half)
    v1 = sim.read_particles()["v"].astype(np.float64)
    sim.step(wl.steps - half)
    out = sim.read_particles()
    t = wl.steps * wl.dt
    s_num = (out["x"][:, 0] - x0[:, 0]).mean()
    if theta == GOLDEN["sliding_box_sticks_deg"]["value"]:
        assert _acc(theta) < 0
        assert abs(out["v"][:, 0].mean() - v1[:, 0].mean()) < 0.05 * _acc(20) * t / 2
        assert abs(s_num) < 0.15 * 0.5 * _acc(20) * t * t
    else:
        s_ana = 0.5 * _acc(theta) * t * t
        assert abs(s_num - s_ana) < 0.06 * s_ana, (s_num, s_ana)
        assert abs(out["v"][:, 0].mean() - _acc(theta) * t) < 0.04 * _acc(theta) * t


def test_sliding_box_matches_oracle_trajectory(oracle_mod):
    """500 steps at 25 deg: FP32 GPU positions within 1e-4 of the 2 m box
    length of the FP64 oracle's."""
    wl = W.sliding_block(25.0, mu=MU, E=1e7, dt=6e-5, steps=500)
    sim = mpm.Simulation.from_workload(wl)
    sim.step(wl.steps)
    got = sim.read_particles()["x"]
    x, v, Cm, F = oracle_for(wl).run(wl.x.astype(np.float64), nsteps=wl.steps)
    L = (wl.hi[0] - wl.lo[0]) * wl.dx
    assert np.abs(got - x).max() <= 1e-4 * L


def test_sliding_box_sparse_equals_dense(oracle_mod):
    wl = W.sliding_block(30.0, mu=MU, E=1e7, dt=6e-5, steps=300)
    a = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC | mpm.DENSE_GRID)
    a.step(wl.steps)
    b.step(wl.steps)
    pa, pb = a.read_particles(), b.read_particles()
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(pa[k].view(np.uint32), pb[k].view(np.uint32)), k
