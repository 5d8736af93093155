"""Parity at the benchmark sizes, in the launch configuration bench.py times
(fast sparse mode, block size 4, device-resident inputs on the torch stream):
the 1,048,576-particle granular column and the 8,000,000-particle landslide.

The oracle cannot step these sizes whole, so after a few GPU steps (non-trivial
v, C, F) the FP32 state is read back and
  * the active set is compared whole and bit-exact (the oracle's dense block
    mask and serial scan stay cheap at these sizes),
  * P2G is compared on 64 sampled active nodes that the oracle sums one by one
    (orc_p2g_nodes), with the same bars as the small tests,
  * the grid update on the same nodes, from the GPU's own m, mv, f,
  * G2P on 200 sampled particles from the GPU's own grid velocities,
  * total mass is conserved to FP32 accuracy.
"""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import U32, eq_keys, oracle_for, phi_index as _phi_index, sparse_node_coords

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,steps", [("column_collapse_1M", 3), ("column_collapse_1M", 500), ("landslide_8M", 3),
                                        ("landslide_8M", 300)])
def test_full_size_parity(oracle_mod, name, steps):
    """At the start of the run and after some hundred steps of flow, when the
    cells' particle counts have spread (fuller cells, more rounds per P2G work
    unit, more plastic particles)."""
    import torch
    wl = W.column_collapse() if name == "column_collapse_1M" else W.landslide()
    o = oracle_for(wl)
    sim = mpm.Simulation.from_workload(wl, stream=torch.cuda.current_stream(), device_inputs=True)
    sim.step(steps)
    st = sim.read_particles()
    x, v, Cm, F = st["x"], st["v"], st["C"], st["F"]
    phi = wl.phi

    # active set: whole and bit-exact
    sim.rebuild_active()
    keys = sim.read_active()
    assert np.array_equal(keys, eq_keys(o.active_blocks(x)))

    # P2G on sampled nodes
    sim.p2g()
    g = sim.read_grid()
    nodes_all = sparse_node_coords(keys, 4)
    rng = np.random.default_rng(7)
    idx = rng.choice(np.flatnonzero(g["m"] > 0), 64, replace=False)
    nodes = nodes_all[idx]
    m, mv, f, af = o.p2g_nodes(nodes, x, v, Cm, F, phi, with_scale=True)
    assert np.all(np.abs(g["m"][idx] - m) <= 1e-6 * np.abs(g["m"]).max())
    assert np.all(np.abs(g["mv"][idx] - mv) <= 1e-6 * max(np.abs(g["mv"]).max(), 1e-30))
    assert np.all(np.abs(g["f"][idx].astype(np.float64) - f) <= 64 * U32 * af[:, None] + 1e-30)
    mp = wl.rho * wl.dx ** 3 / wl.ppc
    assert abs(g["m"].astype(np.float64).sum() - mp * wl.n) <= 1e-6 * mp * wl.n

    # grid update on the same nodes
    sim.grid_update()
    g = sim.read_grid()
    for q in idx:
        mq = float(g["m"][q])
        want = o.grid_node(nodes_all[q], mq, g["mv"][q].astype(np.float64), g["f"][q].astype(np.float64))
        scale = (np.abs(g["mv"][q]).max() + wl.dt * np.abs(g["f"][q]).max()) / mq + wl.dt * 9.81
        assert np.all(np.abs(g["v"][q] - want) <= 1e-5 * scale + 1e-12)

    # G2P on sampled particles
    sim.g2p()
    out = sim.read_particles()
    vmax = np.abs(g["v"]).max()
    h = wl.dx
    for p in rng.choice(wl.n, 200, replace=False):
        nd, w, gw = o.weights(x[p].astype(np.float64))
        v27 = g["v"][_phi_index(keys, nd)].astype(np.float64)
        x1, v1, C1, F1 = o.g2p_one(v27, x[p], F[p], None if phi is None else float(phi[p]))
        assert np.all(np.abs(out["v"][p] - v1) <= 8 * U32 * vmax + 1e-12)
        assert np.all(np.abs(out["x"][p] - x1) <= 4 * U32 * np.abs(x1).max() + 8 * U32 * wl.dt * vmax)
        assert np.all(np.abs(out["C"][p] - C1) <= 64 * U32 * vmax / h + 1e-9)
        fb = 16 * U32 * (1 + 27 * wl.dt * vmax / h) * np.abs(F[p]).max()
        assert np.all(np.abs(out["F"][p] - F1) <= 64 * fb + 1e-6)
    sim.close()


def test_full_size_ensemble_parity(oracle_mod):
    """The 64-column ensemble (8,242,000 particles) as bench.py runs it: the
    active set of three scenarios against the oracle (shifted keys), P2G on
    sampled nodes and G2P on sampled particles of those scenarios, each from
    that scenario's own oracle."""
    import torch
    ens = W.column_ensemble()
    sim = mpm.Simulation.from_workload(ens, stream=torch.cuda.current_stream(), device_inputs=True)
    sim.step(3)
    st = sim.read_particles()
    sim.rebuild_active()
    keys = sim.read_active()
    sim.p2g()
    g = sim.read_grid()
    nodes_all = sparse_node_coords(keys, 4)
    pitch = (ens.hi[0] // 4) - (ens.lo[0] // 4) + 1
    c = np.concatenate([[0], np.cumsum(ens.scenario_counts)])
    rng = np.random.default_rng(11)
    blocks = mpm.unpack_keys(keys)
    scen_of_block = (blocks[:, 0] - ens.lo[0] // 4) // pitch
    for s in rng.choice(len(ens.scenario_counts), 3, replace=False):
        sl = slice(int(c[s]), int(c[s + 1]))
        m_wl = W.ensemble_member(ens, s)
        o = oracle_for(m_wl)
        x, v, Cm, F = st["x"][sl], st["v"][sl], st["C"][sl], st["F"][sl]
        # the scenario's active blocks, shifted into its slot along x
        want = np.asarray(o.active_blocks(x), np.int64).copy()
        want[:, 0] += s * pitch
        assert np.array_equal(keys[scen_of_block == s], eq_keys(want))
        # P2G on sampled nodes of this scenario (local node = global - s * pitch * 4 along x)
        mine = np.flatnonzero((np.repeat(scen_of_block, 64) == s) & (g["m"] > 0))
        idx = rng.choice(mine, 32, replace=False)
        local = nodes_all[idx].copy()
        local[:, 0] -= s * pitch * 4
        m, mv, f, af = o.p2g_nodes(local, x, v, Cm, F, m_wl.phi, with_scale=True)
        mine_m = g["m"][np.repeat(scen_of_block, 64) == s]
        assert np.all(np.abs(g["m"][idx] - m) <= 1e-6 * np.abs(mine_m).max())
        mine_mv = g["mv"][np.repeat(scen_of_block, 64) == s]
        assert np.all(np.abs(g["mv"][idx] - mv) <= 1e-6 * max(np.abs(mine_mv).max(), 1e-30))
        assert np.all(np.abs(g["f"][idx].astype(np.float64) - f) <= 64 * U32 * af[:, None] + 1e-30)
    sim.close()
