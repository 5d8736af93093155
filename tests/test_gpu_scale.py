"""Parity at scale: the 134,189,056-particle granular column (362 x 362 x 128
cells of the 1M column's box; about 40 GB on the device), in the launch
configuration bench.py times (fast sparse mode, device-resident inputs).

The oracle cannot hold this state whole, so after three GPU steps:
  * the active set is compared whole and bit-exact with its definition, the
    union of every particle's stencil blocks, evaluated with plain torch
    operations on the device, one block offset at a time;
  * P2G on 16 sampled active nodes against the oracle, which is given exactly
    the particles within reach of each node (|x/h - node| <= 1.5 per axis;
    the B-spline weight and its slope vanish beyond);
  * G2P on 100 sampled particles from the GPU's own grid velocities;
  * total mass is conserved to FP32 accuracy.
"""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import U32, oracle_for, phi_index, sparse_node_coords

pytestmark = pytest.mark.gpu


def _stencil_blocks(x, h):
    """Eq. (key) of every block that holds a stencil node of some particle,
    ascending: floor(x/h - 1/2) is the base node, its blocks span base / 4 to
    (base + 2) / 4 per axis."""
    import torch
    base = torch.floor(x.double() / h - 0.5).long()
    b0 = torch.div(base, 4, rounding_mode="floor")
    b1 = torch.div(base + 2, 4, rounding_mode="floor")
    del base
    parts = []
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = torch.tensor([dx, dy, dz], device=x.device)
                b = (b0 + d)[((b0 + d) <= b1).all(1)] + (1 << 20)
                parts.append(torch.unique((b[:, 0] << 42) | (b[:, 1] << 21) | b[:, 2]))
                del b
    return torch.unique(torch.cat(parts)).cpu().numpy().astype(np.uint64)


def test_scale_134M_parity(oracle_mod):
    import torch
    wl = W.column_collapse(cells_xy=362)
    n = wl.n
    assert n == 362 * 362 * 128 * 8
    o = oracle_for(wl)
    sim = mpm.Simulation.from_workload(wl, stream=torch.cuda.current_stream(), device_inputs=True)
    wl.x = None   # 1.6 GB of host memory, no longer needed
    sim.step(3)
    dev = torch.device("cuda")
    st = {"x": torch.empty((n, 3), device=dev), "v": torch.empty((n, 3), device=dev),
          "C": torch.empty((n, 3, 3), device=dev), "F": torch.empty((n, 3, 3), device=dev)}
    sim.read_particles(st)
    assert all(bool(torch.isfinite(t).all()) for t in st.values())

    # active set: whole and bit-exact
    sim.rebuild_active()
    keys = sim.read_active()
    assert np.all(keys[1:] > keys[:-1])
    assert np.array_equal(keys, _stencil_blocks(st["x"], wl.dx))

    # P2G on sampled nodes, from the particles that reach them
    sim.p2g()
    g = sim.read_grid()
    mp = wl.rho * wl.dx ** 3 / wl.ppc
    assert abs(g["m"].astype(np.float64).sum() - mp * n) <= 1e-6 * mp * n
    nodes_all = sparse_node_coords(keys, 4)
    rng = np.random.default_rng(11)
    fx = st["x"].double() / wl.dx
    for q in rng.choice(np.flatnonzero(g["m"] > 0), 16, replace=False):
        node = nodes_all[q]
        near = torch.nonzero(((fx - torch.tensor(node, device=dev, dtype=torch.float64)).abs() <= 1.5).all(1))[:, 0]
        sub = {k: t[near].cpu().numpy() for k, t in st.items()}
        m, mv, f, af = o.p2g_nodes(node[None], sub["x"], sub["v"], sub["C"], sub["F"], None, with_scale=True)
        assert abs(g["m"][q] - m[0]) <= 1e-6 * np.abs(g["m"]).max()
        assert np.all(np.abs(g["mv"][q] - mv[0]) <= 1e-6 * max(np.abs(g["mv"]).max(), 1e-30))
        assert np.all(np.abs(g["f"][q].astype(np.float64) - f[0]) <= 64 * U32 * af[0] + 1e-30)
    del fx

    # G2P on sampled particles
    sim.grid_update()
    g = sim.read_grid()
    sim.g2p()
    out = {k: torch.empty_like(t) for k, t in st.items()}
    sim.read_particles(out)
    vmax = np.abs(g["v"]).max()
    h = wl.dx
    ps = rng.choice(n, 100, replace=False)
    x0, F0 = st["x"][ps].cpu().numpy(), st["F"][ps].cpu().numpy()
    got = {k: t[ps].cpu().numpy() for k, t in out.items()}
    for i in range(len(ps)):
        nd, w, gw = o.weights(x0[i].astype(np.float64))
        v27 = g["v"][phi_index(keys, nd)].astype(np.float64)
        x1, v1, C1, F1 = o.g2p_one(v27, x0[i], F0[i], None)
        assert np.all(np.abs(got["v"][i] - v1) <= 8 * U32 * vmax + 1e-12)
        assert np.all(np.abs(got["x"][i] - x1) <= 4 * U32 * np.abs(x1).max() + 8 * U32 * wl.dt * vmax)
        assert np.all(np.abs(got["C"][i] - C1) <= 64 * U32 * vmax / h + 1e-9)
        fb = 16 * U32 * (1 + 27 * wl.dt * vmax / h) * np.abs(F0[i]).max()
        assert np.all(np.abs(got["F"][i] - F1) <= 64 * fb + 1e-6)
    sim.close()
