"""Active set and compact map on the GPU vs the oracle (bit-exact), plus the
overflow / regrowth path of Alg. 5-7 and the error paths of the rebuild."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import eq_keys, make_sim, oracle_for, small_blob

pytestmark = pytest.mark.gpu


def _gpu_keys(sim):
    sim.rebuild_active()
    return sim.read_active()


@pytest.mark.parametrize("B", [1, 4])
@pytest.mark.parametrize("seed", [0, 1])
def test_active_set_bit_exact_random(oracle_mod, B, seed):
    wl, Cm, F = small_blob(n=5000, seed=seed, block_size=B)
    sim = mpm.Simulation(mpm.config_from_workload(wl), wl.x, wl.v, Cm, F)
    got = _gpu_keys(sim)
    want = eq_keys(oracle_for(wl).active_blocks(wl.x))
    assert got.dtype == np.uint64 and np.array_equal(got, want)
    nb, nn = sim.stats()["n_active_blocks"], sim.stats()["n_active_nodes"]
    assert nb == len(want) and nn == len(want) * B ** 3


@pytest.mark.parametrize("B", [1, 4])
def test_active_set_bit_exact_cube(oracle_mod, B):
    wl = W.elastic_cube()
    sim = make_sim(wl, block_size=B)
    got = _gpu_keys(sim)
    want = eq_keys(oracle_for(wl, B=B).active_blocks(wl.x))
    assert np.array_equal(got, want)
    if B == 4:
        assert len(got) == 6 ** 3            # cells 24..39 -> nodes 23..41 -> blocks 5..10


def test_active_set_exact_cell_boundaries(oracle_mod):
    """Particles exactly on cell faces (x/h = k + 1/2) and on nodes."""
    h = 1.0 / 32
    g = np.arange(10, 20, 0.5)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32) * np.float32(h)
    wl = W.Workload("grid_points", (0, 0, 0), (32, 32, 32), h, 1e-4, (0, 0, -9.81), W.NEOHOOKEAN, 1e5, 0.3,
                    1000.0, 30.0, 8.0, W.FLOOR_NONE, 0.0, 0.0, x)
    for B in (1, 4):
        sim = make_sim(wl, block_size=B)
        assert np.array_equal(_gpu_keys(sim), eq_keys(oracle_for(wl, B=B).active_blocks(x)))


def test_single_particle(oracle_mod):
    h = 1.0 / 32
    for xh in ([10.3, 10.3, 10.3], [11.7, 11.7, 11.7], [11.5, 12.0, 13.25]):
        x = (np.array([xh]) * h).astype(np.float32)
        wl = W.Workload("one", (0, 0, 0), (32, 32, 32), h, 1e-4, (0, 0, -9.81), W.NEOHOOKEAN, 1e5, 0.3, 1000.0,
                        30.0, 8.0, W.FLOOR_NONE, 0.0, 0.0, x)
        sim = make_sim(wl)
        assert np.array_equal(_gpu_keys(sim), eq_keys(oracle_for(wl).active_blocks(x)))
        sim.step(3)


def test_active_set_after_motion(oracle_mod):
    """After 40 steps of the elastic cube the set rebuilt from the moved FP32
    positions equals the oracle's set for the same positions."""
    wl = W.elastic_cube()
    wl.v = np.tile(np.array([[0.8, -0.5, 0.3]], np.float32), (wl.n, 1))
    sim = make_sim(wl)
    sim.step(40)
    x = sim.read_particles()["x"]
    assert np.array_equal(_gpu_keys(sim), eq_keys(oracle_for(wl).active_blocks(x)))


def test_dense_mode_lists_every_block(oracle_mod):
    wl, Cm, F = small_blob(n=500)
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=mpm.DENSE_GRID), wl.x, wl.v, Cm, F)
    keys = _gpu_keys(sim)
    b = np.arange(0, 32 // 4 + 1)
    want = eq_keys(np.stack(np.meshgrid(b, b, b, indexing="ij"), -1).reshape(-1, 3))
    assert np.array_equal(keys, want)


# ---------------------------------------------------------- Alg. 7 and errors

@pytest.mark.parametrize("kw", [dict(hash_capacity=16, block_capacity=16), dict(max_probe=1),
                                dict(block_capacity=1), dict(hash_capacity=2, block_capacity=1, max_probe=2)])
def test_overflow_regrowth_keeps_exact_set(oracle_mod, kw):
    wl, Cm, F = small_blob(n=4000, seed=5)
    sim = mpm.Simulation(mpm.config_from_workload(wl, **kw), wl.x, wl.v, Cm, F)
    got = _gpu_keys(sim)
    assert np.array_equal(got, eq_keys(oracle_for(wl).active_blocks(wl.x)))
    st = sim.stats()
    if kw.get("max_probe") != 1:
        assert st["rebuild_rounds"] >= 1
    assert st["hash_capacity"] >= len(got)
    sim.step(2)


def test_overflow_cap_reports_error(oracle_mod):
    wl, Cm, F = small_blob(n=4000, seed=6)
    sim = mpm.Simulation(mpm.config_from_workload(wl, hash_capacity=4, block_capacity=4, max_rebuilds=1),
                         wl.x, wl.v, Cm, F)
    with pytest.raises(mpm.MpmError) as e:
        sim.rebuild_active()
    assert e.value.status == mpm.ERR_HASH_OVERFLOW


def test_out_of_domain_is_reported(oracle_mod):
    wl, Cm, F = small_blob(n=100)
    x = wl.x.copy()
    x[7] = np.float32(0.2 / 32)            # stencil base would be -1
    sim = mpm.Simulation(mpm.config_from_workload(wl), x, wl.v, Cm, F)
    with pytest.raises(mpm.MpmError) as e:
        sim.rebuild_active()
    assert e.value.status == mpm.ERR_OUT_OF_DOMAIN


def test_nonfinite_position_is_reported(oracle_mod):
    wl, Cm, F = small_blob(n=100)
    x = wl.x.copy()
    x[3, 1] = np.nan
    sim = mpm.Simulation(mpm.config_from_workload(wl), x, wl.v, Cm, F)
    with pytest.raises(mpm.MpmError) as e:
        sim.step(1)
    assert e.value.status == mpm.ERR_NUMERIC


def test_phase_order_is_enforced(oracle_mod):
    wl, Cm, F = small_blob(n=100)
    sim = mpm.Simulation(mpm.config_from_workload(wl), wl.x, wl.v, Cm, F)
    with pytest.raises(mpm.MpmError) as e:
        sim.p2g()
    assert e.value.status == mpm.ERR_STATE
    sim.rebuild_active()
    with pytest.raises(mpm.MpmError):
        sim.g2p()
    sim.p2g()
    sim.grid_update()
    sim.g2p()


@pytest.mark.parametrize("B", [1, 4])
@pytest.mark.parametrize("flags", [0, mpm.SCAN_COMPACTION])
def test_negative_coordinates_and_box_edges(oracle_mod, B, flags):
    """A box with negative node indices (Eq. (key)'s bias b in use) and
    particles whose stencils touch the first and the last node of the box on
    every axis: bit-exact active set, then P2G against the oracle."""
    dx = 1.0 / 16
    lo, hi = (-40, -9, -23), (7, 30, 2)
    rng = np.random.default_rng(17)
    n = 3000
    x = np.empty((n, 3), np.float32)
    for a in range(3):
        # stencil base in [lo, hi - 2]: x/h in [lo + 0.5, hi - 0.5)
        x[:, a] = ((lo[a] + 0.5) + rng.random(n) * (hi[a] - lo[a] - 1.0 - 1e-3)) * dx
    # extremes on every axis
    for a in range(3):
        x[a, a] = np.float32((lo[a] + 0.5) * dx)
        x[3 + a, a] = np.float32((hi[a] - 0.5 - 1e-3) * dx)
    wl = W.Workload("edges", lo, hi, dx, 1e-4, (0.0, 0.0, -9.81), W.NEOHOOKEAN, 1e4, 0.3, 1000.0, 30.0, 8.0,
                    W.FLOOR_NONE, 0.0, 0.0, x, block_size=B, wall_layers=0)
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=flags), x)
    keys = _gpu_keys(sim)
    o = oracle_for(wl)
    assert np.array_equal(keys, eq_keys(o.active_blocks(x)))
    b = mpm.unpack_keys(keys)
    assert b.min(0).tolist() == [lo[a] // B for a in range(3)]
    assert b.max(0).tolist() == [hi[a] // B for a in range(3)]
    sim.p2g()
    g = sim.read_grid()
    m, mv, f = o.p2g(x)
    from tests.helpers import sparse_node_coords
    nodes = sparse_node_coords(keys, B)
    ok = np.all((nodes >= np.array(lo)) & (nodes <= np.array(hi)), axis=1)   # blocks overhang the box
    idx = o.node_index(nodes[ok])
    assert np.abs(g["m"][ok] - m[idx]).max() <= 1e-6 * np.abs(m).max()
    assert np.abs(g["mv"][ok] - mv[idx]).max() <= 1e-6 * np.abs(mv).max()
    assert np.all(g["m"][~ok] == 0)


@pytest.mark.parametrize("B", [1, 4])
@pytest.mark.parametrize("flags", [0, mpm.SCAN_COMPACTION])
def test_key_range_extremes(oracle_mod, B, flags):
    """Eq. (key) packs a node or block index i as i + 2^20 in 21 bits, so the
    valid range is [-2^20, 2^20 - 1].  A box in the corner at the top of that
    range in x and at the bottom in y (h = 1): the active set is bit-exact and
    P2G matches the oracle.  Positions lie on a 1/8 grid, which float32
    represents exactly at this magnitude (24 significant bits)."""
    top, bottom = (1 << 20) - 1, -(1 << 20)
    lo, hi = (top - 40, bottom, -12), (top, bottom + 30, 17)
    rng = np.random.default_rng(23)
    n = 2000
    x = np.empty((n, 3), np.float64)
    for a in range(3):
        # stencil base in [lo, hi - 2]: x/h in [lo + 0.5, hi - 0.5)
        x[:, a] = lo[a] + 0.5 + rng.integers(0, int((hi[a] - lo[a] - 1) * 8), n) / 8.0
    for a in range(3):   # the first and the last stencil base on every axis
        x[a, a] = lo[a] + 0.5
        x[3 + a, a] = hi[a] - 0.5 - 0.125
    x32 = x.astype(np.float32)
    assert np.array_equal(x32.astype(np.float64), x)
    wl = W.Workload("key_range", lo, hi, 1.0, 1e-4, (0.0, 0.0, -9.81), W.NEOHOOKEAN, 1e4, 0.3, 1000.0, 30.0, 8.0,
                    W.FLOOR_NONE, 0.0, 0.0, x32, block_size=B, wall_layers=0)
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=flags), x32)
    keys = _gpu_keys(sim)
    o = oracle_for(wl)
    assert np.array_equal(keys, eq_keys(o.active_blocks(x32)))
    b = mpm.unpack_keys(keys)
    assert b.min(0).tolist() == [lo[a] // B for a in range(3)]
    assert b.max(0).tolist() == [hi[a] // B for a in range(3)]
    sim.p2g()
    g = sim.read_grid()
    m, mv, f = o.p2g(x32)
    from tests.helpers import sparse_node_coords
    nodes = sparse_node_coords(keys, B)
    ok = np.all((nodes >= np.array(lo)) & (nodes <= np.array(hi)), axis=1)
    idx = o.node_index(nodes[ok])
    assert np.abs(g["m"][ok] - m[idx]).max() <= 1e-6 * np.abs(m).max()
    assert np.abs(g["mv"][ok] - mv[idx]).max() <= 1e-6 * np.abs(mv).max()
    assert np.all(g["m"][~ok] == 0)
