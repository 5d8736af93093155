"""Host-side pieces that need no GPU: workload generators, key packing helpers
and the bench's reporting helpers."""
import math

import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W


def test_elastic_cube_shape():
    wl = W.elastic_cube()
    assert wl.n == 16 ** 3 * 8 == 32768 and wl.x.dtype == np.float32
    c = np.floor(wl.x / np.float32(wl.dx)).astype(int)
    assert c.min() == 24 and c.max() == 39
    counts = np.unique(c[:, 0] * 4096 + c[:, 1] * 64 + c[:, 2], return_counts=True)[1]
    assert np.all(counts == 8)                                   # 8 particles per cell


def test_column_collapse_counts():
    assert W.column_collapse().n == 1_048_576
    assert W.column_collapse(cells_xy=64).n == 4_194_304
    wl = W.column_collapse()
    z = wl.x[:, 2] / wl.dx
    assert z.min() >= 3.0 and z.max() <= 131.0 and abs(wl.x[:, 0].mean() - 2.0) < 1e-3


def test_landslide_small_is_above_terrain_and_seeded():
    a = W.landslide(release_cells=(20, 16, 4), grid=(128, 64, 96), release_x0=10)
    b = W.landslide(release_cells=(20, 16, 4), grid=(128, 64, 96), release_x0=10)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.phi, b.phi)
    assert a.n == 20 * 16 * 4 * 8
    assert 25.0 <= a.phi.min() and a.phi.max() <= 35.0
    i = np.floor(a.x[:, 0] / a.dx).astype(int)
    j = np.floor(a.x[:, 1] / a.dx).astype(int)
    hmax = np.maximum.reduce([a.terrain[j, i], a.terrain[j + 1, i], a.terrain[j, i + 1], a.terrain[j + 1, i + 1]])
    assert np.all(a.x[:, 2] > hmax)
    g = np.array(a.gravity)
    assert abs(np.linalg.norm(g) - 9.81) < 1e-9 and abs(math.degrees(math.atan2(g[0], -g[2])) - 35.0) < 1e-9


def test_fbm_statistics():
    H = W.fbm_heightmap(257, 129, seed=1)
    assert abs(H.mean() - 8.0) < 1e-3 and abs(H.std() - 4.0) < 1e-3
    assert np.array_equal(H, W.fbm_heightmap(257, 129, seed=1))
    assert not np.array_equal(H, W.fbm_heightmap(257, 129, seed=2))


def test_unpack_keys_roundtrip():
    rng = np.random.default_rng(0)
    b = rng.integers(-(1 << 20), (1 << 20) - 1, size=(1000, 3))
    keys = ((b[:, 0] + (1 << 20)) << 42 | (b[:, 1] + (1 << 20)) << 21 | (b[:, 2] + (1 << 20))).astype(np.uint64)
    assert np.array_equal(mpm.unpack_keys(keys), b)


def test_bench_traffic_lookup_and_clock_summary(tmp_path):
    import bench
    assert bench.measured_traffic("no_such_workload", "p2g") is None
    s = bench.ClockSampler(0)
    s.source = "nvidia-smi"
    s.rows = bench.ClockSampler.parse_smi(["1900, 2032, 700.5, Not Active, Not Active, Not Active, Active",
                                           "1950, 2032, 710.0, Not Active, Not Active, Not Active, Not Active",
                                           "garbage line"])
    out = s.summary()
    assert out["sm_mhz"] == 1925.0 and out["sm_max_mhz"] == 2032.0 and out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 2 and abs(out["power_w_median"] - 705.25) < 1e-9


def test_binding_rejects_arrays_of_the_wrong_size():
    """Every array crossing the boundary holds exactly n x k float32 values:
    anything else is refused in the binding, before the library could read or
    write past the buffer."""
    from paper_2605_28525_b300 import mpm
    n = 10
    ok = mpm.check_array(np.zeros((n, 3), np.float64), n, 3, "x")
    assert ok.dtype == np.float32 and ok.flags.c_contiguous and ok.shape == (n, 3)
    assert mpm.check_array(np.zeros((n, 3, 3)), n, 9, "F").size == n * 9
    assert mpm.check_array(None, n, 3, "v") is None
    for bad, k in ((np.zeros((n - 1, 3)), 3), (np.zeros((n, 2)), 3), (np.zeros(n * 3 + 1), 3), (np.zeros((n, 3, 2)), 9)):
        with pytest.raises(ValueError):
            mpm.check_array(bad, n, k, "a")
    # outputs are written in place: no silent conversion
    with pytest.raises(ValueError):
        mpm.check_array(np.zeros((n, 3), np.float64), n, 3, "x", output=True)
    with pytest.raises(ValueError):
        mpm.check_array(np.zeros((3, n), np.float32).T, n, 3, "x", output=True)
    ro = np.zeros((n, 3), np.float32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        mpm.check_array(ro, n, 3, "x", output=True)
    assert mpm.check_array(np.zeros((n, 3), np.float32), n, 3, "x", output=True) is not None


def test_binding_rejects_bad_inputs_before_creating_a_context():
    from paper_2605_28525_b300 import mpm, workloads as W
    wl = W.elastic_cube(steps=1)
    cfg = mpm.config_from_workload(wl)
    with pytest.raises(ValueError):
        mpm.Simulation(cfg, wl.x, v=wl.v[:-1] if wl.v is not None else np.zeros((wl.n - 1, 3), np.float32))
    with pytest.raises(ValueError):
        mpm.Simulation(cfg, wl.x, F=np.zeros((wl.n, 4), np.float32))
    with pytest.raises(ValueError):
        mpm.Simulation(cfg, wl.x, phi=np.zeros(wl.n + 1, np.float32))
    with pytest.raises(ValueError):
        mpm.Simulation(cfg, wl.x, terrain=np.zeros(7, np.float32))


def test_openmp_oracle_build_matches_serial(oracle_mod):
    """The all-core build of the oracle (the bench's all-core CPU baseline)
    computes the serial oracle's trajectory up to FP64 summation order."""
    import numpy as np
    from paper_2605_28525_b300 import workloads as W
    x, v, Cm, F = W.random_state(3000, (10,) * 3, (22,) * 3, 1.0 / 32, seed=9, fscale=0.02)
    kw = dict(lo=(0, 0, 0), hi=(32, 32, 32), h=1.0 / 32, dt=1e-4, B=4, material=oracle_mod.DRUCKER_PRAGER, E=1e6,
              phi_deg=30.0, floor_kind=oracle_mod.FLOOR_COULOMB, floor_z=11.0 / 32, floor_mu=0.4)
    a = oracle_mod.Oracle(**kw).run(x, v, Cm, F, nsteps=3)
    b = oracle_mod.Oracle(openmp=True, **kw).run(x, v, Cm, F, nsteps=3)
    for u, w in zip(a, b):
        assert np.abs(u - w).max() <= 1e-12 * np.abs(u).max()
