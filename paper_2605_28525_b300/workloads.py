"""Seeded synthetic inputs shaped like the paper's workloads.

This module only places particles and builds height maps; it holds none of the
MPM arithmetic and is shared as *data* by the CUDA path and by the CPU oracle.
It imports numpy only (never the native library), so the oracle-side tests can
use it without touching CUDA.

Workloads (paper Sec. 2.2 examples; exact sizes in the design notes):
  * ``elastic_cube``      -- 16^3-cell Neo-Hookean cube at 8 particles/cell in a
                             64^3 box, dx = 1/64 (32,768 particles).
  * ``column_collapse``   -- granular column (Drucker-Prager, phi = 30 deg) on a
                             Coulomb floor in a 512x512x256 box, dx = 1/128;
                             32x32x128 cells (1,048,576 particles) or 64x64x128
                             cells (4,194,304 particles).
  * ``landslide``         -- fBm terrain (6 octaves, Hurst 0.7) in a slope-aligned
                             frame, 2048x1024x256 box, dx = 0.5 m, 250x250x16-cell
                             release (8,000,000 particles), per-particle phi in
                             [25, 35] deg.
  * ``sliding_block``     -- elastic block on a Coulomb floor with tilted gravity
                             (the paper's sliding-box benchmark, Sec. 2.2.1).
  * ``diff_column``       -- the differentiable column: a 32^3-cell
                             Drucker-Prager cube (262,144 particles, phi = 30
                             deg, E = 5e6 Pa) in a 128x128x64 box at dx = 1/32,
                             400 steps of 2e-4 s (dx coarser than the column
                             collapse so that 400 steps see the collapse start).
  * ``column_ensemble``   -- independent granular columns, one per scenario,
                             each in its own 256x256x128 box at dx = 1/128:
                             particle counts log-uniform in [1e4, 5e5], phi
                             uniform in [20, 40] deg, height/width uniform in
                             [0.5, 4].
Particles are placed 2x2x2 per cell, each uniformly jittered inside its
sub-cell, from a numpy PCG64 stream with the stated seed.  Positions are
rounded to float32 once, here, so every consumer sees identical values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

NEOHOOKEAN, DRUCKER_PRAGER = 0, 1
FLOOR_NONE, FLOOR_STICKY, FLOOR_SLIP, FLOOR_COULOMB = 0, 1, 2, 3


@dataclasses.dataclass
class Workload:
    name: str
    lo: tuple
    hi: tuple
    dx: float
    dt: float
    gravity: tuple
    material: int
    E: float
    nu: float
    rho: float
    phi_deg: float
    ppc: float
    floor_kind: int
    floor_z: float
    floor_mu: float
    x: np.ndarray                       # (n, 3) float32
    v: Optional[np.ndarray] = None      # (n, 3) float32 or None (rest)
    phi: Optional[np.ndarray] = None    # (n,) float32 degrees or None
    terrain: Optional[np.ndarray] = None  # (ny, nx) float32 heights at node columns
    terrain_mu: float = 0.0
    steps: int = 1
    block_size: int = 4
    wall_layers: int = 2
    scenario_counts: Optional[np.ndarray] = None   # particles per scenario (ensembles), in order

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def dense_nodes(self) -> int:
        return int(np.prod([self.hi[a] - self.lo[a] + 1 for a in range(3)]))

    def describe(self) -> dict:
        return {"workload": self.name, "particles": self.n,
                "grid": "x".join(str(self.hi[a] - self.lo[a]) for a in range(3)),
                "dx": self.dx, "dt": self.dt, "block": self.block_size}


def jittered_cells(cells_lo, cells_hi, dx, seed, ppc_axis=2, z_base=None):
    """Particles 2x2x2 per cell, jittered uniformly inside each sub-cell.

    cells_lo/hi are integer cell bounds [lo, hi) per axis.  When ``z_base`` is
    given (shape (nx, ny) of integer cell offsets), column (i, j) is shifted up
    by z_base[i - lo0, j - lo1] cells.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = [int(cells_hi[a] - cells_lo[a]) for a in range(3)]
    s = ppc_axis
    ci, cj, ck, si, sj, sk = np.meshgrid(np.arange(nc[0]), np.arange(nc[1]), np.arange(nc[2]),
                                         np.arange(s), np.arange(s), np.arange(s), indexing="ij")
    cell = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1).astype(np.float64)
    sub = np.stack([si.ravel(), sj.ravel(), sk.ravel()], axis=1).astype(np.float64)
    if z_base is not None:
        cell[:, 2] += z_base[ci.ravel(), cj.ravel()]
    jit = rng.random(cell.shape)
    pos = (np.asarray(cells_lo, np.float64) + cell + (sub + jit) / s) * dx
    return pos.astype(np.float32)


def elastic_cube(seed: int = 0, steps: int = 200) -> Workload:
    """64^3 box, dx = 1/64, cube of cells [24, 40)^3, NH E = 1e6, rho = 1000."""
    dx = 1.0 / 64.0
    x = jittered_cells((24, 24, 24), (40, 40, 40), dx, seed)
    return Workload("elastic_cube_32k", (0, 0, 0), (64, 64, 64), dx, 1e-4, (0.0, 0.0, -9.81),
                    NEOHOOKEAN, 1e6, 0.3, 1000.0, 0.0, 8.0, FLOOR_STICKY, 3 * dx, 0.0, x, steps=steps)


def column_collapse(cells_xy: int = 32, cells_z: int = 128, seed: int = 0, steps: int = 2000,
                    phi_deg: float = 30.0, box_xy: int = 512) -> Workload:
    """box_xy x box_xy x 256 box (512 by default) at dx = 1/128; DP column
    centred in x and y (at (2, 2) m by default) on a Coulomb floor at z = 3 dx.
    The particles do not depend on box_xy other than by the shift that keeps
    the column centred."""
    dx = 1.0 / 128.0
    c0 = box_xy // 2 - cells_xy // 2
    x = jittered_cells((c0, c0, 3), (c0 + cells_xy, c0 + cells_xy, 3 + cells_z), dx, seed)
    n = x.shape[0]
    return Workload("column_collapse_%dk" % (n // 1024) if n < 1 << 20 else "column_collapse_%dM" % (n >> 20),
                    (0, 0, 0), (box_xy, box_xy, 256), dx, 2e-5, (0.0, 0.0, -9.81),
                    DRUCKER_PRAGER, 1e7, 0.3, 2000.0, phi_deg, 8.0, FLOOR_COULOMB, 3 * dx, 0.5, x,
                    steps=steps)


def fbm_heightmap(nx: int, ny: int, seed: int = 1, octaves: int = 6, hurst: float = 0.7,
                  base_cells: int = 512, rms: float = 4.0, mean: float = 8.0) -> np.ndarray:
    """Fractional Brownian motion relief: sum of bilinear value-noise octaves.

    Octave o has wavelength base_cells / 2^o nodes and amplitude 2^(-hurst o);
    the sum is shifted to zero mean, scaled to the given RMS and offset by
    ``mean``.  Returns (ny, nx) float32, x fastest.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((ny, nx), np.float64)
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    for o in range(octaves):
        wl = base_cells / (2.0 ** o)
        gx = int(math.ceil(nx / wl)) + 2
        gy = int(math.ceil(ny / wl)) + 2
        lattice = rng.standard_normal((gy, gx))
        fx = xs / wl
        fy = ys / wl
        ix = np.floor(fx).astype(np.int64)
        iy = np.floor(fy).astype(np.int64)
        tx = fx - ix
        ty = fy - iy
        a = lattice[np.ix_(iy, ix)]
        b = lattice[np.ix_(iy, ix + 1)]
        c = lattice[np.ix_(iy + 1, ix)]
        d = lattice[np.ix_(iy + 1, ix + 1)]
        layer = (a * (1 - tx)[None, :] + b * tx[None, :]) * (1 - ty)[:, None] + \
                (c * (1 - tx)[None, :] + d * tx[None, :]) * ty[:, None]
        out += (2.0 ** (-hurst * o)) * layer
    out -= out.mean()
    out *= rms / max(out.std(), 1e-30)
    out += mean
    return out.astype(np.float32)


def landslide(seed: int = 0, terrain_seed: int = 1, phi_seed: int = 2, steps: int = 5000,
              release_cells=(250, 250, 16), grid=(2048, 1024, 256), release_x0: int = 100) -> Workload:
    """Slope-aligned frame: x runs down the 35 deg mean slope, gravity is tilted."""
    dx = 0.5
    theta = math.radians(35.0)
    g = (9.81 * math.sin(theta), 0.0, -9.81 * math.cos(theta))
    H = fbm_heightmap(grid[0] + 1, grid[1] + 1, seed=terrain_seed)
    rx, ry, rz = release_cells
    x0 = release_x0
    y0 = grid[1] // 2 - ry // 2
    # release column (i, j) starts one cell above the highest terrain node of that cell
    hmax = np.maximum.reduce([H[y0:y0 + ry, x0:x0 + rx], H[y0 + 1:y0 + ry + 1, x0:x0 + rx],
                              H[y0:y0 + ry, x0 + 1:x0 + rx + 1], H[y0 + 1:y0 + ry + 1, x0 + 1:x0 + rx + 1]])
    zb = (np.ceil(hmax.astype(np.float64) / dx).astype(np.int64) + 1).T  # (rx, ry)
    x = jittered_cells((x0, y0, 0), (x0 + rx, y0 + ry, rz), dx, seed, z_base=zb)
    rng = np.random.Generator(np.random.PCG64(phi_seed))
    phi = rng.uniform(25.0, 35.0, size=x.shape[0]).astype(np.float32)
    return Workload("landslide_8M" if x.shape[0] == 8_000_000 else "landslide_%d" % x.shape[0],
                    (0, 0, 0), grid, dx, 1e-3, g, DRUCKER_PRAGER, 1e7, 0.3, 1800.0, 30.0, 8.0,
                    FLOOR_NONE, 0.0, 0.0, x, phi=phi, terrain=H, terrain_mu=0.5, steps=steps)


def sliding_block(theta_deg: float, mu: float = math.tan(math.radians(15.0)), seed: int = 0,
                  dx: float = 1.0 / 32.0, cells=(8, 4, 4), E: float = 1e6, steps: int = 400,
                  dt: float = 2e-4) -> Workload:
    """Elastic block resting on a Coulomb floor; gravity tilted by theta about y."""
    th = math.radians(theta_deg)
    g = (9.81 * math.sin(th), 0.0, -9.81 * math.cos(th))
    x = jittered_cells((8, 8, 3), (8 + cells[0], 8 + cells[1], 3 + cells[2]), dx, seed)
    return Workload("sliding_block_%g" % theta_deg, (0, 0, 0), (64, 24, 16), dx, dt, g,
                    NEOHOOKEAN, E, 0.3, 1000.0, 0.0, 8.0, FLOOR_COULOMB, 3 * dx, mu, x, steps=steps)


def random_state(n: int, lo_cell, hi_cell, dx: float, seed: int = 3, vscale: float = 0.5,
                 cscale: float = 5.0, fscale: float = 0.02):
    """Non-trivial particle state for transfer parity tests: positions uniform in
    a cell box, velocities, affine matrices and deformation gradients near I."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo_cell, np.float64) * dx
    hi = np.asarray(hi_cell, np.float64) * dx
    x = (lo + rng.random((n, 3)) * (hi - lo)).astype(np.float32)
    v = (vscale * rng.standard_normal((n, 3))).astype(np.float32)
    Cm = (cscale * rng.standard_normal((n, 3, 3))).astype(np.float32)
    F = (np.eye(3)[None] + fscale * rng.standard_normal((n, 3, 3))).astype(np.float32)
    return x, v, Cm, F


def column_ensemble(n_scenarios: int = 64, seed: int = 4, n_min: int = 10_000, n_max: int = 500_000,
                    steps: int = 1000) -> Workload:
    """Independent Drucker-Prager columns, one per scenario, each centred in
    its own 256x256x128-node box (dx = 1/128) on a Coulomb floor at z = 3 dx.
    Per scenario: a particle count drawn log-uniform in [n_min, n_max], phi
    uniform in [20, 40] deg and a height/width ratio uniform in [0.5, 4]; the
    column is w x w x h cells at 8 particles per cell with w^2 h close to
    count / 8.  Positions are in each scenario's own frame, concatenated in
    scenario order; ``scenario_counts`` gives the split."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = 1.0 / 128.0
    xs, phis, counts = [], [], []
    for s in range(n_scenarios):
        n_target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        phi = rng.uniform(20.0, 40.0)
        aspect = rng.uniform(0.5, 4.0)
        w = max(2, int(round((n_target / (8.0 * aspect)) ** (1.0 / 3.0))))
        h = max(2, min(120, int(round(aspect * w))))
        c0 = 128 - w // 2
        x = jittered_cells((c0, c0, 3), (c0 + w, c0 + w, 3 + h), dx, seed * 1000 + s)
        xs.append(x)
        phis.append(np.full(x.shape[0], phi, np.float32))
        counts.append(x.shape[0])
    return Workload("column_ensemble_%d" % n_scenarios, (0, 0, 0), (256, 256, 128), dx, 2e-5, (0.0, 0.0, -9.81),
                    DRUCKER_PRAGER, 1e7, 0.3, 2000.0, 30.0, 8.0, FLOOR_COULOMB, 3 * dx, 0.5,
                    np.concatenate(xs), phi=np.concatenate(phis), steps=steps,
                    scenario_counts=np.asarray(counts, np.int64))


def ensemble_member(ens: Workload, s: int) -> Workload:
    """Scenario s of an ensemble as a stand-alone workload (same box and
    constants, its own particles)."""
    c = np.concatenate([[0], np.cumsum(ens.scenario_counts)])
    a, b = int(c[s]), int(c[s + 1])
    return dataclasses.replace(ens, name="%s[%d]" % (ens.name, s), x=ens.x[a:b],
                               v=None if ens.v is None else ens.v[a:b],
                               phi=None if ens.phi is None else ens.phi[a:b], scenario_counts=None)


def diff_column(cells: int = 32, seed: int = 6, steps: int = 400, phi_deg: float = 30.0, E: float = 5e6,
                dx: float = 1.0 / 32.0, box=(128, 128, 64)) -> Workload:
    """Drucker-Prager column of cells^3 cells at 8 particles per cell, centred
    on a Coulomb floor (mu = 0.5 at z <= 3 dx) in a box of box nodes."""
    c0x, c0y = box[0] // 2 - cells // 2, box[1] // 2 - cells // 2
    x = jittered_cells((c0x, c0y, 3), (c0x + cells, c0y + cells, 3 + cells), dx, seed)
    return Workload("diff_column_%dk" % (x.shape[0] // 1000), (0, 0, 0), tuple(box), dx, 2e-4, (0.0, 0.0, -9.81),
                    DRUCKER_PRAGER, E, 0.3, 2000.0, phi_deg, 8.0, FLOOR_COULOMB, 3 * dx, 0.5, x, steps=steps)
