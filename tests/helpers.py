"""Shared helpers of the test-suite (test infrastructure only)."""
import numpy as np

import oracle
from paper_2605_28525_b300 import mpm, workloads as W

U32 = 2.0 ** -24        # unit roundoff of float32


def oracle_for(wl, B=None):
    return oracle.Oracle(lo=wl.lo, hi=wl.hi, h=wl.dx, dt=wl.dt, g=wl.gravity, B=B or wl.block_size,
                         material=wl.material, E=wl.E, nu=wl.nu, rho=wl.rho, phi_deg=wl.phi_deg, ppc=wl.ppc,
                         floor_kind=wl.floor_kind, floor_z=wl.floor_z, floor_mu=wl.floor_mu,
                         terrain=None if wl.terrain is None else wl.terrain.astype(np.float64),
                         terrain_mu=wl.terrain_mu, wall_layers=wl.wall_layers)


def eq_keys(blocks):
    b = np.asarray(blocks, np.int64)
    return ((b[:, 0] + (1 << 20)) << 42 | (b[:, 1] + (1 << 20)) << 21 | (b[:, 2] + (1 << 20))).astype(np.uint64)


def sparse_node_coords(keys, B):
    """Node tuple of every compact node index phi = Phi*B^3 + l, l = x + B(y + B z)."""
    b = mpm.unpack_keys(keys)
    l = np.arange(B ** 3)
    off = np.stack([l % B, (l // B) % B, l // (B * B)], axis=1)
    return (b[:, None, :] * B + off[None, :, :]).reshape(-1, 3)


def normwise(a, b):
    """||a - b||_inf / ||b||_inf over a component family (0 if both vanish)."""
    den = np.abs(b).max()
    num = np.abs(np.asarray(a, np.float64) - b).max()
    if den == 0:
        return 0.0 if num == 0 else np.inf
    return num / den


def make_sim(wl, flags=0, **kw):
    return mpm.Simulation.from_workload(wl, flags=flags, **kw)


def small_blob(n=3000, seed=3, dx=1.0 / 32, lo=10, hi=20, box=32, material=W.NEOHOOKEAN, E=1e5,
               vscale=0.5, cscale=5.0, fscale=0.02, g=(0.0, 0.0, -9.81), dt=1e-4, block_size=4):
    """A random particle cloud with non-trivial v, C, F inside a small box."""
    x, v, Cm, F = W.random_state(n, (lo,) * 3, (hi,) * 3, dx, seed=seed, vscale=vscale, cscale=cscale,
                                 fscale=fscale)
    wl = W.Workload("blob", (0, 0, 0), (box, box, box), dx, dt, g, material, E, 0.3, 1000.0, 30.0, 8.0,
                    W.FLOOR_NONE, 0.0, 0.0, x, v=v, block_size=block_size)
    return wl, Cm, F


def phi_index(keys, nodes):
    """phi index of node tuples given the active block keys (Phi order, B = 4)."""
    kb = eq_keys(np.asarray(nodes) // 4)
    r = np.searchsorted(keys, kb)
    assert np.all(keys[r] == kb)
    nodes = np.asarray(nodes)
    l = (nodes[:, 0] % 4) + 4 * ((nodes[:, 1] % 4) + 4 * (nodes[:, 2] % 4))
    return r * 64 + l
