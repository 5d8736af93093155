"""FP64 dense-grid CPU oracle of the explicit MPM step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2605_28525_b300``) and never imports it.  The arithmetic lives in
``mpm_oracle.c`` (plain C, FP64, serial, dense grid); this module only builds
that file with gcc and marshals numpy arrays through ctypes.

Paper sections followed (Zhao et al., "Unified sparse framework for large-scale
simulations using the material point method"):
  * Sec. 4.1 -- B-spline transfer, APIC P2G, forces, explicit Euler, G2P.
  * Sec. 4.2, Alg. 2-4 -- dense block mask, serial exclusive scan, compact map.

Parity status per function (what pins each one, see ``tests/test_oracle_*.py``):
  weights / D_p             -- pinned (box * hat convolution definition of the
                               quadratic B-spline, partition of unity, linear
                               reproduction, closed-form D_p, grad identities)
  active_blocks             -- pinned (brute-force set enumeration, hand cases)
  p2g                       -- pinned (exact mass / momentum / APIC angular
                               momentum conservation, zero net force and torque,
                               stress virial sum f x^T = -sum V0 tau)
  grid_update               -- pinned (free-fall closed form, Coulomb sliding
                               block closed form, hand-worked BC cases)
  g2p                       -- pinned (rigid translation, free fall, affine field
                               with F0 != I)
  kirchhoff (NH, Hencky)    -- pinned (derivative of the stored energy, zero for
                               rigid motion, linear-elastic limit, objectivity)
  dp_project                -- pinned (Mohr-Coulomb triaxial-compression match,
                               tip, volume kept, alpha = 0 limit, objectivity)
  svd3                      -- pinned (numpy.linalg.svd on random matrices)
A mutation test plants ten plausible mistakes in copies of the C file and
requires every one of them to fail a pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_HDR = os.path.join(_HERE, "mpm_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libmpm_oracle.so")
# A planted-mistake copy of the oracle can be loaded instead (used only by the
# mutation test that proves the pins catch such mistakes).
_OVERRIDE = os.environ.get("MPM_ORACLE_LIB")

NEOHOOKEAN, DRUCKER_PRAGER = 0, 1
FLOOR_NONE, FLOOR_STICKY, FLOOR_SLIP, FLOOR_COULOMB = 0, 1, 2, 3


# The all-core build of the same source (gcc -fopenmp): P2G into per-thread
# grids added in thread order, grid update and G2P split over the threads.  It
# is a timing baseline only; the parity reference is the serial build.
_LIB_OMP = os.path.join(_HERE, "_build", "libmpm_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile mpm_oracle.c into a shared library with gcc (idempotent);
    `openmp` builds the all-core variant beside the serial one."""
    out = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    stale = force or not os.path.exists(out) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(out)
    if stale:
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared"] +
                              (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [
        ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3),
        ("h", C.c_double), ("dt", C.c_double), ("g", C.c_double * 3),
        ("B", C.c_int32), ("material", C.c_int32),
        ("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
        ("phi_deg", C.c_double), ("ppc", C.c_double),
        ("floor_kind", C.c_int32), ("floor_z", C.c_double), ("floor_mu", C.c_double),
        ("terrain", C.POINTER(C.c_double)), ("terrain_nx", C.c_int32), ("terrain_ny", C.c_int32),
        ("terrain_mu", C.c_double),
        ("wall_layers", C.c_int32),
    ]


_libs = {}


def lib(openmp: bool = False):
    """The serial oracle library (the parity reference), or with `openmp` the
    all-core build of the same source."""
    if openmp not in _libs:
        _libs[openmp] = _declare(C.CDLL(build(openmp=True) if openmp else (_OVERRIDE if _OVERRIDE else build())))
    return _libs[openmp]


def _declare(L):
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    P = C.POINTER(Params)
    L.orc_weights.argtypes = [P, dp, ip, dp, dp]
    L.orc_Dp.argtypes = [P, dp, dp]
    L.orc_active_blocks.argtypes = [P, C.c_int64, dp, ip, C.c_int64]
    L.orc_active_blocks.restype = C.c_int64
    L.orc_kirchhoff.argtypes = [P, dp, C.c_double, dp]
    L.orc_dp_project.argtypes = [P, dp, C.c_double, dp, C.POINTER(C.c_int)]
    L.orc_svd3.argtypes = [dp, dp, dp, dp]
    L.orc_p2g.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_p2g_abs.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_p2g_nodes.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, C.c_int64, ip, dp, dp, dp, dp]
    L.orc_grid_update.argtypes = [P, dp, dp, dp, dp]
    L.orc_grid_node.argtypes = [P, ip, C.c_double, dp, dp, dp]
    L.orc_g2p_one.argtypes = [P, dp, C.c_double, dp, dp, dp, dp]
    L.orc_g2p.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp]
    L.orc_run.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, C.c_int32]
    return L


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """Bound parameter set; every method returns fresh numpy arrays."""

    def __init__(self, *, lo, hi, h, dt, g=(0.0, 0.0, -9.81), B=4, material=NEOHOOKEAN,
                 E=1e6, nu=0.3, rho=1000.0, phi_deg=30.0, ppc=8.0,
                 floor_kind=FLOOR_NONE, floor_z=0.0, floor_mu=0.0,
                 terrain=None, terrain_mu=0.0, wall_layers=2, openmp=False):
        self.openmp = bool(openmp)   # the all-core build (timing only)
        self.p = Params()
        self.p.lo[:] = [int(v) for v in lo]
        self.p.hi[:] = [int(v) for v in hi]
        self.p.h, self.p.dt = float(h), float(dt)
        self.p.g[:] = [float(v) for v in g]
        self.p.B, self.p.material = int(B), int(material)
        self.p.E, self.p.nu, self.p.rho = float(E), float(nu), float(rho)
        self.p.phi_deg, self.p.ppc = float(phi_deg), float(ppc)
        self.p.floor_kind, self.p.floor_z, self.p.floor_mu = int(floor_kind), float(floor_z), float(floor_mu)
        self._terrain = None
        if terrain is not None:
            t = np.ascontiguousarray(terrain, dtype=np.float64)  # shape (ny, nx), x fastest
            self._terrain = t
            self.p.terrain = _d(t)
            self.p.terrain_ny, self.p.terrain_nx = t.shape
        self.p.terrain_mu = float(terrain_mu)
        self.p.wall_layers = int(wall_layers)
        self.dims = tuple(int(hi[a]) - int(lo[a]) + 1 for a in range(3))
        self.lo = tuple(int(v) for v in lo)

    @property
    def nnodes(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def node_index(self, n):
        n = np.asarray(n, dtype=np.int64)
        return ((n[..., 0] - self.lo[0]) * self.dims[1] + (n[..., 1] - self.lo[1])) * self.dims[2] + (
            n[..., 2] - self.lo[2])

    def weights(self, x):
        x = _f64(x, (3,))
        nodes = np.zeros((27, 3), np.int32)
        w = np.zeros(27)
        gw = np.zeros((27, 3))
        lib(self.openmp).orc_weights(C.byref(self.p), _d(x), _i(nodes), _d(w), _d(gw))
        return nodes, w, gw

    def Dp(self, x):
        x = _f64(x, (3,))
        D = np.zeros((3, 3))
        lib(self.openmp).orc_Dp(C.byref(self.p), _d(x), _d(D))
        return D

    def active_blocks(self, x):
        x = _f64(x, (-1, 3))
        cap = max(64, 27 * len(x))
        out = np.zeros((cap, 3), np.int32)
        n = lib(self.openmp).orc_active_blocks(C.byref(self.p), len(x), _d(x), _i(out), cap)
        if n < 0:
            raise ValueError("orc_active_blocks failed (%d)" % n)
        return out[:n].copy()

    def kirchhoff(self, F, phi_deg=None):
        F = _f64(F, (3, 3))
        tau = np.zeros((3, 3))
        rc = lib(self.openmp).orc_kirchhoff(C.byref(self.p), _d(F), float(self.p.phi_deg if phi_deg is None else phi_deg),
                                 _d(tau))
        if rc:
            raise ValueError("invalid stress state")
        return tau

    def dp_project(self, F, phi_deg=None):
        F = _f64(F, (3, 3))
        out = np.zeros((3, 3))
        cs = C.c_int(-1)
        rc = lib(self.openmp).orc_dp_project(C.byref(self.p), _d(F), float(self.p.phi_deg if phi_deg is None else phi_deg),
                                  _d(out), C.byref(cs))
        if rc:
            raise ValueError("invalid state")
        return out, cs.value

    @staticmethod
    def svd3(A):
        A = _f64(A, (3, 3))
        U, S, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
        lib().orc_svd3(_d(A), _d(U), _d(S), _d(V))
        return U, S, V

    def _state(self, x, v, C_, F, phi):
        n = len(np.asarray(x).reshape(-1, 3))
        x = _f64(x, (n, 3))
        v = _f64(v if v is not None else np.zeros((n, 3)), (n, 3))
        C_ = _f64(C_ if C_ is not None else np.zeros((n, 3, 3)), (n, 3, 3))
        F = _f64(F if F is not None else np.broadcast_to(np.eye(3), (n, 3, 3)), (n, 3, 3))
        phi = None if phi is None else _f64(phi, (n,))
        return n, x, v, C_, F, phi

    def p2g(self, x, v=None, C_=None, F=None, phi=None):
        n, x, v, C_, F, phi = self._state(x, v, C_, F, phi)
        m = np.zeros(self.nnodes)
        mv = np.zeros((self.nnodes, 3))
        f = np.zeros((self.nnodes, 3))
        rc = lib(self.openmp).orc_p2g(C.byref(self.p), n, _d(x), _d(v), _d(C_), _d(F),
                           _d(phi) if phi is not None else None, _d(m), _d(mv), _d(f))
        if rc:
            raise ValueError("orc_p2g failed (%d)" % rc)
        return m, mv, f

    def p2g_abs(self, x, v=None, C_=None, F=None, phi=None):
        n, x, v, C_, F, phi = self._state(x, v, C_, F, phi)
        am = np.zeros(self.nnodes)
        amv = np.zeros((self.nnodes, 3))
        af = np.zeros((self.nnodes, 3))
        rc = lib(self.openmp).orc_p2g_abs(C.byref(self.p), n, _d(x), _d(v), _d(C_), _d(F),
                               _d(phi) if phi is not None else None, _d(am), _d(amv), _d(af))
        if rc:
            raise ValueError("orc_p2g_abs failed (%d)" % rc)
        return am, amv, af

    def p2g_nodes(self, nodes, x, v=None, C_=None, F=None, phi=None, with_scale=False):
        n, x, v, C_, F, phi = self._state(x, v, C_, F, phi)
        q = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1, 3)
        m = np.zeros(len(q))
        mv = np.zeros((len(q), 3))
        f = np.zeros((len(q), 3))
        af = np.zeros(len(q))
        rc = lib(self.openmp).orc_p2g_nodes(C.byref(self.p), n, _d(x), _d(v), _d(C_), _d(F),
                                 _d(phi) if phi is not None else None, len(q), _i(q), _d(m), _d(mv), _d(f),
                                 _d(af) if with_scale else None)
        if rc:
            raise ValueError("orc_p2g_nodes failed (%d)" % rc)
        return (m, mv, f, af) if with_scale else (m, mv, f)

    def grid_update(self, m, mv, f):
        m = _f64(m, (-1,))
        mv = _f64(mv, (-1, 3))
        f = _f64(f, (-1, 3))
        vn = np.zeros_like(mv)
        lib(self.openmp).orc_grid_update(C.byref(self.p), _d(m), _d(mv), _d(f), _d(vn))
        return vn

    def grid_node(self, n, m, mv, f):
        n = np.ascontiguousarray(n, dtype=np.int32).reshape(3)
        mv = _f64(mv, (3,))
        f = _f64(f, (3,))
        out = np.zeros(3)
        lib(self.openmp).orc_grid_node(C.byref(self.p), _i(n), float(m), _d(mv), _d(f), _d(out))
        return out

    def g2p_one(self, vn27, x, F, phi_deg=None):
        vn27 = _f64(vn27, (27, 3))
        x = _f64(x, (3,)).copy()
        v = np.zeros(3)
        C_ = np.zeros((3, 3))
        F = _f64(F, (3, 3)).copy()
        rc = lib(self.openmp).orc_g2p_one(C.byref(self.p), _d(vn27), float(self.p.phi_deg if phi_deg is None else phi_deg),
                               _d(x), _d(v), _d(C_), _d(F))
        if rc:
            raise ValueError("orc_g2p_one failed (%d)" % rc)
        return x, v, C_, F

    def g2p(self, vn, x, v=None, C_=None, F=None, phi=None):
        n, x, v, C_, F, phi = self._state(x, v, C_, F, phi)
        x, v, C_, F = x.copy(), v.copy(), C_.copy(), F.copy()
        vn = _f64(vn, (-1, 3))
        rc = lib(self.openmp).orc_g2p(C.byref(self.p), n, _d(vn), _d(x), _d(v), _d(C_), _d(F),
                           _d(phi) if phi is not None else None)
        if rc:
            raise ValueError("orc_g2p failed (%d)" % rc)
        return x, v, C_, F

    def run(self, x, v=None, C_=None, F=None, phi=None, nsteps=1):
        n, x, v, C_, F, phi = self._state(x, v, C_, F, phi)
        x, v, C_, F = x.copy(), v.copy(), C_.copy(), F.copy()
        rc = lib(self.openmp).orc_run(C.byref(self.p), n, _d(x), _d(v), _d(C_), _d(F),
                           _d(phi) if phi is not None else None, int(nsteps))
        if rc:
            raise ValueError("orc_run failed (%d)" % rc)
        return x, v, C_, F

    def dense_nodes(self):
        """Node tuples of every dense index, shape (nnodes, 3)."""
        i, j, k = np.meshgrid(*[np.arange(self.lo[a], self.lo[a] + self.dims[a]) for a in range(3)],
                              indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
