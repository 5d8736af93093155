"""Python binding of the C-ABI in include/mpm.h (argument marshalling only).

Every step of the MPM path runs in the CUDA kernels of ``libmpm_b300.so``;
this module only fills the config struct, passes pointers (numpy host arrays
or torch CUDA tensors) and turns status codes into exceptions.  There is no
fallback: if the library is missing or a call fails, it raises.

Function names mirror the C entry points: ``mpm_create`` -> ``Simulation``,
``mpm_rebuild_active`` -> ``Simulation.rebuild_active`` and so on.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
# MPM_B300_LIB selects another build of the library (e.g. libmpm_b300_checked.so)
LIB_PATH = os.environ.get("MPM_B300_LIB") or os.path.join(_HERE, "libmpm_b300.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_HASH_OVERFLOW, ERR_OUT_OF_DOMAIN, ERR_NUMERIC, ERR_CUDA, ERR_STATE = range(8)
NEOHOOKEAN, DRUCKER_PRAGER = 0, 1
FLOOR_NONE, FLOOR_STICKY, FLOOR_SLIP, FLOOR_COULOMB = 0, 1, 2, 3
DETERMINISTIC, DENSE_GRID, SYNC_STEPS, NO_GRAPHS, SCAN_COMPACTION = 1, 2, 4, 8, 16

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class MpmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, message))
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("domain_lo", C.c_int32 * 3), ("domain_hi", C.c_int32 * 3),
        ("dx", C.c_double), ("dt", C.c_double), ("gravity", C.c_double * 3),
        ("block_size", C.c_int32), ("material", C.c_int32),
        ("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double), ("phi_deg", C.c_double),
        ("particle_volume", C.c_double),
        ("floor_kind", C.c_int32), ("floor_z", C.c_double), ("floor_mu", C.c_double),
        ("terrain_height", C.POINTER(C.c_float)), ("terrain_nx", C.c_int32), ("terrain_ny", C.c_int32),
        ("terrain_mu", C.c_double),
        ("wall_layers", C.c_int32),
        ("flags", C.c_uint32),
        ("hash_capacity", C.c_int64), ("block_capacity", C.c_int64),
        ("max_probe", C.c_int32), ("max_rebuilds", C.c_int32),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n_particles", C.c_int64), ("n_active_blocks", C.c_int64), ("n_active_nodes", C.c_int64),
        ("n_particle_blocks", C.c_int64), ("n_dense_nodes", C.c_int64), ("hash_capacity", C.c_int64),
        ("block_capacity", C.c_int64), ("rebuild_rounds", C.c_int64), ("steps", C.c_int64),
        ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64), ("flags", C.c_int32),
        ("block_size", C.c_int32), ("n_scenarios", C.c_int32), ("reserved", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("p2g_ctas_per_sm", C.c_int32), ("g2p_threads", C.c_int32), ("g2p_regs", C.c_int32),
                ("reserved", C.c_int32), ("p2g_ms", C.c_double), ("g2p_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None

# every symbol the header declares (checked by tests/test_abi.py against include/mpm.h)
EXPORTS = ("mpm_config_default", "mpm_create", "mpm_rebuild_active", "mpm_p2g", "mpm_grid_update", "mpm_g2p",
           "mpm_step", "mpm_read_particles", "mpm_write_particles", "mpm_read_active", "mpm_read_grid",
           "mpm_get_stats", "mpm_status_string", "mpm_last_error", "mpm_destroy", "mpm_active_blocks_noalloc",
           "mpm_create_ensemble", "mpm_autotune", "mpm_get_tuning", "mpm_set_tuning", "mpm_state_bytes",
           "mpm_save_state", "mpm_load_state", "mpm_adjoint_step")


def lib():
    """Load libmpm_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("native library %s is missing: run `python -m paper_2605_28525_b300.build` "
                          "(or __graft_entry__.build())" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, fp, i64 = C.c_void_p, C.POINTER(C.c_float), C.c_int64
    L.mpm_config_default.argtypes = [C.POINTER(Config)]
    L.mpm_create.argtypes = [C.POINTER(Config), i64, vp, vp, vp, vp, vp, C.c_int, vp, C.POINTER(vp)]
    L.mpm_autotune.argtypes = [vp, C.c_int32, C.POINTER(Tuning)]
    L.mpm_state_bytes.argtypes = [vp]
    L.mpm_state_bytes.restype = C.c_int64
    L.mpm_save_state.argtypes = [vp, vp]
    L.mpm_load_state.argtypes = [vp, vp]
    L.mpm_adjoint_step.argtypes = [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.mpm_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.mpm_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.mpm_create_ensemble.argtypes = [C.POINTER(Config), C.c_int32, C.POINTER(C.c_int64), vp, vp, vp, vp, vp,
                                      C.c_int, vp, C.POINTER(vp)]
    L.mpm_rebuild_active.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.mpm_p2g.argtypes = [vp]
    L.mpm_grid_update.argtypes = [vp]
    L.mpm_g2p.argtypes = [vp]
    L.mpm_step.argtypes = [vp, C.c_int32]
    L.mpm_read_particles.argtypes = [vp, vp, vp, vp, vp, C.c_int]
    L.mpm_write_particles.argtypes = [vp, vp, vp, vp, vp, C.c_int]
    L.mpm_read_active.argtypes = [vp, C.POINTER(C.c_uint64), i64, C.POINTER(i64)]
    L.mpm_read_grid.argtypes = [vp, fp, fp, fp, fp, i64]
    L.mpm_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.mpm_status_string.argtypes = [C.c_int]
    L.mpm_status_string.restype = C.c_char_p
    L.mpm_last_error.argtypes = [vp]
    L.mpm_last_error.restype = C.c_char_p
    L.mpm_destroy.argtypes = [vp]
    L.mpm_destroy.restype = None
    L.mpm_active_blocks_noalloc.argtypes = [vp, i64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_double,
                                            C.c_int32, vp, i64, C.POINTER(i64), vp]
    _lib = L
    return L


def _status_name(s):
    try:
        return lib().mpm_status_string(int(s)).decode()
    except Exception:  # library not loadable while formatting an error
        return "status"


def _check(status, ctx=None):
    if status != OK:
        msg = lib().mpm_last_error(ctx).decode(errors="replace")
        raise MpmError(status, msg)


def default_config() -> Config:
    cfg = Config()
    _check(lib().mpm_config_default(C.byref(cfg)))
    return cfg


def config_from_workload(wl: "W.Workload", flags: int = 0, block_size: Optional[int] = None,
                         hash_capacity: int = 0, block_capacity: int = 0, max_probe: int = 0,
                         max_rebuilds: int = 0) -> Config:
    cfg = default_config()
    cfg.domain_lo[:] = list(wl.lo)
    cfg.domain_hi[:] = list(wl.hi)
    cfg.dx, cfg.dt = float(wl.dx), float(wl.dt)
    cfg.gravity[:] = [float(g) for g in wl.gravity]
    cfg.block_size = int(block_size or wl.block_size)
    cfg.material = int(wl.material)
    cfg.E, cfg.nu, cfg.rho, cfg.phi_deg = float(wl.E), float(wl.nu), float(wl.rho), float(wl.phi_deg)
    cfg.particle_volume = float(wl.dx) ** 3 / float(wl.ppc)
    cfg.floor_kind, cfg.floor_z, cfg.floor_mu = int(wl.floor_kind), float(wl.floor_z), float(wl.floor_mu)
    cfg.terrain_mu = float(wl.terrain_mu)
    cfg.wall_layers = int(wl.wall_layers)
    cfg.flags = int(flags)
    cfg.hash_capacity, cfg.block_capacity = int(hash_capacity), int(block_capacity)
    cfg.max_probe, cfg.max_rebuilds = int(max_probe), int(max_rebuilds)
    return cfg


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), 1
    a = np.ascontiguousarray(a, dtype=np.float32)
    return C.c_void_p(a.ctypes.data), 0


def check_array(a, n: int, k: int, name: str, output: bool = False):
    """An array crossing the boundary as n x k float32 values: a torch CUDA
    tensor (float32, contiguous) or a numpy array.  Input numpy arrays are
    converted to contiguous float32 (the converted array is returned and must
    be kept alive until the call); output numpy arrays must already be
    contiguous, writeable float32, since the library writes into them.  The
    library reads or writes exactly n * k values, so any other size is an
    error here rather than an access past the buffer there."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if not a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("%s: a device tensor must be CUDA, float32 and contiguous" % name)
        if a.numel() != n * k:
            raise ValueError("%s: %d values, expected %d x %d" % (name, a.numel(), n, k))
        return a
    if output:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous and a.flags.writeable):
            raise ValueError("%s: an output array must be a contiguous, writeable float32 numpy array" % name)
    else:
        a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n * k:
        raise ValueError("%s: %d values, expected %d x %d" % (name, a.size, n, k))
    return a


class Simulation:
    """One mpm_ctx.  Inputs: numpy float32 arrays (host) or torch CUDA tensors."""

    def __init__(self, cfg: Config, x, v=None, C_=None, F=None, phi=None, stream=None, terrain=None,
                 scenario_counts=None):
        L = lib()
        self._keep = []
        if terrain is not None:
            t = np.ascontiguousarray(terrain, dtype=np.float32)
            if t.ndim != 2:
                raise ValueError("terrain: a (ny, nx) height map, got shape %s" % (t.shape,))
            self._keep.append(t)
            cfg.terrain_height = t.ctypes.data_as(C.POINTER(C.c_float))
            cfg.terrain_ny, cfg.terrain_nx = t.shape
        self.cfg = cfg
        if x is None:
            raise ValueError("x is required")
        arrays = [x, v, C_, F, phi]
        on_dev = [hasattr(a, "data_ptr") for a in arrays if a is not None]
        if on_dev and any(on_dev) != all(on_dev):
            raise ValueError("mix of device and host inputs")
        device = bool(on_dev and on_dev[0])
        n = int(x.shape[0]) if len(x.shape) else 0
        arrays = [check_array(a, n, k, name) for a, k, name in
                  zip(arrays, (3, 3, 9, 9, 1), ("x", "v", "C", "F", "phi"))]
        if not device:
            self._keep.extend(a for a in arrays if a is not None)
        ptrs = [_ptr(a)[0] for a in arrays]
        self.n = n
        self._stream = stream
        sptr = None
        if stream is not None:
            sptr = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = C.c_void_p()
        if scenario_counts is None:
            st = L.mpm_create(C.byref(cfg), n, *ptrs, 1 if device else 0, sptr, C.byref(h))
        else:
            counts = np.ascontiguousarray(scenario_counts, dtype=np.int64)
            st = L.mpm_create_ensemble(C.byref(cfg), len(counts), counts.ctypes.data_as(C.POINTER(C.c_int64)),
                                       *ptrs, 1 if device else 0, sptr, C.byref(h))
        _check(st, None)
        self.h = h

    @classmethod
    def from_workload(cls, wl: "W.Workload", flags: int = 0, stream=None, device_inputs: bool = False, **kw):
        cfg = config_from_workload(wl, flags=flags, **kw)
        if device_inputs:
            import torch
            x = torch.from_numpy(wl.x).cuda()
            v = torch.from_numpy(wl.v).cuda() if wl.v is not None else None
            phi = torch.from_numpy(wl.phi).cuda() if wl.phi is not None else None
            return cls(cfg, x, v, None, None, phi, stream=stream, terrain=wl.terrain,
                       scenario_counts=wl.scenario_counts)
        return cls(cfg, wl.x, wl.v, None, None, wl.phi, stream=stream, terrain=wl.terrain,
                   scenario_counts=wl.scenario_counts)

    # ---- the step and its phases
    def rebuild_active(self):
        nb, nn = C.c_int64(), C.c_int64()
        _check(lib().mpm_rebuild_active(self.h, C.byref(nb), C.byref(nn)), self.h)
        return nb.value, nn.value

    def p2g(self):
        _check(lib().mpm_p2g(self.h), self.h)

    def grid_update(self):
        _check(lib().mpm_grid_update(self.h), self.h)

    def g2p(self):
        _check(lib().mpm_g2p(self.h), self.h)

    def step(self, nsteps: int = 1):
        _check(lib().mpm_step(self.h, int(nsteps)), self.h)

    # ---- state
    def read_particles(self, out=None):
        """Returns dict x (n,3), v (n,3), C (n,3,3), F (n,3,3) as numpy, or fills
        the given torch CUDA tensors / numpy arrays in `out`."""
        if out is None:
            out = {"x": np.empty((self.n, 3), np.float32), "v": np.empty((self.n, 3), np.float32),
                   "C": np.empty((self.n, 3, 3), np.float32), "F": np.empty((self.n, 3, 3), np.float32)}
        for key, k in (("x", 3), ("v", 3), ("C", 9), ("F", 9)):
            check_array(out.get(key), self.n, k, key, output=True)
        ps = [_ptr(out.get(k)) for k in ("x", "v", "C", "F")]
        on_dev = [p[1] for p in ps if p[1] is not None]
        if on_dev and any(on_dev) != all(on_dev):
            raise ValueError("mix of device and host outputs")
        dev = 1 if (on_dev and on_dev[0]) else 0
        _check(lib().mpm_read_particles(self.h, *[p[0] for p in ps], dev), self.h)
        return out

    def write_particles(self, x=None, v=None, C_=None, F=None):
        arrs = [x, v, C_, F]
        on_dev = [hasattr(a, "data_ptr") for a in arrs if a is not None]
        if on_dev and any(on_dev) != all(on_dev):
            raise ValueError("mix of device and host inputs")
        dev = bool(on_dev and on_dev[0])
        arrs = [check_array(a, self.n, k, name) for a, k, name in zip(arrs, (3, 3, 9, 9), ("x", "v", "C", "F"))]
        ptrs = [_ptr(a)[0] for a in arrs]
        _check(lib().mpm_write_particles(self.h, *ptrs, 1 if dev else 0), self.h)

    def read_active(self):
        n = C.c_int64()
        _check(lib().mpm_read_active(self.h, None, 0, C.byref(n)), self.h)
        keys = np.zeros(max(n.value, 1), np.uint64)
        _check(lib().mpm_read_active(self.h, keys.ctypes.data_as(C.POINTER(C.c_uint64)), len(keys),
                                     C.byref(n)), self.h)
        return keys[:n.value]

    def read_grid(self):
        st = self.stats()
        nn = st["n_active_nodes"]
        m = np.zeros(max(nn, 1), np.float32)
        mv = np.zeros((max(nn, 1), 3), np.float32)
        f = np.zeros((max(nn, 1), 3), np.float32)
        v = np.zeros((max(nn, 1), 3), np.float32)
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
        _check(lib().mpm_read_grid(self.h, fp(m), fp(mv), fp(f), fp(v), max(nn, 1)), self.h)
        return {"m": m[:nn], "mv": mv[:nn], "f": f[:nn], "v": v[:nn]}

    def autotune(self, repeats: int = 5) -> dict:
        """mpm_autotune: time the launch shapes on the current state, keep the fastest."""
        t = Tuning()
        _check(lib().mpm_autotune(self.h, int(repeats), C.byref(t)), self.h)
        return t.as_dict()

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().mpm_get_tuning(self.h, C.byref(t)), self.h)
        return t.as_dict()

    def set_tuning(self, p2g_ctas_per_sm: int, g2p_threads: int, g2p_regs: int):
        t = Tuning(p2g_ctas_per_sm, g2p_threads, g2p_regs, 0, 0.0, 0.0)
        _check(lib().mpm_set_tuning(self.h, C.byref(t)), self.h)

    # ---- checkpoints and the adjoint (device buffers: torch CUDA tensors)
    def state_bytes(self) -> int:
        return int(lib().mpm_state_bytes(self.h))

    def _state_buffer(self, buf, name):
        if not (hasattr(buf, "data_ptr") and buf.is_cuda and buf.is_contiguous()):
            raise ValueError("%s: a contiguous CUDA tensor" % name)
        if buf.numel() * buf.element_size() < self.state_bytes():
            raise ValueError("%s: %d bytes, the state needs %d" % (name, buf.numel() * buf.element_size(),
                                                                 self.state_bytes()))

    def save_state(self, dst):
        self._state_buffer(dst, "dst")
        _check(lib().mpm_save_state(self.h, C.c_void_p(dst.data_ptr())), self.h)

    def load_state(self, src):
        self._state_buffer(src, "src")
        _check(lib().mpm_load_state(self.h, C.c_void_p(src.data_ptr())), self.h)

    def adjoint_step(self, adj_next, adj_cur):
        """mpm_adjoint_step: adj_next, adj_cur are (n, 24) float32 CUDA tensors
        (x, v, C, F adjoints in id order); returns this step's (dL/dE, dL/dphi)."""
        for a, name in ((adj_next, "adj_next"), (adj_cur, "adj_cur")):
            if not hasattr(a, "data_ptr"):
                raise ValueError("%s: a CUDA tensor" % name)
            check_array(a, self.n, 24, name)
        dE, dphi = C.c_double(0.0), C.c_double(0.0)
        _check(lib().mpm_adjoint_step(self.h, C.c_void_p(adj_next.data_ptr()), C.c_void_p(adj_cur.data_ptr()),
                                      C.byref(dE), C.byref(dphi)), self.h)
        return dE.value, dphi.value

    def stats(self):
        s = Stats()
        _check(lib().mpm_get_stats(self.h, C.byref(s)), self.h)
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- key helpers (Eq. (key), m = 21, b = 2^20)
KEY_BITS, KEY_BIAS = 21, 1 << 20


def unpack_keys(keys):
    keys = np.asarray(keys, dtype=np.uint64)
    mask = np.uint64((1 << KEY_BITS) - 1)
    i = ((keys >> np.uint64(2 * KEY_BITS)) & mask).astype(np.int64) - KEY_BIAS
    j = ((keys >> np.uint64(KEY_BITS)) & mask).astype(np.int64) - KEY_BIAS
    k = (keys & mask).astype(np.int64) - KEY_BIAS
    return np.stack([i, j, k], axis=1)


def torch_allocator():
    """(alloc, free) callbacks that route the library's device memory through
    PyTorch's caching allocator.  Keep the returned objects alive as long as
    the context lives."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            s = stream if stream else 0
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), FREE_FN(_free)
