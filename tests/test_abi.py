"""The C-ABI library loads on a CPU-only host, exports every function that
include/mpm.h declares, and rejects invalid configurations before touching
the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2605_28525_b300 import build, mpm
    build.build()
    return mpm


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:mpm_status|const char\s*\*|void|int64_t)\s+(mpm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mpm_create", "mpm_rebuild_active", "mpm_step", "mpm_read_particles", "mpm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(native):
    lib = C.CDLL(native.LIB_PATH)
    names = _declared_functions()
    assert names == sorted(native.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(native):
    L = native.lib()
    seen = set()
    for s in range(8):
        txt = L.mpm_status_string(s).decode()
        assert txt and txt not in seen
        seen.add(txt)
    assert L.mpm_status_string(99).decode() == "unknown status"


def _try_create(native, **over):
    cfg = native.default_config()
    for k, v in over.items():
        if k in ("domain_lo", "domain_hi", "gravity"):
            getattr(cfg, k)[:] = v
        else:
            setattr(cfg, k, v)
    x = np.full((4, 3), 0.5, np.float32)
    h = C.c_void_p()
    st = native.lib().mpm_create(C.byref(cfg), over.get("_n", 4), x.ctypes.data_as(C.c_void_p), None, None, None,
                                 None, 0, None, C.byref(h))
    return st, native.lib().mpm_last_error(None).decode()


@pytest.mark.parametrize("over, why", [
    (dict(dx=0.03), "power of two"),
    (dict(block_size=3), "block_size"),
    (dict(dt=0.0), "dt"),
    (dict(nu=0.5), "nu"),
    (dict(rho=0.0), "rho"),
    (dict(material=7), "material"),
    (dict(floor_kind=9), "floor"),
    (dict(hash_capacity=100), "power of two"),
    (dict(domain_lo=[0, 0, 0], domain_hi=[2, 64, 64]), "3 cells"),
    (dict(domain_lo=[-(1 << 20) - 1, 0, 0]), "Eq. (key)"),
    (dict(domain_lo=[0, 0, 0], domain_hi=[1 << 19, 1 << 19, 1 << 10]), "2^32"),
    (dict(_n=0), "particle count"),
    (dict(flags=1, block_size=1), "block_size 4"),
])
def test_invalid_configs_rejected_on_host(native, over, why):
    st, msg = _try_create(native, **over)
    assert st == native.ERR_INVALID_ARG
    assert why in msg, msg


def test_python_binding_raises_without_library(monkeypatch, tmp_path):
    from paper_2605_28525_b300 import mpm
    monkeypatch.setattr(mpm, "_lib", None)
    monkeypatch.setattr(mpm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mpm.lib()


def test_null_arguments_are_invalid(native):
    """Every entry point that takes a context answers MPM_ERR_INVALID_ARG to
    a NULL one (and to a NULL required pointer) before touching the device,
    so these run without a GPU."""
    L, E = native.lib(), native.ERR_INVALID_ARG
    i64 = C.c_int64()
    t, s = native.Tuning(), native.Stats()
    dE, dphi = C.c_double(), C.c_double()
    buf = (C.c_float * 8)()
    assert L.mpm_rebuild_active(None, C.byref(i64), C.byref(i64)) == E
    assert L.mpm_p2g(None) == E
    assert L.mpm_grid_update(None) == E
    assert L.mpm_g2p(None) == E
    assert L.mpm_step(None, 1) == E
    assert L.mpm_read_particles(None, buf, None, None, None, 0) == E
    assert L.mpm_write_particles(None, buf, None, None, None, 0) == E
    assert L.mpm_read_active(None, None, 0, C.byref(i64)) == E
    assert L.mpm_read_grid(None, None, None, None, None, 0) == E
    assert L.mpm_get_stats(None, C.byref(s)) == E
    assert L.mpm_autotune(None, 1, C.byref(t)) == E
    assert L.mpm_get_tuning(None, C.byref(t)) == E
    assert L.mpm_set_tuning(None, C.byref(t)) == E
    assert L.mpm_save_state(None, C.cast(buf, C.c_void_p)) == E
    assert L.mpm_load_state(None, C.cast(buf, C.c_void_p)) == E
    assert L.mpm_adjoint_step(None, buf, buf, C.byref(dE), C.byref(dphi)) == E
    assert L.mpm_state_bytes(None) == 0
    L.mpm_destroy(None)   # no-op
    # creation: NULL config, positions or output handle
    cfg = native.default_config()
    x = np.full((4, 3), 0.5, np.float32)
    h = C.c_void_p()
    xp = x.ctypes.data_as(C.c_void_p)
    assert L.mpm_create(None, 4, xp, None, None, None, None, 0, None, C.byref(h)) == E
    assert L.mpm_create(C.byref(cfg), 4, None, None, None, None, None, 0, None, C.byref(h)) == E
    assert L.mpm_create(C.byref(cfg), 4, xp, None, None, None, None, 0, None, None) == E
    counts = (C.c_int64 * 2)(2, 0)
    assert L.mpm_create_ensemble(C.byref(cfg), 2, counts, xp, None, None, None, None, 0, None, C.byref(h)) == E
    assert L.mpm_create_ensemble(C.byref(cfg), 0, None, xp, None, None, None, None, 0, None, C.byref(h)) == E
    assert not h.value
