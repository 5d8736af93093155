"""mpm_active_blocks_noalloc: the active-block keys of a particle cloud for
callers that cannot allocate device memory.

Such callers include code that runs while a framework owns the whole GPU
through its own pool, loops that must not allocate after start-up, and
plug-ins that are given device buffers but no allocator.  The entry point
keeps its hash table and sort scratch in one fixed device array instead of
allocating, so these tests check that it returns exactly what the ordinary
path (mpm_create + mpm_rebuild_active + mpm_read_active) returns, on calls
made back to back through the shared array, and that it refuses sets larger
than that array.

This file is collected last on purpose: it needs the GPU, and a failure here
should not stop the rest of the suite from running first.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import small_blob

pytestmark = pytest.mark.gpu


def _noalloc(x, wl, block_size, cap=1 << 16):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    out = torch.zeros(cap, dtype=torch.int64, device="cuda")
    lo = (C.c_int32 * 3)(*wl.lo)
    hi = (C.c_int32 * 3)(*wl.hi)
    n = C.c_int64(-1)
    st = mpm.lib().mpm_active_blocks_noalloc(C.c_void_p(xd.data_ptr()), xd.shape[0], lo, hi, float(wl.dx),
                                              int(block_size), C.c_void_p(out.data_ptr()), cap, C.byref(n),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    keys = out[: max(n.value, 0)].cpu().numpy().view(np.uint64)
    return st, keys, n.value


def _context_keys(wl, x, block_size):
    cfg = mpm.config_from_workload(wl, block_size=block_size)
    with mpm.Simulation(cfg, x) as sim:
        sim.rebuild_active()
        return sim.read_active()


def test_noalloc_equals_context_path_on_consecutive_calls():
    cube = W.elastic_cube()
    blob, _, _ = small_blob(n=5000, seed=21)
    cases = [(cube, cube.x, 4), (blob, blob.x, 4), (cube, cube.x, 4), (blob, blob.x, 1)]
    for wl, x, B in cases:   # back to back, so each call reuses the previous call's array
        want = _context_keys(wl, x, B)
        for _ in range(2):
            st, got, n = _noalloc(x, wl, B)
            assert st == mpm.OK, mpm.lib().mpm_last_error(None).decode()
            assert n == len(want)
            assert np.array_equal(got, want)


def test_noalloc_rejects_sets_beyond_its_fixed_size_and_recovers():
    # one particle per block on a 42^3 lattice of blocks: 74,088 > 65,536 blocks
    h = 1.0 / 32
    g = np.arange(42) * 4 + 1.3
    x = (np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * h).astype(np.float32)
    wl = W.Workload("lattice", (0, 0, 0), (172, 172, 172), h, 1e-4, (0, 0, -9.81), W.NEOHOOKEAN, 1e5, 0.3,
                    1000.0, 30.0, 8.0, W.FLOOR_NONE, 0.0, 0.0, x)
    st, _, _ = _noalloc(x, wl, 4)
    assert st == mpm.ERR_INVALID_ARG
    assert "65536" in mpm.lib().mpm_last_error(None).decode()
    # the next call starts from a cleared array
    cube = W.elastic_cube()
    st, got, _ = _noalloc(cube.x, cube, 4)
    assert st == mpm.OK and np.array_equal(got, _context_keys(cube, cube.x, 4))
