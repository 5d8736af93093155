"""mpm_active_blocks_noalloc: the active-block keys of a particle cloud for
callers that cannot allocate device memory.

Such callers include code that runs while a framework owns the whole GPU
through its own pool, loops that must not allocate after start-up, and
plug-ins that are given device buffers but no allocator.  The entry point
keeps its hash table and sort scratch in one fixed device array instead of
allocating, so these tests check that it returns exactly the active set of
the definition (the FP64 oracle's dense block mask and scan) and what the
ordinary path (mpm_create + mpm_rebuild_active + mpm_read_active) returns,
on calls made back to back through the shared array; that a second call
leaves the device's free memory unchanged; and that it refuses sets larger
than that array, or whose keys crowd one stretch of its table beyond the
probe limit.

This file is collected last on purpose: it needs the GPU, and a failure here
should not stop the rest of the suite from running first.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import eq_keys, oracle_for, small_blob

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


def test_noalloc_equals_oracle_and_context_path_on_consecutive_calls(oracle_mod):
    cube = W.elastic_cube()
    blob, _, _ = small_blob(n=5000, seed=21)
    cases = [(cube, cube.x, 4), (blob, blob.x, 4), (cube, cube.x, 4), (blob, blob.x, 1)]
    for wl, x, B in cases:   # back to back, so each call reuses the previous call's array
        want = eq_keys(oracle_for(wl, B).active_blocks(x))
        assert np.array_equal(_context_keys(wl, x, B), want)
        for _ in range(2):
            st, got, n = _noalloc(x, wl, B)
            assert st == mpm.OK, mpm.lib().mpm_last_error(None).decode()
            assert n == len(want)
            assert np.array_equal(got, want)


def test_noalloc_second_call_allocates_nothing():
    """After the first call has loaded the array onto the device, a call
    leaves the device's free memory exactly as it found it."""
    import torch
    cube = W.elastic_cube()
    xd = torch.from_numpy(np.ascontiguousarray(cube.x)).cuda()
    out = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
    lo, hi, n = (C.c_int32 * 3)(*cube.lo), (C.c_int32 * 3)(*cube.hi), C.c_int64(-1)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        return mpm.lib().mpm_active_blocks_noalloc(C.c_void_p(xd.data_ptr()), xd.shape[0], lo, hi, float(cube.dx), 4,
                                                   C.c_void_p(out.data_ptr()), out.shape[0], C.byref(n), stream)

    assert call() == mpm.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert call() == mpm.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def _splitmix64_finaliser(z):
    """The published SplitMix64 output function (Steele, Lea and Flood 2014),
    the table's hash, on a uint64 array."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def test_noalloc_rejects_crowded_table_and_recovers():
    """129 blocks whose Eq. (key) keys share one home slot of the 2^17-slot
    table (found here by a host-side search): the last of them finds no free
    slot within the 128-probe limit, and the call says so."""
    slots, want = (1 << 17), 129
    nb = (512, 512, 128)
    found = []
    bj, bk = np.meshgrid(np.arange(nb[1], dtype=np.uint64), np.arange(nb[2], dtype=np.uint64), indexing="ij")
    bias = np.uint64(1 << 20)
    for bi in range(nb[0]):
        key = ((np.uint64(bi) + bias) << np.uint64(42)) | ((bj + bias) << np.uint64(21)) | (bk + bias)
        hit = (_splitmix64_finaliser(key.ravel()) & np.uint64(slots - 1)) == 0
        for j, k in zip(bj.ravel()[hit], bk.ravel()[hit]):
            found.append((bi, int(j), int(k)))
        if len(found) >= want:
            break
    assert len(found) >= want
    h = 1.0 / 32
    # one particle per block, its stencil (nodes 4b+1..4b+3) inside the block
    x = ((4 * np.array(found[:want], dtype=np.float64) + 2.0) * h).astype(np.float32)
    wl = W.Workload("crowded", (0, 0, 0), tuple(4 * v - 1 for v in nb), h, 1e-4, (0, 0, -9.81), W.NEOHOOKEAN,
                    1e5, 0.3, 1000.0, 30.0, 8.0, W.FLOOR_NONE, 0.0, 0.0, x)
    st, _, _ = _noalloc(x, wl, 4)
    assert st == mpm.ERR_INVALID_ARG
    assert "128 probes" in mpm.lib().mpm_last_error(None).decode()
    # one block fewer fits: the probe sequence of the last key ends at its 128th slot
    st, got, n = _noalloc(x[: want - 1], wl, 4)
    assert st == mpm.OK and n == want - 1
    assert np.array_equal(got, np.sort(eq_keys(np.array(found[: want - 1]))))
    cube = W.elastic_cube()
    st, got, _ = _noalloc(cube.x, cube, 4)
    assert st == mpm.OK and np.array_equal(got, _context_keys(cube, cube.x, 4))


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
