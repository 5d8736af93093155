"""Device memory through a caller allocator (mpm_config.alloc / free).

The results do not depend on the allocator. Every device buffer of a context
goes through it and comes back through free. A failing allocation is reported
as MPM_ERR_OOM, at creation and in a step that has to grow its arrays, without
leaking what was already taken; once memory is available again, the context
carries on."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W

pytestmark = pytest.mark.gpu


def _bits(sim):
    st = sim.read_particles()
    return {k: np.ascontiguousarray(v).view(np.uint32) for k, v in st.items()}


class CountingAllocator:
    """torch's caching allocator behind the library's callbacks, recording
    the live buffers; `fail` makes every allocation return NULL."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail = False
        self.alloc = mpm.ALLOC_FN(self._alloc)
        self.free = mpm.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.fail:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream if stream else 0)
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, nbytes, stream, user):
        assert ptr in self.live
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)

    def config(self, wl, flags=0):
        cfg = mpm.config_from_workload(wl, flags=flags)
        cfg.alloc, cfg.free = self.alloc, self.free
        return cfg


def test_torch_allocator_gives_the_same_bits():
    import torch
    wl = W.elastic_cube(steps=1)
    wl.v = np.tile(np.array([[0.4, -0.2, 0.1]], np.float32), (wl.n, 1))
    alloc, free = mpm.torch_allocator()
    cfg = mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC)
    cfg.alloc, cfg.free = alloc, free
    before = torch.cuda.memory_allocated()
    a = mpm.Simulation(cfg, wl.x, wl.v)
    b = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    a.step(20)
    b.step(20)
    for k, v in _bits(a).items():
        assert np.array_equal(v, _bits(b)[k]), k
    assert torch.cuda.memory_allocated() - before >= a.stats()["device_bytes"] > 0
    a.close()
    assert torch.cuda.memory_allocated() == before


def test_every_buffer_goes_through_the_allocator_and_back():
    wl = W.elastic_cube(steps=1)
    al = CountingAllocator()
    sim = mpm.Simulation(al.config(wl), wl.x, wl.v)
    sim.step(10)
    assert al.live and sum(al.live.values()) == sim.stats()["device_bytes"]
    sim.close()
    assert not al.live


def test_failed_creation_is_out_of_memory_and_gives_everything_back():
    wl = W.elastic_cube(steps=1)
    al = CountingAllocator()
    al.fail = True
    with pytest.raises(mpm.MpmError) as e:
        mpm.Simulation(al.config(wl), wl.x, wl.v)
    assert e.value.status == mpm.ERR_OOM
    assert al.calls >= 1 and not al.live


def test_failed_step_is_out_of_memory_and_the_context_recovers(oracle_mod):
    wl = W.elastic_cube(steps=1)
    wl.v = np.tile(np.array([[0.4, -0.2, 0.1]], np.float32), (wl.n, 1))
    al = CountingAllocator()
    sim = mpm.Simulation(al.config(wl, flags=mpm.DETERMINISTIC), wl.x, wl.v)
    ref = mpm.Simulation.from_workload(wl, flags=mpm.DETERMINISTIC)
    al.fail = True                      # the first step sizes the grid and the sort buffers
    with pytest.raises(mpm.MpmError) as e:
        sim.step(1)
    assert e.value.status == mpm.ERR_OOM
    assert sim.stats()["steps"] == 0
    al.fail = False
    sim.step(5)
    ref.step(5)
    for k, v in _bits(sim).items():
        assert np.array_equal(v, _bits(ref)[k]), k
    sim.close()
    assert not al.live
