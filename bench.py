"""Throughput of the sparse-grid MPM step on B300 (particle-updates/s).

One "step" is one full explicit MPM step through the C-ABI: the active-set
rebuild (cell keys, hashed insert, compaction, particle sort), P2G, the grid
update and G2P with the Drucker-Prager return map.  The default workload is
the 8,000,000-particle synthetic landslide (2048x1024x256 potential grid,
dx = 0.5 m, terrain level set), the largest single-GPU configuration of the
method's benchmarks.  All inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

Rank 0 prints ONE JSON line.  Under torchrun every rank runs an independent
replica (the method does not shard across GPUs); value = all particles of all
ranks x K / max-over-ranks timed seconds.  `--impl reference` times the FP64
CPU oracle (the plain, slow dense-grid implementation the tests check
against) on the same workload, K bounded steps after W warm-up steps.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-updates/s per MPM step incl. sparse rebuild, vs dense-grid GPU path"
UNIT = "particle-updates/s"

# Algorithmic bytes per particle of the dominant kernels (FP32 state, the
# figures of the method's byte model): P2G reads x, v, C, F (96 B); G2P reads
# x, F and writes x, v, C, F (144 B).  The grid traffic of the active nodes is
# added per node (P2G: 28 B of m, mv, f accumulated; G2P: 12 B of v read).
ALG_BYTES = {"p2g": (96, 28), "g2p": (144, 12)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _init_pg(ws, backend):
    if ws <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_traffic(workload: str, kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed after the counters were taken."""
    import hashlib
    src = os.path.join(ROOT, "paper_2605_28525_b300", "csrc", "transfer.cu")
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[0] == workload and f[1] == kernel and f[3] == sha:
                return int(f[2])
    except OSError:
        pass
    return None


def measured_flops_per_particle(kernel: str):
    """FP32 operations per particle of a transfer kernel from the committed ncu
    capture of the 1M column (profiles/flops.txt), or None when the kernel
    source changed after the counters were taken."""
    import hashlib
    src = os.path.join(ROOT, "paper_2605_28525_b300", "csrc", "transfer.cu")
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
        for line in open(os.path.join(ROOT, "profiles", "flops.txt")):
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[0] == "column_collapse_1M" and f[1] == kernel \
                    and f[3] == sha:
                return int(f[2]) / 1048576.0
    except OSError:
        pass
    return None


def alu_check(wl, phases: dict, sm_mhz):
    """FP32 rate of P2G and G2P against the FFMA peak at the sampled SM clock
    (148 SMs x 128 lanes x 2 flop per cycle): the ALU cross-check beside the
    HBM roofline.  The operation counts are the Drucker-Prager column's, so
    other materials get none."""
    from paper_2605_28525_b300 import workloads as W
    if not sm_mhz or wl.material != W.DRUCKER_PRAGER:
        return None
    n = wl.n
    peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    out = {"peak_tflops": peak, "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x median SM clock",
           "flop_source": "per-particle FP32 operations (FFMA, FMUL, FADD and their packed forms) of the 1M "
                          "Drucker-Prager column's ncu capture (profiles/flops.txt)"}
    for k in ("p2g", "g2p"):
        f = measured_flops_per_particle(k)
        if f is None:
            out[k] = None
            continue
        tf = f * n / (phases[k] * 1e-3) / 1e12
        out[k] = {"flop_per_particle": f, "achieved_tflops": tf, "frac": tf / peak}
    return out


def make_workload(name: str):
    from paper_2605_28525_b300 import workloads as W
    if name == "column_collapse_1M":
        return W.column_collapse()
    if name == "column_collapse_4M":
        return W.column_collapse(cells_xy=64)
    if name == "column_collapse_127M":   # 362 x 362 x 128 cells: 134,189,056 particles, about 40 GB on the device
        return W.column_collapse(cells_xy=362)
    if name == "column_collapse_454M":   # 488 x 488 x 250 cells: 476,288,000 particles, about 140 GB on the device
        return W.column_collapse(cells_xy=488, cells_z=250)
    if name == "landslide_8M":
        return W.landslide()
    if name == "elastic_cube_32k":
        return W.elastic_cube()
    if name == "column_ensemble_64":
        return W.column_ensemble()
    if name == "diff_column_262k":
        return W.diff_column()
    raise SystemExit("unknown workload %s" % name)


class ClockSampler:
    """SM clocks, power and clock-event (throttle) reasons sampled through
    NVML (the library nvidia-smi reads) from a background thread every ~2 ms
    while the timed region runs; nvidia-smi's 200 ms loop when NVML is
    missing.  Read-only: no setting of the GPU is touched."""
    def __init__(self, device_index: int):
        self.index = device_index
        self.rows = []          # (sm_mhz, max_mhz, power_w, [reasons])
        self.source = None
        self.nvml_error = None
        self._stop = None

    class _Nvml:
        """The few read-only NVML calls the sampler needs, through pynvml when
        it is installed, else straight from the driver's libnvidia-ml."""

        def __init__(self, uuid: str, index: int):
            try:
                import pynvml as nv
                nv.nvmlInit()
                try:
                    self.h = nv.nvmlDeviceGetHandleByUUID(uuid)
                except Exception:
                    self.h = nv.nvmlDeviceGetHandleByIndex(index)
                self.clock = lambda: nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM)
                self.max_clock = lambda: nv.nvmlDeviceGetMaxClockInfo(self.h, nv.NVML_CLOCK_SM)
                self.reasons = lambda: nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                self.power = lambda: nv.nvmlDeviceGetPowerUsage(self.h)
                return
            except ImportError:
                pass
            import ctypes as C
            L = C.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = C.c_void_p()
            if L.nvmlDeviceGetHandleByUUID(uuid.encode(), C.byref(h)) != 0:
                if L.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(h)) != 0:
                    raise RuntimeError("no NVML handle")
            self.h = h

            def q(fn, *args, kind=C.c_uint):
                out = kind()
                if fn(h, *args, C.byref(out)) != 0:
                    raise RuntimeError("NVML query failed")
                return out.value
            self.clock = lambda: q(L.nvmlDeviceGetClockInfo, C.c_int(1))           # NVML_CLOCK_SM
            self.max_clock = lambda: q(L.nvmlDeviceGetMaxClockInfo, C.c_int(1))
            try:
                rfn = L.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:          # older drivers: the same call under its former name
                rfn = L.nvmlDeviceGetCurrentClocksThrottleReasons
            self.reasons = lambda: q(rfn, kind=C.c_ulonglong)
            self.power = lambda: q(L.nvmlDeviceGetPowerUsage)

    # clock-event reason bits (nvml.h)
    REASON_BITS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
                   ("hw_thermal_slowdown", 0x40), ("hw_power_brake", 0x80))

    def _run_nvml(self, nv):
        # at least one sample, also when a short timed region ends before the
        # thread's first pass
        mx = nv.max_clock()
        while True:
            sm = nv.clock()
            r = nv.reasons()
            try:
                pw = nv.power() / 1000.0
            except Exception:
                pw = None
            self.rows.append((float(sm), float(mx), pw, [n for n, m in self.REASON_BITS if r & m]))
            if self._stop.wait(0.002):
                break

    def __enter__(self):
        import threading
        self._stop = threading.Event()
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.index).uuid)
            nv = self._Nvml(uuid if uuid.startswith("GPU-") else "GPU-" + uuid, self.index)
            self.source = "nvml"
            self._thr = threading.Thread(target=self._run_nvml, args=(nv,), daemon=True)
            self._thr.start()
        except Exception as e:     # no NVML binding or device: fall back to nvidia-smi
            self.nvml_error = "%s: %s" % (type(e).__name__, e)
            self._thr = None
            self._smi = None
            try:
                self._path = "/tmp/mpm_bench_clocks_%d.csv" % os.getpid()
                self._f = open(self._path, "w")
                self._smi = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                     "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                     "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                     "--format=csv,noheader,nounits", "-lms", "200"], stdout=self._f, stderr=subprocess.DEVNULL)
                self.source = "nvidia-smi"
            except OSError:
                self._smi = None
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._thr is not None:
            self._thr.join(timeout=5)
        elif getattr(self, "_smi", None) is not None:
            self._smi.terminate()
            self._smi.wait(timeout=10)
            self._f.close()
            self.rows.extend(self.parse_smi(open(self._path)))

    @staticmethod
    def parse_smi(lines):
        """Rows of the nvidia-smi query above: sm, max sm, power, then four
        reason columns ("Active" / "Not Active")."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 7 and p[0].replace(".", "").isdigit():
                pw = float(p[2]) if p[2].replace(".", "").isdigit() else None
                rows.append((float(p[0]), float(p[1]), pw, [names[k] for k in range(4) if p[3 + k].lower() == "active"]))
        return rows

    def summary(self):
        if not self.rows:
            return None
        sm = [r[0] for r in self.rows]
        pw = [r[2] for r in self.rows if r[2] is not None]
        return {"sm_mhz": float(np.median(sm)), "sm_min_mhz": min(sm), "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": sorted({n for r in self.rows for n in r[3]}),
                "power_w_median": float(np.median(pw)) if pw else None,
                "samples": len(self.rows), "source": self.source,
                **({"nvml_error": self.nvml_error} if self.nvml_error else {})}


L2_BYTES = 126 * 10 ** 6
STATE_BYTES_PER_PARTICLE = 2 * 32 * 4      # two SoA buffers of 32 float components


def time_steps(sim, nsteps, flush=None):
    """Device time (ms) per step with CUDA events on the library's stream.
    Without `flush`: one sim.step(nsteps) call between the events (the steps
    are queued on the device, one host synchronisation at the end).  With
    `flush`: sim.step(1) per step, the L2 flushed between steps outside the
    events."""
    import torch
    st = torch.cuda.current_stream()
    if flush is None:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.step(nsteps)
        b.record(st)
        b.synchronize()
        return [a.elapsed_time(b) / nsteps] * nsteps
    out = []
    for _ in range(nsteps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.step(1)
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def time_phases(sim, nsteps, flush=None):
    """Device time (ms) of each phase of the step, through the phase entry
    points (same kernels as sim.step).  The rebuild reads its status on the
    host, so the GPU would go idle until the host has queued P2G; a fixed
    clock wait on the GPU (torch.cuda._sleep, about 0.1 ms, outside every
    interval) lets the host queue P2G, the grid update and G2P first, so that
    no host latency falls inside their intervals.  The rebuild interval
    includes its own status read."""
    import torch
    st = torch.cuda.current_stream()
    acc = {"rebuild": [], "p2g": [], "grid": [], "g2p": []}
    for _ in range(nsteps):
        if flush is not None:
            flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(st)
        sim.rebuild_active()
        ev[5].record(st)
        torch.cuda._sleep(200000)
        ev[1].record(st)
        sim.p2g()
        ev[2].record(st)
        sim.grid_update()
        ev[3].record(st)
        sim.g2p()
        ev[4].record(st)
        ev[4].synchronize()
        acc["rebuild"].append(ev[0].elapsed_time(ev[5]))
        for k, name in ((1, "p2g"), (2, "grid"), (3, "g2p")):
            acc[name].append(ev[k].elapsed_time(ev[k + 1]))
    return {k: float(np.mean(v)) for k, v in acc.items()}


def e2e_steps(sim, n, nsteps):
    """End-to-end through the public API with host buffers: each step uploads
    the particle state from pinned host memory, steps, and reads it back."""
    import torch
    pin = lambda *s: torch.empty(*s, dtype=torch.float32, pin_memory=True).numpy()
    state = sim.read_particles({"x": pin(n, 3), "v": pin(n, 3), "C": pin(n, 3, 3), "F": pin(n, 3, 3)})
    out = {"x": pin(n, 3), "v": pin(n, 3), "C": pin(n, 3, 3), "F": pin(n, 3, 3)}
    ts = []
    for _ in range(nsteps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.write_particles(state["x"], state["v"], state["C"].reshape(n, 9), state["F"].reshape(n, 9))
        sim.step(1)
        sim.read_particles(out)
        ts.append(time.perf_counter() - t0)
        state, out = out, state
    h2d = n * (3 + 3 + 9 + 9) * 4
    return float(np.mean(ts)), h2d, h2d


def link_copies(nbytes, reps=3):
    """Plain pinned host <-> device copies of `nbytes` each way (one
    cudaMemcpyAsync per direction, CUDA events on the copying stream): the
    host link's own rate, against which the end-to-end step is read.
    Returns (host->device GB/s, device->host GB/s, ms for both)."""
    import torch
    n = max(1, nbytes // 4)
    h = torch.empty(n, dtype=torch.float32, pin_memory=True)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    d.copy_(h, non_blocking=True)
    h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    up, down = [], []
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        d.copy_(h, non_blocking=True)
        ev[1].record()
        h.copy_(d, non_blocking=True)
        ev[2].record()
        ev[2].synchronize()
        up.append(ev[0].elapsed_time(ev[1]))
        down.append(ev[1].elapsed_time(ev[2]))
    tu, td = float(np.median(up)), float(np.median(down))
    del h, d
    return 4 * n / tu / 1e6, 4 * n / td / 1e6, tu + td


def cpu_baseline(wl, nsteps, openmp=False):
    """The FP64 oracle as it stands on `nsteps` full steps of `wl` (its dense
    grid covers the whole box of `wl`): one host core, or with `openmp` its
    all-core build (P2G into per-thread grids, grid update and G2P split over
    the cores).  Returns (particle-updates/s, seconds, threads used)."""
    import oracle
    o = oracle.Oracle(lo=wl.lo, hi=wl.hi, h=wl.dx, dt=wl.dt, g=wl.gravity, B=wl.block_size, material=wl.material,
                      E=wl.E, nu=wl.nu, rho=wl.rho, phi_deg=wl.phi_deg, ppc=wl.ppc, floor_kind=wl.floor_kind,
                      floor_z=wl.floor_z, floor_mu=wl.floor_mu,
                      terrain=None if wl.terrain is None else wl.terrain.astype(np.float64),
                      terrain_mu=wl.terrain_mu, wall_layers=wl.wall_layers, openmp=openmp)
    t0 = time.perf_counter()
    o.run(wl.x, wl.v, None, None, wl.phi, nsteps=nsteps)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0)))) if openmp else 1
    return wl.n * nsteps / dt, dt, threads


def adjoint_leg(wl, iters: int, every: int = 20):
    """The differentiable column: the plain forward, one value-and-gradient
    through the checkpointed adjoint, and an Adam calibration of phi from 30
    deg towards a phi = 34 deg target run (deterministic mode throughout)."""
    import torch
    from paper_2605_28525_b300 import adjoint as A, mpm
    target = A.column_target(wl, 34.0, wl.steps)
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC), wl.x, wl.v)
    sim.step(1)
    sim.close()
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC), wl.x, wl.v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(wl.steps)
    sim.read_particles()
    t_fwd = time.perf_counter() - t0
    sim.close()
    t_grad = []
    for _ in range(2):   # the first call also pays one-time allocations and graph captures
        t0 = time.perf_counter()
        L, dphi, dE = A.column_value_and_grad(wl, wl.phi_deg, wl.E, target, wl.steps, every)
        t_grad.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    hist = A.calibrate_phi(wl, target, wl.phi_deg, iters=iters, lr=0.5, every=every)
    t_cal = time.perf_counter() - t0
    return {"workload": wl.name, "particles": wl.n, "steps": wl.steps, "checkpoint_every": every,
            "forward_s": t_fwd, "value_and_grad_s": t_grad[1], "value_and_grad_first_call_s": t_grad[0],
            "cost_vs_forward": t_grad[1] / t_fwd,
            "loss": L, "dL_dphi_per_deg": dphi, "dL_dE": dE, "target_phi_deg": 34.0,
            "calibration": {"iters": iters, "phi_deg": [hist[0][0], hist[-1][0]], "loss": [hist[0][1], hist[-1][1]],
                            "seconds": t_cal, "seconds_per_iter": t_cal / max(iters, 1)}}


def ensemble_leg(steps: int, stream):
    """The batched ensemble (64 column collapses of uneven size, each in its
    own sparse grid, every launch covering all of them) timed like the main
    line: queued steps between CUDA events, inputs resident on the device."""
    import torch
    from paper_2605_28525_b300 import mpm, workloads as W
    wl = W.column_ensemble()
    sim = mpm.Simulation.from_workload(wl, flags=0, stream=stream, device_inputs=True)
    for _ in range(3):
        sim.step(1)
    tuning = sim.autotune(3)
    sim.step(1)
    torch.cuda.synchronize()
    ms = float(np.mean(time_steps(sim, steps, None)))
    st = sim.stats()
    sim.close()
    torch.cuda.empty_cache()
    return {"workload": wl.name, "scenarios": int(len(wl.scenario_counts)), "particles": wl.n, "steps": steps,
            "ms_per_step": ms, "value": wl.n / (ms * 1e-3), "unit": UNIT, "active_blocks": st["n_active_blocks"],
            "tuning": {k: tuning[k] for k in ("p2g_ctas_per_sm", "g2p_threads", "g2p_regs")},
            "step_launch": "one mpm_step call of K steps (one CUDA graph per step, every launch covering all scenarios)"}


def occupancy_sweep(boxes=(128, 256, 512, 1024), steps: int = 20):
    """The 1M column in boxes of growing width (same body): sparse and dense
    GPU steps against the node occupancy, as the paper's sparse-vs-dense
    figure does for its examples."""
    import torch
    from paper_2605_28525_b300 import mpm, workloads as W
    out = []
    for b in boxes:
        wl = W.column_collapse(box_xy=b)
        row = {"box": "%dx%dx256" % (b, b)}
        for name, flags in (("sparse", 0), ("dense", mpm.DENSE_GRID)):
            sim = mpm.Simulation.from_workload(wl, flags=flags, stream=torch.cuda.current_stream(), device_inputs=True)
            for _ in range(3):
                sim.step(1)
            ms = float(np.mean(time_steps(sim, steps, None)))
            st = sim.stats()
            sim.close()
            row[name + "_ms"] = ms
            if name == "sparse":
                row["occupancy_nodes"] = st["n_active_nodes"] / st["n_dense_nodes"]
        row["speedup"] = row["dense_ms"] / row["sparse_ms"]
        out.append(row)
        torch.cuda.empty_cache()
    return out


REF_SAMPLE_PARTICLES = 65536


def reference_sample(wl, target: int = REF_SAMPLE_PARTICLES, margin: int = 6):
    """A spatial sample of a workload for the reference arm, so that each of
    its steps is bounded: the oracle's cost is its dense grid over the whole
    box plus its particles, so a particle subset alone would not bound it.
    The sample is every particle whose base cell lies in an x-y window of the
    particles' bounding box, scaled by (target / n)^(1/2) per axis and centred
    (so each sampled column keeps its full height, floor or terrain contact
    included); the oracle's box is the sample's cells plus `margin` cells
    (beyond the sticky wall layers and the stencil) and the matching slice of
    the terrain.  Workloads of at most `target` particles are used whole."""
    import dataclasses
    if wl.n <= target:
        return wl, "the whole workload"
    h = wl.dx
    base = np.floor(wl.x.astype(np.float64) / h - 0.5).astype(np.int64)
    blo, bhi = base.min(0), base.max(0) + 1
    ext = bhi - blo
    size = np.maximum(1, np.round(ext[:2] * (target / wl.n) ** 0.5).astype(np.int64))
    c0 = blo[:2] + (ext[:2] - size) // 2
    c1 = c0 + size
    sel = np.all((base[:, :2] >= c0) & (base[:, :2] < c1), axis=1)
    slo, shi = base[sel].min(0), base[sel].max(0) + 1
    lo = np.maximum(np.asarray(wl.lo, np.int64), slo - margin)
    hi = np.minimum(np.asarray(wl.hi, np.int64), shi + 2 + margin)
    terrain = None
    if wl.terrain is not None:
        terrain = wl.terrain[lo[1] - wl.lo[1]:hi[1] - wl.lo[1] + 1, lo[0] - wl.lo[0]:hi[0] - wl.lo[0] + 1]
    sub = dataclasses.replace(wl, lo=tuple(int(a) for a in lo), hi=tuple(int(a) for a in hi), x=wl.x[sel],
                              v=None if wl.v is None else wl.v[sel], phi=None if wl.phi is None else wl.phi[sel],
                              terrain=terrain, scenario_counts=None)
    what = "the %d particles of a %dx%d-cell window through the body, on a dense %s node grid" % (
        sub.n, size[0], size[1], "x".join(str(sub.hi[a] - sub.lo[a] + 1) for a in range(3)))
    return sub, what


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = make_workload(args.workload)
    if wl.scenario_counts is not None:          # the oracle runs one scenario of an ensemble
        from paper_2605_28525_b300 import workloads as W
        wl = W.ensemble_member(wl, 0)
    full = wl
    wl, what = reference_sample(full)
    import oracle
    o_args = dict(lo=wl.lo, hi=wl.hi, h=wl.dx, dt=wl.dt, g=wl.gravity, B=wl.block_size, material=wl.material,
                  E=wl.E, nu=wl.nu, rho=wl.rho, phi_deg=wl.phi_deg, ppc=wl.ppc, floor_kind=wl.floor_kind,
                  floor_z=wl.floor_z, floor_mu=wl.floor_mu, wall_layers=wl.wall_layers,
                  terrain=None if wl.terrain is None else wl.terrain.astype(np.float64), terrain_mu=wl.terrain_mu)
    o = oracle.Oracle(**o_args)
    x, v, Cm, F = o.run(wl.x, wl.v, None, None, wl.phi, nsteps=args.warmup)
    t0 = time.perf_counter()
    o.run(x, v, Cm, F, wl.phi, nsteps=args.steps)
    dt = time.perf_counter() - t0
    value = wl.n * args.steps / dt
    sample = "%d FP64 oracle steps after %d warm-up steps, each over a spatial sample of %s (%d particles): %s" % (
        args.steps, args.warmup, full.name, full.n, what)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(full.describe(), l2="n/a (host)", reference_sample=what),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="landslide_8M")
    ap.add_argument("--dense-steps", type=int, default=5)
    ap.add_argument("--cpu-steps", type=int, default=100,
                    help="oracle steps of the CPU baseline, over the reference arm's spatial sample")
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble sub-record (column_ensemble_64)")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--adjoint", action="store_true",
                    help="add the differentiable-column leg (diff_column_262k: gradients and calibration)")
    ap.add_argument("--adjoint-iters", type=int, default=50)
    ap.add_argument("--sweep", action="store_true",
                    help="add the sparse-vs-dense occupancy sweep of the 1M column (boxes 128..1024 wide)")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes p2g_ctas_per_sm,g2p_threads,g2p_regs instead of the autotuner's choice")
    ap.add_argument("--compaction", default="hash", choices=["hash", "scan"],
                    help="active-set realisation: the hash (Sec. 4.3) or the scan (Sec. 4.2)")
    ap.add_argument("--deterministic", action="store_true",
                    help="MPM_DETERMINISTIC: fixed-order P2G reduction and (block, cell, id) order (bitwise reproducible)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2605_28525_b300 import mpm, workloads as W
    torch.cuda.set_device(local)
    dist = _init_pg(ws, "nccl")
    dev = torch.device("cuda", local)
    wl = make_workload(args.workload)
    # Between timed steps the L2 is flushed unless the particle state alone
    # (read and written once per step) is more than twice its size.
    big = wl.n * STATE_BYTES_PER_PARTICLE > 2 * L2_BYTES
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush = None if (big or args.no_flush) else flush_buf
    l2_note = ("not flushed: particle state %.0f MB (read + written every step) > 2 x %d MB L2" % (
        wl.n * STATE_BYTES_PER_PARTICLE / 1e6, L2_BYTES // 10 ** 6)) if flush is None else "flushed between steps"
    stream = torch.cuda.current_stream()

    mode = mpm.DETERMINISTIC if args.deterministic else 0
    cflags = (mpm.SCAN_COMPACTION if args.compaction == "scan" else 0) | mode
    sim = mpm.Simulation.from_workload(wl, flags=cflags, stream=stream, device_inputs=True)
    for _ in range(args.warmup):
        sim.step(1)
    if args.tuning:                 # fixed launch shapes (e.g. under a profiler, where the autotuner's timing is off)
        sim.set_tuning(*(int(v) for v in args.tuning.split(",")))
        tuning = sim.tuning()
    else:
        tuning = sim.autotune(3)    # the library's own autotuner: launch shapes only, no result changes
    sim.step(1)                     # recapture the step graphs with the chosen shapes
    torch.cuda.synchronize()
    launches0 = sim.stats()["kernel_launches"]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        per_step = time_steps(sim, args.steps, flush)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sim.stats()["kernel_launches"] - launches0
    total_ms = max_over_ranks(sum(per_step), dist, dev)
    n_all = sum_over_ranks(wl.n, dist, dev)
    value = n_all * args.steps / (total_ms / 1e3)
    st = sim.stats()

    phases = time_phases(sim, max(3, min(args.steps, 10)), flush_buf)
    dom = max(("p2g", "g2p"), key=lambda k: phases[k])
    pb, nb = ALG_BYTES[dom]
    alg_bytes = wl.n * pb + st["n_active_nodes"] * nb
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6400.0))
    achieved = alg_bytes / (phases[dom] * 1e-3) / 1e9
    # the counters were taken in the fast mode; the deterministic P2G is another kernel
    traffic = None if args.deterministic else measured_traffic(wl.name, dom)
    # both transfer kernels against their own byte models, the dominant one included
    per_kernel = {}
    for k in ("p2g", "g2p"):
        kb = wl.n * ALG_BYTES[k][0] + st["n_active_nodes"] * ALG_BYTES[k][1]
        ka = kb / (phases[k] * 1e-3) / 1e9
        per_kernel[k] = {"achieved": ka, "frac": ka / peak, "alg_bytes_per_launch": kb, "kernel_ms": phases[k],
                         "traffic": None if args.deterministic else measured_traffic(wl.name, k)}

    e2e = None
    if not args.no_e2e:
        t_e2e, h2d, d2h = e2e_steps(sim, wl.n, max(3, min(args.steps, 5)))
        e2e = {"value": wl.n * ws / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        up, down, copy_ms = link_copies(h2d)
        # the same bytes as plain pinned copies: what the host link alone takes
        e2e["link"] = {"h2d_gbs": up, "d2h_gbs": down, "copies_ms_per_step": copy_ms,
                       "e2e_ms_per_step": 1e3 * t_e2e}
    sim.close()

    dense = None
    if not args.no_dense and wl.scenario_counts is None:   # ensembles run on the sparse grid only
        dsim = mpm.Simulation.from_workload(wl, flags=mpm.DENSE_GRID | mode, stream=stream, device_inputs=True)
        for _ in range(3):
            dsim.step(1)
        d_ms = time_steps(dsim, args.dense_steps, flush)
        dsim.close()
        dense_value = wl.n / (np.mean(d_ms) / 1e3)
        dense = {"value": dense_value * ws, "unit": UNIT, "ms_per_step": float(np.mean(d_ms)),
                 "sparse_speedup": (wl.n / (total_ms / args.steps / 1e3)) / dense_value,
                 "occupancy_nodes": st["n_active_nodes"] / st["n_dense_nodes"]}

    ens = None
    if not args.no_ensemble and rank == 0 and wl.scenario_counts is None:
        ens = ensemble_leg(args.ensemble_steps, stream)
    sweep = occupancy_sweep() if (args.sweep and rank == 0) else None
    adj = None
    if args.adjoint and rank == 0:
        adj = adjoint_leg(W.diff_column() if wl.name != "diff_column_262k" else wl, args.adjoint_iters)

    cpu = None
    if rank == 0 and not args.no_cpu:
        from paper_2605_28525_b300 import workloads as W
        cwl = wl if wl.scenario_counts is None else W.ensemble_member(wl, 0)   # the oracle runs one scenario
        swl, what = reference_sample(cwl)
        cv, cdt, _ = cpu_baseline(swl, args.cpu_steps)
        ov, odt, othr = cpu_baseline(swl, args.cpu_steps, openmp=True)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d FP64 oracle steps of %s, one core, over %s; %.1f s" % (args.cpu_steps, cwl.name, what, cdt),
               "all_cores": {"value": ov, "unit": UNIT, "cores": othr, "kind": "oracle (OpenMP build of the same source)",
                             "sample": "the same %d steps and sample on %d threads; %.1f s" % (args.cpu_steps, othr, odt)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(wl.describe(), l2=l2_note, step_launch="one mpm_step call of K steps (CUDA graphs)"
                           if flush is None else "mpm_step(1) per step",
                           parallelism="replicas" if ws > 1 else "single GPU", compaction=args.compaction,
                           mode="deterministic" if args.deterministic else "fast",
                           tuning={k: tuning[k] for k in ("p2g_ctas_per_sm", "g2p_threads", "g2p_regs")},
                           active_blocks=st["n_active_blocks"], particle_blocks=st["n_particle_blocks"]),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "alg_bytes_per_launch": alg_bytes, "kernel_ms": phases[dom], "kernels": per_kernel},
            "phases_ms": phases,
            "alu_check": None if args.deterministic else alu_check(wl, phases, (clk.summary() or {}).get("sm_mhz")),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "dense_gpu": dense,
            "gpu_launches": launches,
            **({"ensemble": ens} if ens is not None else {}),
            **({"adjoint": adj} if adj is not None else {}),
            **({"occupancy_sweep": sweep} if sweep is not None else {}),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
