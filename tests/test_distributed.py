"""Multi-rank reporting of bench.py on CPU: two gloo ranks, each an
independent replica; the job value uses the max of the ranks' timed seconds
and the sum of their particles.  And the reference arm (the FP64 oracle on
the host): one JSON line from rank 0, nothing from the others."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(1.5 + rank, dist)
    n = bench.sum_over_ranks(1000 * (rank + 1), dist)
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 3000.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0 and bench.sum_over_ranks(7) == 7.0


def _bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_bench_reference_arm_prints_one_json_line():
    """bench.py --impl reference runs the FP64 oracle on the host (no GPU)
    and prints one JSON line with the fields the driver reads."""
    import json
    r = _bench(["--impl", "reference", "--workload", "elastic_cube_32k", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_reference_arm_other_ranks_are_silent():
    r = _bench(["--impl", "reference", "--workload", "elastic_cube_32k", "--steps", "1", "--warmup", "3"],
               {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2", "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": "29571"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
