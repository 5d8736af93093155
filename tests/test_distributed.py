"""Multi-rank reporting of bench.py on CPU: two gloo ranks, each an
independent replica; the job value uses the max of the ranks' timed seconds
and the sum of their particles."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


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
