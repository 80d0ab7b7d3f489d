"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

The forward path has no exchange step, so N GPUs run N independent replicas (weak
scaling). The only cross-rank operations are the timing reductions: the job time is the
maximum over ranks and the units processed are summed. These run here on gloo ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    t = bench.reduce_over_ranks(1.5 + rank, w, "max", device=torch.device("cpu"))
    n = bench.reduce_over_ranks(1000.0 * (rank + 1), w, "sum", device=torch.device("cpu"))
    # whole-job throughput: units of all ranks over the slowest rank's time
    value = n / t
    dist.destroy_process_group()
    q.put((r, w, lr, t, n, value))


def test_two_gloo_ranks_reduce_time_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == pytest.approx(2.5)      # max over ranks
        assert r[4] == pytest.approx(3000.0)   # units summed over ranks
        assert r[5] == pytest.approx(1200.0)


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.0, 1, "max") == 3.0
    assert bench.reduce_over_ranks(3.0, 1, "sum") == 3.0
