"""Multi-rank host logic on CPU (gloo, world size 2).

The likelihood shards by walkers with no data-path collective: each rank
evaluates its own walker block; the benchmark only takes the max of the
per-rank times and sums the walkers.  These tests run that aggregation and a
walker-sharded reduction of per-walker values across two gloo ranks.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # per-rank step times (ms) and walker counts
    t = torch.tensor([100.0 + 50.0 * rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    walkers = torch.tensor([1024])
    dist.all_reduce(walkers, op=dist.ReduceOp.SUM)
    # walker-sharded values gathered in rank order (the one exchange an
    # ensemble step across GPUs would need)
    local = torch.arange(4, dtype=torch.float64) + 10 * rank
    out = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, local)
    if rank == 0:
        q.put((float(t.item()), int(walkers.item()), torch.cat(out).tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tmax, walkers, gathered = res
    assert tmax == 150.0
    assert walkers == 2048
    assert gathered == [0.0, 1.0, 2.0, 3.0, 10.0, 11.0, 12.0, 13.0]
    # whole-job throughput: all ranks' walkers over the slowest rank's time
    assert walkers / (tmax / 1e3) == pytest.approx(2048 / 0.15)
