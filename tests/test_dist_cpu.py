"""Multi-rank aggregation used by bench.py under torchrun, exercised with the gloo backend on CPU
(world size 2): times combine by maximum over ranks, work by sum, so value = all ranks' work over
the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mx, sm = bench.aggregate(dist, [1.0 + rank, 10.0 * rank], [100.0 * (rank + 1)])
    out[rank] = (mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_gloo_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(world):
        mx, sm = out[r]
        assert mx == [2.0, 10.0] and sm == [300.0]


def test_aggregate_single_process():
    import bench

    assert bench.aggregate(None, [3.0], [4.0]) == ([3.0], [4.0])
