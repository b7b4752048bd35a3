"""The benchmark's multi-rank aggregation (replicas, one per GPU) on CPU
ranks with the gloo backend: the job time is the slowest rank's and the
throughput counts the units of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = 1.0 + 0.5 * rank
    units = 1000 * (rank + 1)
    t, u = bench.reduce_over_ranks(seconds, units, world, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, u = res[r]
        assert t == 1.5 and u == 3000


def test_reduce_over_ranks_single_rank():
    import bench
    assert bench.reduce_over_ranks(2.0, 7, 1, "cpu") == (2.0, 7)
