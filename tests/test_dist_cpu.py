"""Host logic of the multi-rank benchmark path on CPU: two gloo ranks agree on
the slowest rank's time and on the weak-scaling aggregate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


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
    t = bench.max_over_ranks(10.0 + rank, world)
    v = bench.aggregate_throughput(1_000_000, t, world)
    bench.barrier(world)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    t, v = out[0]
    assert t == 11.0                                     # slowest rank
    assert abs(v - 2 * 1_000_000 / 11e-3 / 1e9) < 1e-12  # units of both ranks over the slowest time
