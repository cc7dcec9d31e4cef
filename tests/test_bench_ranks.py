"""The multi-rank path of bench.py on CPU: two gloo ranks stand in for two
GPUs running independent replicas (the path has no data exchange).  Each
rank reports its own time; every rank must see the slowest one after the
barrier, and the whole-job rate is the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        bench._barrier(dist, cuda=False)
        t = bench._max_over_ranks(dist, 1.5 + rank, device="cpu")  # rank 1 is the slower one
        rate = bench.aggregate_rate(1000.0, dist.get_world_size(), t)
        bench._barrier(dist, cuda=False)
        out[rank] = (t, rate)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2000.0 / 2.5)
