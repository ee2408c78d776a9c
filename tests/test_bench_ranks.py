"""The multi-rank (replicas) logic of bench.py on CPU: two gloo ranks, each with its own step time;
the reported time is the maximum over ranks, the same on every rank."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [12.5, 30.25]
    out[rank] = bench.max_over_ranks(times[rank], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_max_over_two_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 30.25, 1: 30.25}


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
