"""The multi-GPU path is independent replicas (no exchange step in the method):
the benchmark's aggregation over ranks is checked with two gloo ranks on CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, nbytes = bench.replica_reduce(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, torch.device("cpu"))
    results[rank] = (ms, nbytes)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    manager = mp.Manager()
    results = manager.dict()
    mp.spawn(_rank, args=(world, port, results), nprocs=world, join=True)
    for r in range(world):
        assert results[r] == (15.0, 3000)


def test_single_process_aggregation():
    import bench

    assert bench.replica_reduce(12.5, 777) == (12.5, 777)
