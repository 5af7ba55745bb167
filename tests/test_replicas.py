"""The multi-GPU path is replicas only: each rank solves its own cell, and the
bench's aggregation takes the slowest rank's time and all ranks' load steps.
Exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 * (rank + 1)                  # rank 1 is the slow one
    total, value = bench.replica_throughput(ms, 20, dist, "cpu")
    out[rank] = (total, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_max_time():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        total, value = out[r]
        assert total == 200.0
        assert value == pytest.approx(2 * 20 / 0.2)


def test_single_replica():
    import bench
    total, value = bench.replica_throughput(50.0, 10)
    assert total == 50.0 and value == pytest.approx(200.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup = 1
        steps = 1
        gpus = 2
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))
    assert bench.run_reference(A()) is None
    assert not called
