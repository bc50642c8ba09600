"""Host logic of the multi-GPU mode, which runs replicas only (the whole step
on every rank, no collective on the data path): the timing barrier and the
max-over-ranks reduction of bench.py, and the reference arm's rule that only
rank 0 works, exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # each replica reports its own step time; the job's time is the slowest
        out[rank] = bench.max_over_ranks(1.5 + rank, world, device="cpu")
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_works_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench.scenes, "config", lambda *a, **k: called.append(a))

    class Args:
        workload, scale, steps, warmup, gpus, cpu_workers = 4, 1.0, 1, 1, 2, 0

    assert bench.main_reference(Args()) is None
    assert called == []  # rank 1 builds no workload and prints nothing
