"""Multi-rank logic of bench.py on CPU: two gloo ranks, each a replica; the job
time is the slowest rank's and the throughput counts every rank's work."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.0 + rank  # rank 1 is the slow replica
        m = bench.max_over_ranks(t, world)
        bench.barrier(world)
        out[rank] = (m, bench.job_throughput(world, 5, 2.0 * 64 ** 3, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_throughput():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 2.0
        assert v == pytest.approx(2 * 5 * 2.0 * 64 ** 3 / 2.0)


def test_reference_arm_only_rank0(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference"]) == 0
    assert capsys.readouterr().out == ""
