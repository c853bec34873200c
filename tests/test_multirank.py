"""The replicas-only multi-GPU path of bench.py, exercised with gloo ranks on CPU.

Each rank solves problems of its own (no exchange inside a problem); the job's
time is the slowest rank's and its throughput counts every rank's problems."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, elapsed, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.replica_throughput(elapsed[rank], 3)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_throughput_takes_slowest_rank(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    elapsed = [1.5, 4.0][:world]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, elapsed, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t, v = out[r]
        assert t == max(elapsed)
        assert abs(v - world * 3 / max(elapsed)) < 1e-12


def test_single_process_is_identity():
    import bench
    t, v = bench.replica_throughput(2.0, 4)
    assert t == 2.0 and v == 2.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=3)) == 0
    assert capsys.readouterr().out == ""
