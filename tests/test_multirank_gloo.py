"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2):
the timed region's length is the slowest rank's, every rank agrees on it, and
the whole-job throughput counts every rank's work (weak scaling, replicas only:
no collective touches the data path).  The reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]
    got = bench.max_over_ranks(local_ms, torch.device("cpu"))
    value = bench.weak_scaling_value(world, 10, 2.0 * 8192 ** 3, got)
    q.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_value_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [5.0, 5.0]               # the slowest rank's time everywhere
    expect = 2 * 10 * 2.0 * 8192 ** 3 / 5e-3 / 1e9
    assert all(abs(r[2] - expect) < 1e-6 * expect for r in res)


def test_single_process_is_local_time():
    import torch
    import bench
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    class A:  # the fields run_reference reads
        n, p, steps, warmup, gpus = 64, 65521, 1, 0, 2
    assert bench.run_reference(A) == 0
    assert capsys.readouterr().out == ""
