"""The N > 1 host path of bench.py on CPU: world-size-2 gloo ranks (replicas only, no data-path
collective).  Each rank times its own region; the job's time is the slowest rank's, and the value
counts the steps of every rank."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank                      # rank 1 is the slower replica
        t_max = bench.max_over_ranks(t_local, "cpu", world)
        q.put((rank, t_max, bench.job_value(10, world, t_max)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [1.5, 1.5]            # both ranks see the slowest time
    assert [g[2] for g in got] == [10 * 2 / 1.5] * 2     # 20 steps over 1.5 s


def test_single_rank_is_local():
    assert bench.max_over_ranks(0.25, "cpu", 1) == 0.25
    assert bench.job_value(4, 1, 0.5) == 8.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0 alone; the other
    ranks return without work and print nothing."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        frac, steps, warmup = 1.0, 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
