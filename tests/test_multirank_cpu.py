"""The multi-GPU bench path on CPU with two gloo ranks (127.0.0.1).

Every rank evaluates its own replica, so the only cross-rank step is the
job time: the maximum over ranks of each rank's timed region. The whole-job
value counts the units of every rank over that time. The reference arm runs
on rank 0 only.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    ms_max = bench.reduce_max_ms(local_ms, world)
    value = bench.job_value(1, 10, world, ms_max)
    out.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_time_and_value():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 150.0  # the slowest replica sets the job time
        assert value == pytest.approx(2 * 10 / 0.150)  # both ranks' evaluations over that time


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=1, warmup=0, workload=bench.DEFAULT_WORKLOAD)
    bench.run_reference(args, bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    assert capsys.readouterr().out == ""


def test_single_rank_reduce_is_identity():
    import bench

    assert bench.reduce_max_ms(12.5, 1) == 12.5
    assert bench.job_value(4096, 5, 1, 20.0) == pytest.approx(4096 * 5 / 0.02)
