"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every rank runs its
own replica of the workload, the job's step time is the slowest rank's, and throughput
counts the candidates of all ranks.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow replica
        t = bench.step_time_over_ranks(ms, dist, "cpu")
        out[rank] = (t, bench.job_throughput(755, world, t))
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_max_over_ranks_and_throughput_is_whole_job():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1]
    t, v = out[0]
    assert t == 15.0
    assert v == pytest.approx(2 * 755 / 0.015)


def test_single_rank_is_unchanged():
    assert bench.step_time_over_ranks(12.5) == 12.5
    assert bench.job_throughput(755, 1, 10.0) == pytest.approx(75500.0)
