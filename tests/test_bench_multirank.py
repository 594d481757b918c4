"""The bench's multi-rank host logic on CPU with the gloo backend (world size
2): whole-job throughput = the sum of the ranks' units over the slowest rank's
time, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    units = [1.0e9, 3.0e9][rank]       # pairs per step of this rank's replica
    ms = [200.0, 500.0][rank]          # its time for 10 steps
    value, ms_step, job_units = bench.job_throughput(units, ms, 10, dist, "cpu")
    q.put((rank, value, ms_step, job_units))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_step, job_units in out:
        assert ms_step == pytest.approx(50.0)          # the slowest rank: 500 ms / 10 steps
        assert job_units == pytest.approx(4.0e9)       # summed over ranks
        assert value == pytest.approx(4.0e9 / 0.050)   # whole-job units per second


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    value, ms_step, units = bench.job_throughput(2.0e9, 100.0, 4)
    assert ms_step == 25.0 and units == 2.0e9 and value == pytest.approx(2.0e9 / 0.025)


def test_reference_arm_skips_nonzero_ranks(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    bench.run_reference(argparse.Namespace(workload="tiny", seed=0, warmup=3, steps=1), 1, 2)
    assert capsys.readouterr().out == ""
