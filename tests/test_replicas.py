"""The multi-GPU form is replicas only (the sweep of one problem does not shard at
these sizes): N independent copies of the workload, whose timings are combined on
the host.  This checks that host path with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r = bench.dist_env()
    assert (ws, r) == (world, rank)
    # rank r took (r + 1) ms for the timed steps and 2 (r + 1) ms end to end
    ms, e2e = bench.max_over_ranks([rank + 1.0, 2.0 * (rank + 1)], dist)
    out[rank] = (ms, e2e, bench.job_throughput(ws, 1000, 10, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(worker, args=(world, free_port(), out), nprocs=world, start_method="spawn")
    for rank in range(world):
        ms, e2e, value = out[rank]
        assert ms == 2.0 and e2e == 4.0
        # 2 replicas x 1000 solves x 10 steps in 2 ms
        assert value == pytest.approx(2 * 1000 * 10 / 2e-3)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.job_throughput(1, 167772160, 20, 8.59 * 20) == pytest.approx(167772160 / 8.59e-3)
