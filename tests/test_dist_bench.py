"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
whole-job time is the maximum over ranks and the throughput counts every
rank's replica of the workload (weak scaling).  No GPU is involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 100.0 + 50.0 * rank          # rank 1 is the slower one
    total = bench.job_time_ms(local, world, "cpu")
    value = bench.job_throughput(1000, world, 3, total)
    dist.barrier()
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_throughput_counts_all_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        total, value = out[r]
        assert total == 150.0
        assert value == pytest.approx(world * 1000 * 3 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_time_ms(42.0, 1) == 42.0
    assert bench.job_throughput(10, 1, 2, 1000.0) == pytest.approx(20.0)
