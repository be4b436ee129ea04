"""The multi-rank bench path on the CPU (gloo, world size 2): each rank
conceals its own batch (weak scaling), step time = max over ranks, units
summed; the per-rank workloads are distinct.  Launched here the way the
bench runs under torchrun, with 127.0.0.1 rendezvous."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.0, 20.0][rank]
    units = [1000, 1500][rank]
    out[rank] = bench.job_throughput(ms, units, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms_max, units, rate = out[r]
        assert ms_max == 20.0 and units == 2500.0
        assert rate == pytest.approx(2500.0 / 0.020)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(5.0, 100, "cpu") == (5.0, 100.0, 100.0 / 0.005)


def test_rank_workloads_are_distinct():
    sys.path.insert(0, ROOT)
    import bench
    b0, b1 = bench.workload_blocks(0, 2), bench.workload_blocks(1, 2)
    assert len(b0) == len(b1) == 2 * 3240
    assert not np.array_equal(b0, b1)
