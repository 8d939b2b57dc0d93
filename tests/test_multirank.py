"""The multi-GPU path of bench.py is N independent replicas (one lattice per
GPU needs no exchange). Its host logic -- max of the step time over ranks, sum
of the work -- runs here as two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [2.0, 3.0][rank]
    ms, gflops = bench.replica_summary(ms_local, 1e9, world, device="cpu")
    out[rank] = (ms, gflops)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, gflops = out[r]
        assert ms == pytest.approx(3.0)  # slowest rank
        assert gflops == pytest.approx(2 * 1e9 / 3e-3 / 1e9)  # work of both ranks


def test_replica_summary_single_rank():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_summary(4.0, 2e9, 1) == (4.0, pytest.approx(500.0))
