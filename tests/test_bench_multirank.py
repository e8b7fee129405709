"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) report the
max-over-ranks step time and the whole-job throughput N * units / max time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms, value = bench.aggregate(ms_local, 1e9, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0
        assert abs(value - world * 1e9 / 0.150) < 1e-3


def test_single_rank_aggregate():
    import bench
    ms, value = bench.aggregate(200.0, 4e9, 1)
    assert ms == 200.0 and abs(value - 2e10) < 1e-3
