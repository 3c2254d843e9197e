"""The multi-GPU path is replicas only (no data-path collective): each rank solves its
own problem and the job time is the maximum over ranks. This checks bench.py's
aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.0, 20.0][rank]  # the second rank is slower
    value, ms_max = bench.replica_throughput(ms_local, 1000, 10, world, dist, device="cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = tmp.get_context("spawn").Manager()  # no fork of this (threaded) process
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == 20.0  # the slowest rank sets the job time on every rank
        assert value == pytest.approx(world * 1000 * 10 / 0.020)


def test_single_rank_needs_no_process_group():
    import bench
    value, ms_max = bench.replica_throughput(5.0, 100, 4, 1, None)
    assert ms_max == 5.0 and value == pytest.approx(100 * 4 / 0.005)
