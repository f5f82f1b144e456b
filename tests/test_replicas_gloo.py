"""The multi-GPU form is replicas only: each rank solves its own copy of the
workload and the benchmark reports the total updates over the slowest rank's
time.  This checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    upd = 1e9 * (rank + 1)
    t, u, n = bench.aggregate_replicas(ms, upd, dist, device="cpu")
    out[rank] = (t, u, n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        t, u, n = out[r]
        assert n == 2
        assert t == 150.0            # max over ranks
        assert u == 3e9              # sum over ranks
    # weak-scaling throughput = total updates / slowest time
    assert out[0][1] / (out[0][0] * 1e-3) == pytest.approx(2e10)


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_replicas(12.5, 7.0, None) == (12.5, 7.0, 1)
