"""The benchmark's multi-rank aggregation (replicas: each rank scores its own copy of the
workload; the job's time is the slowest rank's) with two gloo ranks on CPU."""
import os
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]
    job = bench.job_time_ms(local_ms, dist, torch.device("cpu"))
    out[rank] = (job, bench.job_rate(1000.0, world, job))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        job, rate = out[r]
        assert job == 180.0
        assert abs(rate - 2000.0 / 0.18) < 1e-6
