"""The replicas-only multi-GPU path of bench.py, on two gloo ranks (CPU).

One system's solve does not shard; N GPUs run N independent replicas.  The
only cross-rank step is the reduction of timings: the whole-job rate is every
rank's units over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = [2.0, 3.0][rank]  # the slower rank sets the job time
    out[rank] = (bench.replica_max(t, world, device="cpu"),
                 bench.replica_throughput(10, t, world, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_reduce_to_the_slowest_rank():
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == (3.0, 20 / 3.0)


def test_single_rank_is_the_identity():
    import bench

    assert bench.replica_max(1.5, 1) == 1.5
    assert bench.replica_throughput(7, 2.0, 1) == 3.5
