"""The multi-GPU path of bench.py is replicas only: each rank sweeps its own
problem and the whole-job number is the flops of all ranks over the slowest
rank's time.  This checks that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [120.0, 150.0][rank]
    flops = [3.0e12, 5.0e12][rank]
    t, f = bench.reduce_over_ranks(elapsed, flops, "cpu")
    out[rank] = (t, f, bench.replica_seed(rank))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_replicas():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, f, seed = out[r]
        assert t == 150.0          # the slowest rank's time
        assert f == 8.0e12         # all ranks' work
    assert out[0][2] != out[1][2]  # independent problems
