"""The multi-GPU form is replicas only: each rank transports its own histories with no data
exchange, and the job's time is the slowest rank's.  The cross-rank reduction bench.py uses,
run by two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 95.0][rank]
    t = bench.max_over_ranks(local_ms, dist)
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        assert out[0] == out[1] == 120.0
    # whole-job throughput: all ranks' histories over the slowest rank's time
    n, steps = 1_000_000, 10
    assert world * n * steps / (120.0 / 1e3) == pytest.approx(1.6666e8, rel=1e-3)


def test_max_over_ranks_single_process():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
