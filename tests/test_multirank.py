"""The N > 1 host logic of bench.py (replicas, max-over-ranks timing), run as
world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 1000.0 * (rank + 1)            # rank 1 is the slowest replica
    value, total = bench.aggregate_ranks(local_ms, steps=3, T=2000, world=world)
    out[rank] = (value, total, bench.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # both ranks see the slowest rank's time, and the job's throughput counts both replicas
    for r in range(world):
        value, total, seed = res[r]
        assert total == 2000.0
        assert value == pytest.approx(world * 3 * 2000 / 2.0)
    assert res[0][2] != res[1][2]                # replicas draw different random streams


def test_single_rank_needs_no_process_group():
    import bench
    value, total = bench.aggregate_ranks(500.0, steps=2, T=100, world=1)
    assert total == 500.0 and value == pytest.approx(400.0)
