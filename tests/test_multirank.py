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


def _serve_worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # rank r: 4 requests with latencies 10(r+1)..40(r+1) ms in a wall of 2(r+1) s
    lat = [10.0 * (rank + 1) * k for k in range(1, 5)]
    local = {"requests": 4, "wall_s": 2.0 * (rank + 1), "solves_per_s": 4 / (2.0 * (rank + 1)),
             "iter_per_s": 100.0 / (rank + 1), "p50_ms": 0.0, "p99_ms": 0.0, "converged": 3, "failed": 0}
    out[rank] = bench.aggregate_serving(local, lat, world)
    dist.barrier()
    dist.destroy_process_group()


def test_serving_aggregate_over_two_gloo_ranks():
    import numpy as np
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_serve_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    allat = [10.0, 20.0, 30.0, 40.0, 20.0, 40.0, 60.0, 80.0]
    for r in range(world):
        a = res[r]
        assert a["requests"] == 8 and a["replicas"] == 2 and a["converged"] == 6
        assert a["wall_s"] == 4.0                                  # the slowest replica
        assert a["solves_per_s"] == pytest.approx(8 / 4.0)
        assert a["iter_per_s"] == pytest.approx((100.0 * 2.0 + 50.0 * 4.0) / 4.0)
        assert a["p50_ms"] == pytest.approx(float(np.percentile(allat, 50)))
        assert a["p99_ms"] == pytest.approx(float(np.percentile(allat, 99)))
