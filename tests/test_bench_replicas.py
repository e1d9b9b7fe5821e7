"""bench.py's multi-replica path on CPU: two gloo ranks, the slowest rank sets the time and
the job total counts the units of every rank (one independent replica per GPU)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank          # rank 1 is slower
    units = 16384
    dist.barrier()
    ms, value = bench.aggregate(ms_local, units, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_total_units():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0
        assert abs(value - 2 * 16384 / 0.150) < 1e-6


def test_single_replica_needs_no_group():
    import bench
    ms, value = bench.aggregate(200.0, 16384, 1)
    assert ms == 200.0 and abs(value - 16384 / 0.2) < 1e-9
