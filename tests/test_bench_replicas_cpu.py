"""The host side of bench.py's multi-process (replica) path on CPU: two gloo
ranks, timings reduced to the slowest rank, whole-job units summed over the
replicas.  No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [1.0 + rank, 10.0 - rank]          # rank 0: (1, 10), rank 1: (2, 9)
    q.put((rank, bench.max_over_ranks(mine, world, "cpu"), bench.replica_units(5, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_units_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, vals, units in got:
        assert vals == [2.0, 10.0] and units == 10


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.replica_units(7, 1) == 7
