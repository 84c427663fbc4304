"""Host side of the multi-GPU benchmark path, on CPU with gloo (world size 2):
each rank owns a disjoint shard of (interval, replica) chains of the same
shape (weak scaling, no data-path collective), and the reported throughput is
the units of all ranks over the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    class A:
        intervals = 16
        n_therm = 1
        n_meas = 2

    w = bench.workload(A, rank)
    units = w.n_lattices * 100
    seconds = 1.0 + rank          # rank 1 is the slow one
    value, t = bench.aggregate(units, seconds, dist)
    ids = [w.interval_id[i] * 10 + w.replica_id[i] for i in range(w.n_lattices)]
    import torch
    gathered = [None] * world
    dist.all_gather_object(gathered, (ids, w.n_lattices, w.L[0]))
    if rank == 0:
        out.put((value, t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_disjointly_and_aggregate_with_max_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    value, t, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (ids0, n0, L0), (ids1, n1, L1) = gathered
    assert n0 == n1 and L0 == L1 == 20                 # same shape per rank: weak scaling
    assert not set(ids0) & set(ids1)                   # disjoint chains
    assert t == 2.0                                    # slowest rank
    assert value == (n0 + n1) * 100 / 2.0
