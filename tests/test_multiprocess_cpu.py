"""The multi-GPU host logic on CPU: two gloo ranks shard a batch of independent
solves without communicating on the data path and agree on the job's timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2407_13997_gb300 import inputs
from paper_2407_13997_gb300.replicas import max_over_ranks, shard, sum_over_ranks


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [w.ndofs() for w in inputs.batching_workloads(256, seed=1)]
    mine = shard(sizes, rank, world)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    t = max_over_ranks(1.0 + rank, dist)
    units = sum_over_ranks(sum(sizes[i] for i in mine), dist)
    dist.barrier()
    if rank == 0:
        q.put((parts, t, units, sizes))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_the_batch_and_reduce_the_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts, t, units, sizes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in parts for i in part)
    assert flat == list(range(len(sizes)))                       # a partition
    loads = [sum(sizes[i] for i in part) for part in parts]
    assert abs(loads[0] - loads[1]) <= max(sizes)                # balanced to one unit
    assert t == 2.0                                              # max over ranks
    assert units == sum(sizes)                                   # whole-job units


def test_shard_is_a_deterministic_partition_for_any_world():
    sizes = [w.ndofs() for w in inputs.batching_workloads(64, seed=3)]
    for world in (1, 3, 4, 8):
        parts = [shard(sizes, r, world) for r in range(world)]
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
        assert parts == [shard(sizes, r, world) for r in range(world)]
    with pytest.raises(ValueError):
        shard(sizes, 2, 2)
