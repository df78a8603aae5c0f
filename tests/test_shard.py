"""Batch sharding over ranks: the partition and the host-side gather
(world size 2 over gloo on the CPU)."""
import os

import pytest

from paper_1505_04694_gb300 import shard


def test_partition_balanced_and_complete():
    sizes = [5, 1, 9, 3, 3, 7, 2, 8]
    parts = shard.partition(sizes, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert shard.partition(sizes, 3) == parts  # deterministic
    assert shard.partition(sizes, 1) == [list(range(len(sizes)))]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [10, 4, 7, 1, 12, 3]
    parts = shard.partition(sizes, world)
    local = {i: {"triangles": sizes[i] * 2, "rank": rank} for i in parts[rank]}
    merged = shard.gather_results(local, rank, world)
    if rank == 0:
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(6))
    parts = shard.partition([10, 4, 7, 1, 12, 3], 2)
    for r, part in enumerate(parts):
        for i in part:
            assert merged[i]["rank"] == r
