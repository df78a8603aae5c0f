"""Batch sharding over ranks: the partition, the host-side gather, and a
sharded adaptation (world size 2 over gloo on the CPU, each rank adapting
its meshes with the oracle) that must equal the unsharded one."""
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


STATS = ("rounds", "collapses", "splits", "flips", "moves", "converged")


def _small_batch():
    from paper_1505_04694_gb300 import inputs

    return inputs.batch_workloads(count=8, seed=13, tmin=200, tmax=2500)


def _oracle_adapt(i, w):
    from oracle import oracle as O

    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    st = o.adapt(O.make_params(seed=w.params.seed))
    xy, tri, m = o.get_mesh()
    return {"xy": xy, "tri": tri, "m": m, "stats": {k: st[k] for k in STATS}}


def _adapt_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = _small_batch()
    merged = shard.adapt_sharded(ws, [w.tri.shape[0] for w in ws], rank, world, _oracle_adapt)
    if rank == 0:
        q.put(merged)
    else:
        assert merged is None
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_adaptation_equals_unsharded():
    import numpy as np

    mp = pytest.importorskip("torch.multiprocessing")
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_adapt_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ws = _small_batch()
    parts = shard.partition([w.tri.shape[0] for w in ws], 2)
    assert all(parts)  # both ranks adapted meshes
    assert sorted(merged) == list(range(len(ws)))
    for i, w in enumerate(ws):
        ref = _oracle_adapt(i, w)
        got = merged[i]
        assert got["stats"] == ref["stats"]
        for k in ("xy", "tri", "m"):
            assert np.array_equal(np.ascontiguousarray(got[k]).view(np.uint8),
                                  np.ascontiguousarray(ref[k]).view(np.uint8)), (i, k)
