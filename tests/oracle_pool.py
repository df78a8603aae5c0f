"""Spawned oracle processes for the full-size parity tests (test
infrastructure: the oracle of a batch mesh, one mesh per task)."""
import multiprocessing as mp

_WS = None
STAT_KEYS = ("rounds", "collapses", "splits", "flips", "moves", "converged")


def batch_mesh(i):
    """Oracle adaptation of mesh i of the 512-mesh batch recipe."""
    global _WS
    from oracle import oracle as O
    from paper_1505_04694_gb300 import inputs

    if _WS is None:
        _WS = inputs.batch_workloads()
    w = _WS[i]
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    st = o.adapt(O.make_params(seed=w.params.seed))
    xy, tri, m = o.get_mesh()
    return i, xy, tri, m, {k: st[k] for k in STAT_KEYS}


def pool(n):
    """A pool of n fresh interpreters (spawned: safe after CUDA is initialised)."""
    return mp.get_context("spawn").Pool(n)
