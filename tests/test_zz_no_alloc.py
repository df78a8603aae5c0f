"""pm_quality_arrays_noalloc_dev, the variant of pm_quality_arrays_dev for
callers that cannot allocate device memory during the call (a framework that
has reserved the device's memory for its own allocator, a latency-bound loop,
a program that forbids allocation after start-up).  It must give the oracle's
quality sum and gradient, and bit for bit the allocating entry point's, call
after call: its fixed scratch array keeps the previous call's contents, so
the calls alternate between sizes in both directions.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04694_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mesh(n, target, seed):
    w = inputs.psi_workload(n, target, True, seed)
    return w.xy, w.tri, w.m


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def test_noalloc_matches_oracle_and_allocating_entry_point():
    torch = pytest.importorskip("torch")
    pm = pytest.importorskip("paper_1505_04694_gb300.pm")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    # larger, smaller, larger again: leftover contents of the array in both directions
    cases = [_mesh(33, 20000, 41), _mesh(17, 3000, 42), _mesh(41, 30000, 43)]
    for xy0, tri0, m0 in cases:
        qo, do, mo = O.OracleMesh(xy0, tri0).set_metric(m0).quality()
        xy = torch.tensor(xy0, dtype=torch.float64, device=dev)
        m = torch.tensor(m0, dtype=torch.float64, device=dev)
        tri = torch.tensor(tri0, dtype=torch.int32, device=dev)
        q_ref = torch.empty(1, dtype=torch.float64, device=dev)
        dxy_ref, dm_ref = torch.empty_like(xy), torch.empty_like(m)
        pm.quality_arrays_dev(xy, m, tri, q_ref, dxy_ref, dm_ref, stream=stream)
        q = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        dxy, dm = torch.full_like(xy, np.nan), torch.full_like(m, np.nan)
        pm.quality_arrays_noalloc_dev(xy, m, tri, q, dxy, dm, stream=stream)
        torch.cuda.synchronize(dev)
        # the two entry points reduce in the same order: equal bit for bit
        assert _bits(q.cpu().numpy()) == _bits(q_ref.cpu().numpy())
        assert np.array_equal(_bits(dxy.cpu().numpy()), _bits(dxy_ref.cpu().numpy()))
        assert np.array_equal(_bits(dm.cpu().numpy()), _bits(dm_ref.cpu().numpy()))
        # against the oracle: per-vertex sums in the same (ascending element)
        # order, bit for bit; the mesh total to 1e-12 (another summation order)
        assert abs(float(q.item()) - qo) <= 1e-12 * abs(qo)
        assert np.array_equal(_bits(dxy.cpu().numpy()), _bits(do))
        assert np.array_equal(_bits(dm.cpu().numpy()), _bits(mo))
        # forward only: the same sum, the gradient arrays untouched
        q2 = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        pm.quality_arrays_noalloc_dev(xy, m, tri, q2, stream=stream)
        torch.cuda.synchronize(dev)
        assert _bits(q2.cpu().numpy()) == _bits(q.cpu().numpy())


def test_noalloc_empty_mesh_bad_ids_and_limit():
    torch = pytest.importorskip("torch")
    pm = pytest.importorskip("paper_1505_04694_gb300.pm")
    dev = torch.device("cuda:0")
    xy0, tri0, m0 = _mesh(9, 400, 44)
    xy = torch.tensor(xy0, dtype=torch.float64, device=dev)
    m = torch.tensor(m0, dtype=torch.float64, device=dev)
    # no elements: the sum is zero and every gradient entry is zero
    tri_empty = torch.empty((0, 3), dtype=torch.int32, device=dev)
    q = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    dxy, dm = torch.full_like(xy, np.nan), torch.full_like(m, np.nan)
    pm.quality_arrays_noalloc_dev(xy, m, tri_empty, q, dxy, dm)
    torch.cuda.synchronize(dev)
    assert float(q.item()) == 0.0
    assert not dxy.any().item() and not dm.any().item()
    # a vertex id outside [0, nv): PM_ERR_INVALID_MESH, NaN outputs, nothing
    # read or written through the bad id; the next call is clean again
    bad = tri0.copy()
    bad[5, 1] = xy0.shape[0] + 1000
    for fn in (pm.quality_arrays_noalloc_dev, pm.quality_arrays_dev):
        tri = torch.tensor(bad, dtype=torch.int32, device=dev)
        q = torch.zeros(1, dtype=torch.float64, device=dev)
        dxy, dm = torch.zeros_like(xy), torch.zeros_like(m)
        with pytest.raises(pm.PmError) as e:
            fn(xy, m, tri, q, dxy, dm)
        assert e.value.status == 2
        assert np.isnan(float(q.item())) and torch.isnan(dxy).all().item()
    tri = torch.tensor(tri0, dtype=torch.int32, device=dev)
    pm.quality_arrays_noalloc_dev(xy, m, tri, q, dxy, dm)
    torch.cuda.synchronize(dev)
    assert np.isfinite(float(q.item()))
    # beyond the fixed array's limit: PM_ERR_CAPACITY before any device work
    xyl, tril = inputs.grid_mesh(257)  # 131,072 elements > 65,536
    xyb = torch.tensor(xyl, dtype=torch.float64, device=dev)
    mb = torch.ones((xyl.shape[0], 3), dtype=torch.float64, device=dev)
    trib = torch.tensor(tril, dtype=torch.int32, device=dev)
    with pytest.raises(pm.PmError) as e:
        pm.quality_arrays_noalloc_dev(xyb, mb, trib, q)
    assert e.value.status == 4
