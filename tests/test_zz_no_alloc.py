"""pm_quality_arrays_noalloc_dev, the variant of pm_quality_arrays_dev for
callers that cannot allocate device memory during the call: it must give the
same quality sum and gradient as the allocating entry point, call after call
(its fixed scratch array keeps the previous call's contents).

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from paper_1505_04694_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mesh(n, target, seed):
    w = inputs.psi_workload(n, target, True, seed)
    return w.xy, w.tri, w.m


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    pm = pytest.importorskip("paper_1505_04694_gb300.pm")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [_mesh(33, 20000, 41), _mesh(17, 3000, 42)]  # two calls, different sizes
    for xy0, tri0, m0 in cases:
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
        qr, qn = float(q_ref.item()), float(q.item())
        assert abs(qn - qr) <= 1e-12 * abs(qr)
        for a, b in ((dxy, dxy_ref), (dm, dm_ref)):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    pm = pytest.importorskip("paper_1505_04694_gb300.pm")
    dev = torch.device("cuda:0")
    xy0, tri0 = inputs.grid_mesh(257)  # 131,072 elements > 65,536
    xy = torch.tensor(xy0, dtype=torch.float64, device=dev)
    m = torch.ones((xy0.shape[0], 3), dtype=torch.float64, device=dev)
    tri = torch.tensor(tri0, dtype=torch.int32, device=dev)
    q = torch.empty(1, dtype=torch.float64, device=dev)
    with pytest.raises(pm.PmError) as e:
        pm.quality_arrays_noalloc_dev(xy, m, tri, q)
    assert e.value.status == 4
