"""The C interface library loads and exports every function declared in
include/pm.h; argument checks answer without any device work (no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def pm():
    from paper_1505_04694_gb300 import build

    build.build()
    from paper_1505_04694_gb300 import pm as binding

    return binding


def test_every_declared_symbol_is_exported(pm):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(pm.lib, n), n
    assert sorted(pm.EXPORTS) == names


def test_argument_checks_need_no_device(pm):
    p = pm.Params().c()
    st = pm.PmStats()
    for fn in (pm.lib.pm_coarsen, pm.lib.pm_refine, pm.lib.pm_swap, pm.lib.pm_smooth,
               pm.lib.pm_adapt, pm.lib.pm_opt_smooth):
        assert fn(None, C.byref(p), C.byref(st)) == 1
    assert pm.lib.pm_adapt_batch(None, 0, None, None) == 1
    out = C.c_void_p()
    assert pm.lib.pm_mesh_create(None, 0, None, 0, None, 1, 0, C.byref(out)) == 1
    assert pm.lib.pm_mesh_destroy(None) == 0
    assert pm.lib.pm_status_string(6) == b"device wait timed out"
    assert b"null" in pm.lib.pm_last_error() or pm.lib.pm_last_error() != b""
    # measurement and test support check their arguments before any device call
    assert pm.lib.pm_fp64_peak(None) == 1
    st32, ms = C.c_int32(), C.c_double()
    assert pm.lib.pm_selftest_wait_timeout(50.0, None, C.byref(ms)) == 1
    assert pm.lib.pm_selftest_wait_timeout(50.0, C.byref(st32), None) == 1
    for bad in (0.0, -1.0, 2000.5, float("nan")):
        assert pm.lib.pm_selftest_wait_timeout(bad, C.byref(st32), C.byref(ms)) == 1
    assert pm.lib.pm_selftest_div3_dev(None, None, 4, None) == 1
    assert pm.lib.pm_selftest_div3_dev(C.c_void_p(16), C.c_void_p(32), -1, None) == 1
    assert pm.lib.pm_selftest_orient_dev(None, None, 4, None) == 1


def test_create_arguments_checked_on_host(pm):
    """Pointer and size arguments are refused before any device work (vertex
    ids and coordinates are checked on the device after the upload, which
    the GPU tests cover)."""
    import numpy as np

    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], np.int32)
    out = C.c_void_p()
    assert pm.lib.pm_mesh_create(None, 3, pm._i(tri), 1, None, 1, 0, C.byref(out)) == 1
    assert pm.lib.pm_mesh_create(pm._d(xy), 2, pm._i(tri), 1, None, 1, 0, C.byref(out)) == 1
    assert pm.lib.pm_mesh_create(pm._d(xy), 3, pm._i(tri), 0, None, 1, 0, C.byref(out)) == 1
    assert pm.lib.pm_mesh_create(pm._d(xy), 3, pm._i(tri), 1, None, 0, 0, C.byref(out)) == 1
    assert not out.value


def test_struct_layouts_match_header(pm):
    assert C.sizeof(pm.PmParams) == 3 * 8 + 6 * 4
    assert C.sizeof(pm.PmStats) == 5 * 8 + 8 + 8


def test_batch_arguments_checked_on_host(pm):
    import numpy as np

    out = C.c_void_p()
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    nv = np.array([3, 3], np.int32)
    ne = np.array([1, 1], np.int32)
    good = np.array([[0, 1, 2], [0, 1, 2]], np.int32)
    # (an id outside its mesh is found on the device after the upload: GPU test)
    f = pm.lib.pm_batch_create
    assert f(pm._d(xy), pm._i(nv), pm._i(good), pm._i(ne), 0, None, 1, 0, C.byref(out)) == 1
    nv1 = np.array([3, 2], np.int32)
    assert f(pm._d(xy), pm._i(nv1), pm._i(good), pm._i(ne), 2, None, 1, 0, C.byref(out)) == 1
    assert f(None, pm._i(nv), pm._i(good), pm._i(ne), 2, None, 1, 0, C.byref(out)) == 1
    assert pm.lib.pm_batch_adapt(None, None, None) == 1
    n = C.c_int32()
    assert pm.lib.pm_batch_size(None, C.byref(n)) == 1
    assert pm.lib.pm_batch_get_mesh(None, None, None, None, None, None) == 1
