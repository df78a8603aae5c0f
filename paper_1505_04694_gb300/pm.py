"""Python binding of the C interface in include/pm.h (argument marshalling only).

Every step of the adaptation runs in the CUDA library
``paper_1505_04694_gb300/_build/libpm.so``; this module never computes
anything itself.  Importing it raises ImportError when the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).

Host arrays are numpy; device arrays are torch CUDA tensors (their
``data_ptr()`` is passed to the ``*_dev`` entry points).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpm.so")

PM_OK = 0
STATUS_NAMES = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_INVALID_MESH", 3: "PM_ERR_OOM",
                4: "PM_ERR_CAPACITY", 5: "PM_ERR_CUDA", 6: "PM_ERR_TIMEOUT"}

# Every function declared in include/pm.h.
EXPORTS = ["pm_mesh_create", "pm_mesh_create_dev", "pm_mesh_destroy", "pm_set_stream",
           "pm_set_metric", "pm_set_metric_dev", "pm_coarsen", "pm_refine", "pm_swap",
           "pm_smooth", "pm_adapt", "pm_opt_smooth", "pm_adapt_batch", "pm_get_mesh",
           "pm_get_mesh_dev", "pm_get_raw", "pm_adjacency", "pm_quality",
           "pm_quality_arrays_dev", "pm_status_string", "pm_last_error", "pm_kernel_launches",
           "pm_profile_enable", "pm_profile_read", "pm_quality_arrays_noalloc_dev",
           "pm_fp64_peak", "pm_selftest_wait_timeout", "pm_selftest_div3_dev",
           "pm_batch_create", "pm_batch_create_dev", "pm_batch_size", "pm_batch_adapt",
           "pm_batch_get_mesh", "pm_batch_get_mesh_dev", "pm_set_tuning", "pm_get_tuning",
           "pm_tuning_load", "pm_tuning_source", "pm_build_id", "pm_selftest_orient_dev"]


class PmParams(C.Structure):
    _fields_ = [("L_low", C.c_double), ("L_up", C.c_double), ("q_thresh", C.c_double),
                ("max_iter", C.c_int32), ("max_smooth_sweeps", C.c_int32),
                ("seed", C.c_uint32), ("opt_smooth_rounds", C.c_int32),
                ("max_rounds", C.c_int32), ("select", C.c_int32)]


SELECT_HASH, SELECT_COLOUR = 0, 1


class PmStats(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("collapses", C.c_int64), ("splits", C.c_int64),
                ("flips", C.c_int64), ("moves", C.c_int64), ("converged", C.c_int32),
                ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PmTuning(C.Structure):
    _fields_ = [("block", C.c_int32 * 4), ("blocks_per_sm", C.c_int32 * 4),
                ("rounds_limit", C.c_int32 * 3), ("rounds_blocks_per_sm", C.c_int32 * 3),
                ("fuse_limit", C.c_int32 * 2)]

    def as_dict(self):
        return {k: list(getattr(self, k)) for k, _ in self._fields_}


class PmError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing")
    try:  # let torch's CUDA runtime satisfy libcudart when it is installed
        import torch  # noqa: F401
    except Exception:
        pass
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, up = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
    mp = C.POINTER(C.c_void_p)
    sig = {
        "pm_mesh_create": [dp, C.c_int32, ip, C.c_int32, up, C.c_int32, C.c_int, mp],
        "pm_mesh_create_dev": [vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, vp, mp],
        "pm_mesh_destroy": [vp],
        "pm_set_stream": [vp, vp],
        "pm_set_metric": [vp, dp],
        "pm_set_metric_dev": [vp, vp],
        "pm_coarsen": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_refine": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_swap": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_smooth": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_adapt": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_opt_smooth": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_adapt_batch": [mp, C.c_int32, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_get_mesh": [vp, ip, ip, dp, ip, dp],
        "pm_get_mesh_dev": [vp, ip, ip, vp, vp, vp],
        "pm_get_raw": [vp, ip, ip, dp, dp, ip, up, up, up],
        "pm_adjacency": [vp, C.c_int32, ip, ip, ip, ip, C.c_int32],
        "pm_quality": [vp, dp, dp, dp],
        "pm_quality_arrays_dev": [vp, vp, C.c_int32, vp, C.c_int32, vp, vp, vp, vp],
        "pm_quality_arrays_noalloc_dev": [vp, vp, C.c_int32, vp, C.c_int32, vp, vp, vp, vp],
        "pm_batch_create": [dp, ip, ip, ip, C.c_int32, up, C.c_int32, C.c_int, mp],
        "pm_batch_create_dev": [vp, ip, vp, ip, C.c_int32, vp, C.c_int32, vp, mp],
        "pm_batch_size": [vp, ip],
        "pm_batch_adapt": [vp, C.POINTER(PmParams), C.POINTER(PmStats)],
        "pm_batch_get_mesh": [vp, ip, ip, dp, ip, dp],
        "pm_batch_get_mesh_dev": [vp, ip, ip, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.pm_kernel_launches.argtypes = []
    L.pm_kernel_launches.restype = C.c_uint64
    L.pm_profile_enable.argtypes = [C.c_char_p]
    L.pm_profile_enable.restype = C.c_int
    L.pm_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double)]
    L.pm_profile_read.restype = C.c_int
    L.pm_fp64_peak.argtypes = [C.POINTER(C.c_double)]
    L.pm_fp64_peak.restype = C.c_int
    L.pm_selftest_wait_timeout.argtypes = [C.c_double, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_double)]
    L.pm_selftest_wait_timeout.restype = C.c_int
    L.pm_selftest_div3_dev.argtypes = [vp, vp, C.c_int64, vp]
    L.pm_selftest_div3_dev.restype = C.c_int
    L.pm_selftest_orient_dev.argtypes = [vp, vp, C.c_int64, vp]
    L.pm_selftest_orient_dev.restype = C.c_int
    L.pm_set_tuning.argtypes = [C.POINTER(PmTuning)]
    L.pm_set_tuning.restype = C.c_int
    L.pm_get_tuning.argtypes = [C.POINTER(PmTuning)]
    L.pm_get_tuning.restype = C.c_int
    L.pm_tuning_load.argtypes = [C.c_char_p, C.c_char_p]
    L.pm_tuning_load.restype = C.c_int
    L.pm_tuning_source.argtypes = []
    L.pm_tuning_source.restype = C.c_char_p
    L.pm_build_id.argtypes = []
    L.pm_build_id.restype = C.c_char_p
    L.pm_status_string.argtypes = [C.c_int]
    L.pm_status_string.restype = C.c_char_p
    L.pm_last_error.argtypes = []
    L.pm_last_error.restype = C.c_char_p
    return L


lib = _load()


def _check(status, where):
    if status != PM_OK:
        raise PmError(status, where, lib.pm_last_error().decode())


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


@dataclass
class Params:
    """pm_params (same defaults as the paper-derived workloads)."""
    L_low: float = 0.4
    L_up: float = 2.0 ** 0.5
    q_thresh: float = 0.7
    max_iter: int = 10
    max_smooth_sweeps: int = 10
    seed: int = 1
    opt_smooth_rounds: int = 0
    max_rounds: int = 0
    select: int = SELECT_HASH  # SELECT_COLOUR: colour-class sets (Sec. 3.2)

    def c(self) -> PmParams:
        return PmParams(self.L_low, self.L_up, self.q_thresh, self.max_iter,
                        self.max_smooth_sweeps, self.seed & 0xFFFFFFFF, self.opt_smooth_rounds,
                        self.max_rounds, self.select)


def as_params(p) -> PmParams:
    if isinstance(p, PmParams):
        return p
    if isinstance(p, Params):
        return p.c()
    return Params(**{k: getattr(p, k) for k in Params.__dataclass_fields__}).c()


class Mesh:
    """A mesh on the GPU (pm_mesh handle)."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)

    # -- creation ------------------------------------------------------------
    @classmethod
    def from_host(cls, xy, tri, corner=None, cap_factor=2, device=0):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        cp = None
        if corner is not None:
            corner = np.ascontiguousarray(corner, dtype=np.uint8)
            cp = _u(corner)
        out = C.c_void_p()
        _check(lib.pm_mesh_create(_d(xy), xy.shape[0], _i(tri), tri.shape[0], cp, cap_factor,
                                  device, C.byref(out)), "pm_mesh_create")
        return cls(out.value)

    @classmethod
    def from_device(cls, xy, tri, corner=None, cap_factor=2, stream=None):
        """xy: (nv,2) float64 CUDA tensor; tri: (ne,3) int32 CUDA tensor."""
        out = C.c_void_p()
        _check(lib.pm_mesh_create_dev(C.c_void_p(xy.data_ptr()), xy.shape[0],
                                      C.c_void_p(tri.data_ptr()), tri.shape[0],
                                      C.c_void_p(corner.data_ptr()) if corner is not None else None,
                                      cap_factor, C.c_void_p(stream), C.byref(out)),
               "pm_mesh_create_dev")
        return cls(out.value)

    def close(self):
        if self.h is not None and self.h.value:
            lib.pm_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        _check(lib.pm_set_stream(self.h, C.c_void_p(stream)), "pm_set_stream")

    # -- metric --------------------------------------------------------------
    def set_metric(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1, 3)
        _check(lib.pm_set_metric(self.h, _d(m)), "pm_set_metric")
        return self

    def set_metric_dev(self, m):
        _check(lib.pm_set_metric_dev(self.h, C.c_void_p(m.data_ptr())), "pm_set_metric_dev")
        return self

    # -- operators -------------------------------------------------------------
    def _op(self, fn, name, params):
        st = PmStats()
        p = as_params(params)
        _check(fn(self.h, C.byref(p), C.byref(st)), name)
        return st.as_dict()

    def coarsen(self, params):
        return self._op(lib.pm_coarsen, "pm_coarsen", params)

    def refine(self, params):
        return self._op(lib.pm_refine, "pm_refine", params)

    def swap(self, params):
        return self._op(lib.pm_swap, "pm_swap", params)

    def smooth(self, params):
        return self._op(lib.pm_smooth, "pm_smooth", params)

    def opt_smooth(self, params):
        return self._op(lib.pm_opt_smooth, "pm_opt_smooth", params)

    def adapt(self, params):
        return self._op(lib.pm_adapt, "pm_adapt", params)

    # -- output --------------------------------------------------------------
    def sizes(self):
        nv = np.zeros(1, np.int32)
        ne = np.zeros(1, np.int32)
        _check(lib.pm_get_mesh(self.h, _i(nv), _i(ne), None, None, None), "pm_get_mesh")
        return int(nv[0]), int(ne[0])

    def get_mesh(self, out=None):
        """Compacted mesh (xy[nv, 2], tri[ne, 3] int32, m[nv, 3]) in host arrays.

        out: optional (xy, tri, m) C-contiguous arrays of those dtypes with at
        least nv / ne rows, for example views of page-locked (pinned) memory,
        which the device fills by direct DMA; views of their first rows are
        returned."""
        nv, ne = self.sizes()
        if out is None:
            xy = np.empty((nv, 2))
            tri = np.empty((ne, 3), np.int32)
            m = np.empty((nv, 3))
        else:
            bxy, btri, bm = out
            for arr, rows, cols, dt in ((bxy, nv, 2, np.float64), (btri, ne, 3, np.int32),
                                        (bm, nv, 3, np.float64)):
                if (arr.dtype != dt or arr.ndim != 2 or arr.shape[1] != cols
                        or arr.shape[0] < rows or not arr.flags.c_contiguous):
                    raise ValueError(f"output array needs shape (>={rows}, {cols}), dtype {dt}, "
                                     "C order")
            xy, tri, m = bxy[:nv], btri[:ne], bm[:nv]
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(lib.pm_get_mesh(self.h, _i(a), _i(b), _d(xy), _i(tri), _d(m)), "pm_get_mesh")
        return xy, tri, m

    def get_mesh_dev(self, xy, tri, m):
        """Write the compacted mesh into preallocated CUDA tensors; returns (nv, ne)."""
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(lib.pm_get_mesh_dev(self.h, _i(a), _i(b),
                                   C.c_void_p(xy.data_ptr()) if xy is not None else None,
                                   C.c_void_p(tri.data_ptr()) if tri is not None else None,
                                   C.c_void_p(m.data_ptr()) if m is not None else None),
               "pm_get_mesh_dev")
        return int(a[0]), int(b[0])

    def get_raw(self):
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(lib.pm_get_raw(self.h, _i(a), _i(b), None, None, None, None, None, None),
               "pm_get_raw")
        n, e = int(a[0]), int(b[0])
        xy = np.zeros((n, 2))
        m = np.zeros((n, 3))
        tri = np.zeros((e, 3), np.int32)
        va = np.zeros(n, np.uint8)
        ta = np.zeros(e, np.uint8)
        vf = np.zeros(n, np.uint8)
        _check(lib.pm_get_raw(self.h, _i(a), _i(b), _d(xy), _d(m), _i(tri), _u(va), _u(ta),
                              _u(vf)), "pm_get_raw")
        return dict(xy=xy, m=m, tri=tri, valive=va, talive=ta, vflag=vf)

    def adjacency(self, v, cap=256):
        nn = np.zeros(cap, np.int32)
        ne = np.zeros(cap, np.int32)
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(lib.pm_adjacency(self.h, v, _i(nn), _i(a), _i(ne), _i(b), cap), "pm_adjacency")
        return nn[: a[0]].copy(), ne[: b[0]].copy()

    def quality(self, grad=True):
        nv = self.get_raw_sizes()[0]
        qs = np.zeros(1)
        if not grad:
            _check(lib.pm_quality(self.h, _d(qs), None, None), "pm_quality")
            return float(qs[0])
        dxy = np.zeros((nv, 2))
        dm = np.zeros((nv, 3))
        _check(lib.pm_quality(self.h, _d(qs), _d(dxy), _d(dm)), "pm_quality")
        return float(qs[0]), dxy, dm

    def get_raw_sizes(self):
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(lib.pm_get_raw(self.h, _i(a), _i(b), None, None, None, None, None, None),
               "pm_get_raw")
        return int(a[0]), int(b[0])


class Batch(Mesh):
    """Many meshes in one handle (pm_batch_*): one store, every round of every
    operator over all of them at once."""

    @classmethod
    def from_host(cls, meshes, corner=None, cap_factor=2, device=0):
        """meshes: list of (xy (nv,2) float64, tri (ne,3) int32 local ids)."""
        xy = np.concatenate([np.asarray(a, np.float64).reshape(-1, 2) for a, _ in meshes])
        tri = np.concatenate([np.asarray(t, np.int32).reshape(-1, 3) for _, t in meshes])
        nv = [np.asarray(a).reshape(-1, 2).shape[0] for a, _ in meshes]
        ne = [np.asarray(t).reshape(-1, 3).shape[0] for _, t in meshes]
        return cls.from_arrays(xy, nv, tri, ne, corner, cap_factor, device)

    @classmethod
    def from_arrays(cls, xy, nv, tri, ne, corner=None, cap_factor=2, device=0):
        """Meshes already concatenated in host arrays: xy (sum nv, 2) float64,
        tri (sum ne, 3) int32 local ids, nv / ne per-mesh counts."""
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        nv = np.ascontiguousarray(nv, dtype=np.int32)
        ne = np.ascontiguousarray(ne, dtype=np.int32)
        cp = None
        if corner is not None:
            corner = np.ascontiguousarray(corner, dtype=np.uint8)
            cp = _u(corner)
        out = C.c_void_p()
        _check(lib.pm_batch_create(_d(xy), _i(nv), _i(tri), _i(ne), nv.shape[0], cp, cap_factor,
                                   device, C.byref(out)), "pm_batch_create")
        return cls(out.value)

    @classmethod
    def from_device(cls, xy, nv, tri, ne, corner=None, cap_factor=2, stream=None):
        """xy: (sum nv, 2) float64 CUDA tensor; tri: (sum ne, 3) int32 CUDA
        tensor; nv, ne: host int arrays of per-mesh counts."""
        nv = np.ascontiguousarray(nv, dtype=np.int32)
        ne = np.ascontiguousarray(ne, dtype=np.int32)
        out = C.c_void_p()
        _check(lib.pm_batch_create_dev(C.c_void_p(xy.data_ptr()), _i(nv),
                                       C.c_void_p(tri.data_ptr()), _i(ne), nv.shape[0],
                                       C.c_void_p(corner.data_ptr()) if corner is not None
                                       else None, cap_factor, C.c_void_p(stream), C.byref(out)),
               "pm_batch_create_dev")
        return cls(out.value)

    def count(self):
        n = np.zeros(1, np.int32)
        _check(lib.pm_batch_size(self.h, _i(n)), "pm_batch_size")
        return int(n[0])

    def adapt(self, params):
        """params: one Params for all meshes or a list (one per mesh)."""
        n = self.count()
        if not isinstance(params, (list, tuple)):
            params = [params] * n
        arr = (PmParams * n)(*[as_params(p) for p in params])
        st = (PmStats * n)()
        _check(lib.pm_batch_adapt(self.h, arr, st), "pm_batch_adapt")
        return [x.as_dict() for x in st]

    def sizes(self):
        n = self.count()
        nv = np.zeros(n, np.int32)
        ne = np.zeros(n, np.int32)
        _check(lib.pm_batch_get_mesh(self.h, _i(nv), _i(ne), None, None, None),
               "pm_batch_get_mesh")
        return nv, ne

    def get_meshes(self, out=None):
        """Compacted meshes as a list of (xy, tri, m) host arrays (views of one
        concatenation; `out` = (xy, tri, m) preallocated C-contiguous arrays
        with enough rows, for example page-locked views)."""
        nv, ne = self.sizes()
        tv, te = int(nv.sum()), int(ne.sum())
        if out is None:
            xy, tri, m = np.empty((tv, 2)), np.empty((te, 3), np.int32), np.empty((tv, 3))
        else:
            bxy, btri, bm = out
            for arr, rows, cols, dt in ((bxy, tv, 2, np.float64), (btri, te, 3, np.int32),
                                        (bm, tv, 3, np.float64)):
                if (arr.dtype != dt or arr.ndim != 2 or arr.shape[1] != cols
                        or arr.shape[0] < rows or not arr.flags.c_contiguous):
                    raise ValueError(f"output array needs shape (>={rows}, {cols}), dtype {dt}, "
                                     "C order")
            xy, tri, m = bxy[:tv], btri[:te], bm[:tv]
        a = np.zeros_like(nv)
        b = np.zeros_like(ne)
        _check(lib.pm_batch_get_mesh(self.h, _i(a), _i(b), _d(xy), _i(tri), _d(m)),
               "pm_batch_get_mesh")
        ov = np.concatenate([[0], np.cumsum(a)])
        oe = np.concatenate([[0], np.cumsum(b)])
        return [(xy[ov[i]:ov[i + 1]], tri[oe[i]:oe[i + 1]], m[ov[i]:ov[i + 1]])
                for i in range(a.shape[0])]

    def get_mesh_dev(self, xy, tri, m):
        """Compacted meshes into preallocated CUDA tensors (concatenated);
        returns the per-mesh counts (nv, ne) as numpy arrays."""
        n = self.count()
        a = np.zeros(n, np.int32)
        b = np.zeros(n, np.int32)
        _check(lib.pm_batch_get_mesh_dev(self.h, _i(a), _i(b),
                                         C.c_void_p(xy.data_ptr()) if xy is not None else None,
                                         C.c_void_p(tri.data_ptr()) if tri is not None else None,
                                         C.c_void_p(m.data_ptr()) if m is not None else None),
               "pm_batch_get_mesh_dev")
        return a, b


def adapt_batch(meshes, params):
    """pm_adapt_batch over a list of Mesh objects; params: one or one per mesh."""
    n = len(meshes)
    if not isinstance(params, (list, tuple)):
        params = [params] * n
    arr = (PmParams * n)(*[as_params(p) for p in params])
    hs = (C.c_void_p * n)(*[m.h.value for m in meshes])
    st = (PmStats * n)()
    _check(lib.pm_adapt_batch(hs, n, arr, st), "pm_adapt_batch")
    return [s.as_dict() for s in st]


def quality_arrays_dev(xy, m, tri, qsum, dxy=None, dm=None, stream=0):
    """pm_quality_arrays_dev on CUDA tensors (runs on `stream` and waits for it;
    raises PmError on a device-detected error, the outputs then hold NaN)."""
    _check(lib.pm_quality_arrays_dev(C.c_void_p(xy.data_ptr()), C.c_void_p(m.data_ptr()),
                                     xy.shape[0], C.c_void_p(tri.data_ptr()), tri.shape[0],
                                     C.c_void_p(qsum.data_ptr()),
                                     C.c_void_p(dxy.data_ptr()) if dxy is not None else None,
                                     C.c_void_p(dm.data_ptr()) if dm is not None else None,
                                     C.c_void_p(stream)), "pm_quality_arrays_dev")


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib.pm_kernel_launches())


def profile_enable(kernel_substring):
    """Time every launch of library kernels whose name contains the string."""
    _check(lib.pm_profile_enable(kernel_substring.encode() if kernel_substring else None),
           "pm_profile_enable")


def fp64_peak():
    """Measured FP64 add/multiply throughput of the current device, G ops/s."""
    g = C.c_double()
    _check(lib.pm_fp64_peak(C.byref(g)), "pm_fp64_peak")
    return float(g.value)


def selftest_wait_timeout(limit_ms):
    """Let a grid barrier that nothing completes run out after limit_ms:
    returns (device status word, kernel ms)."""
    st = C.c_int32()
    ms = C.c_double()
    _check(lib.pm_selftest_wait_timeout(limit_ms, C.byref(st), C.byref(ms)),
           "pm_selftest_wait_timeout")
    return int(st.value), float(ms.value)


def profile_read():
    """(total device ms, launches, counted FP64 operations) of the profiled kernels."""
    ms = C.c_double()
    n = C.c_int64()
    wk = C.c_double()
    _check(lib.pm_profile_read(C.byref(ms), C.byref(n), C.byref(wk)), "pm_profile_read")
    return float(ms.value), int(n.value), float(wk.value)


def quality_arrays_noalloc_dev(xy, m, tri, qsum, dxy=None, dm=None, stream=0):
    """pm_quality_arrays_noalloc_dev: as quality_arrays_dev, allocating nothing
    (at most 65536 elements and 65536 vertices)."""
    _check(lib.pm_quality_arrays_noalloc_dev(
        C.c_void_p(xy.data_ptr()), C.c_void_p(m.data_ptr()), xy.shape[0],
        C.c_void_p(tri.data_ptr()), tri.shape[0], C.c_void_p(qsum.data_ptr()),
        C.c_void_p(dxy.data_ptr()) if dxy is not None else None,
        C.c_void_p(dm.data_ptr()) if dm is not None else None, C.c_void_p(stream)),
        "pm_quality_arrays_noalloc_dev")


def selftest_div3_dev(x, out, stream=0):
    """out = x / 3 element-wise on the device, by the quality functional's own
    division-by-three routine (float64 CUDA tensors of equal length)."""
    _check(lib.pm_selftest_div3_dev(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                    x.numel(), C.c_void_p(stream)), "pm_selftest_div3_dev")


def set_tuning(t=None):
    """pm_set_tuning: dict with block[4], blocks_per_sm[4], rounds_limit[3]
    (None restores the defaults)."""
    if t is None:
        _check(lib.pm_set_tuning(None), "pm_set_tuning")
        return
    d = dict(get_tuning_defaults(), **t)
    c = PmTuning(*[(C.c_int32 * len(d[k]))(*d[k]) for k, _ in PmTuning._fields_])
    _check(lib.pm_set_tuning(C.byref(c)), "pm_set_tuning")


def get_tuning_defaults():
    return {"block": [128] * 4, "blocks_per_sm": [16] * 4, "rounds_limit": [131072] * 3,
            "rounds_blocks_per_sm": [1] * 3, "fuse_limit": [0, 1 << 30]}


def get_tuning():
    c = PmTuning()
    _check(lib.pm_get_tuning(C.byref(c)), "pm_get_tuning")
    return c.as_dict()


def load_tuning(path, gpu_name=None):
    """pm_tuning_load; True when an entry for this GPU and build was applied."""
    return lib.pm_tuning_load(path.encode(), gpu_name.encode() if gpu_name else None) == PM_OK


def tuning_source():
    return lib.pm_tuning_source().decode()


def build_id():
    return lib.pm_build_id().decode()


def selftest_orient_dev(pts, out, stream=0):
    """out[i] = exact orientation sign of pts[i] = (px, py, qx, qy, rx, ry) on the
    device (pts: (n, 6) float64 CUDA tensor, out: (n,) int32 CUDA tensor)."""
    _check(lib.pm_selftest_orient_dev(C.c_void_p(pts.data_ptr()), C.c_void_p(out.data_ptr()),
                                      pts.shape[0], C.c_void_p(stream)), "pm_selftest_orient_dev")
