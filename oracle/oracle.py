"""ctypes binding of the sequential CPU oracle (test infrastructure only).

Mirrors the semantics of the CUDA library one call at a time:
``OracleMesh(xy, tri).set_metric(m); .adapt(params); .get_mesh()``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [("L_low", C.c_double), ("L_up", C.c_double), ("q_thresh", C.c_double),
                ("max_iter", C.c_int32), ("max_smooth_sweeps", C.c_int32),
                ("seed", C.c_uint32), ("opt_smooth_rounds", C.c_int32),
                ("max_rounds", C.c_int32), ("select_mode", C.c_int32)]


class OrStats(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("collapses", C.c_int64), ("splits", C.c_int64),
                ("flips", C.c_int64), ("moves", C.c_int64), ("converged", C.c_int32),
                ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        up = C.POINTER(C.c_uint8)
        L.or_create.restype = P
        L.or_create.argtypes = [dp, C.c_int32, ip, C.c_int32, up, ip]
        L.or_destroy.argtypes = [P]
        L.or_set_metric.argtypes = [P, dp]
        for name in ("or_coarsen", "or_swap", "or_refine", "or_smooth", "or_adapt",
                     "or_opt_smooth"):
            f = getattr(L, name)
            f.argtypes = [P, C.POINTER(OrParams), C.POINTER(OrStats)]
            f.restype = C.c_int32
        L.or_renumber.argtypes = [P]
        L.or_get_mesh.argtypes = [P, ip, ip, dp, ip, dp]
        L.or_get_raw.argtypes = [P, ip, ip, dp, dp, ip, up, up, up]
        L.or_adjacency.argtypes = [P, C.c_int32, ip, ip, ip, ip, C.c_int32]
        L.or_check.argtypes = [P]
        L.or_check.restype = C.c_int32
        L.or_quality_elems.argtypes = [P, dp]
        L.or_quality.argtypes = [P, dp, dp, dp]
        L.or_tri_quality.argtypes = [ip, dp, dp]
        L.or_tri_quality.restype = C.c_double
        L.or_tri_quality_grad.argtypes = [ip, dp, dp, dp]
        L.or_tri_quality_grad.restype = C.c_double
        L.or_edge_length.argtypes = [dp, dp, dp, dp]
        L.or_edge_length.restype = C.c_double
        L.or_orient_sign.argtypes = [dp]
        L.or_orient_sign.restype = C.c_int32
        L.or_fmix32.argtypes = [C.c_uint32]
        L.or_fmix32.restype = C.c_uint32
        L.or_prio.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_prio.restype = C.c_uint32
        L.or_independent_set.argtypes = [P, up, C.c_uint32, C.c_uint32, C.c_int32, up]
        L.or_colour.argtypes = [P, C.c_uint32, C.c_uint32, ip]
        L.or_colour.restype = C.c_int32
        L.or_coarsen_target.argtypes = [P, C.c_int32, C.POINTER(OrParams)]
        L.or_coarsen_target.restype = C.c_int32
        L.or_swap_target.argtypes = [P, C.c_int32, C.POINTER(OrParams), ip]
        L.or_swap_target.restype = C.c_int32
        L.or_set_check_sequential.argtypes = [P, C.c_int32]
        L.or_seq_failed.argtypes = [P]
        L.or_seq_failed.restype = C.c_int32
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def make_params(L_low=0.4, L_up=2.0 ** 0.5, q_thresh=0.7, max_iter=10, max_smooth_sweeps=10,
                seed=1, opt_smooth_rounds=0, max_rounds=0, select_mode=0):
    return OrParams(L_low, L_up, q_thresh, max_iter, max_smooth_sweeps, seed & 0xFFFFFFFF,
                    opt_smooth_rounds, max_rounds, select_mode)


class OracleError(RuntimeError):
    pass


class OracleMesh:
    def __init__(self, xy, tri, corner=None):
        L = lib()
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        st = np.zeros(1, np.int32)
        cp = None
        if corner is not None:
            corner = np.ascontiguousarray(corner, dtype=np.uint8)
            cp = _u(corner)
        self.h = L.or_create(_d(xy), xy.shape[0], _i(tri), tri.shape[0], cp, _i(st))
        if not self.h:
            raise OracleError(f"or_create failed with status {int(st[0])}")
        self.status = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    def set_metric(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1, 3)
        s = lib().or_set_metric(self.h, _d(m))
        if s:
            raise OracleError(f"or_set_metric status {s}")
        return self

    def _op(self, name, params):
        st = OrStats()
        s = getattr(lib(), name)(self.h, C.byref(params), C.byref(st))
        if s:
            raise OracleError(f"{name} status {s}")
        return st.as_dict()

    def coarsen(self, p):
        return self._op("or_coarsen", p)

    def swap(self, p):
        return self._op("or_swap", p)

    def refine(self, p):
        return self._op("or_refine", p)

    def smooth(self, p):
        return self._op("or_smooth", p)

    def opt_smooth(self, p):
        return self._op("or_opt_smooth", p)

    def adapt(self, p):
        return self._op("or_adapt", p)

    def renumber(self):
        lib().or_renumber(self.h)

    def check(self):
        return int(lib().or_check(self.h))

    def set_check_sequential(self, on=True):
        lib().or_set_check_sequential(self.h, 1 if on else 0)

    def seq_failed(self):
        return bool(lib().or_seq_failed(self.h))

    def get_mesh(self):
        nv = np.zeros(1, np.int32)
        ne = np.zeros(1, np.int32)
        L = lib()
        L.or_get_mesh(self.h, _i(nv), _i(ne), None, None, None)
        xy = np.zeros((nv[0], 2))
        tri = np.zeros((ne[0], 3), np.int32)
        m = np.zeros((nv[0], 3))
        L.or_get_mesh(self.h, _i(nv), _i(ne), _d(xy), _i(tri), _d(m))
        return xy, tri, m

    def get_raw(self):
        nv = np.zeros(1, np.int32)
        ne = np.zeros(1, np.int32)
        L = lib()
        L.or_get_raw(self.h, _i(nv), _i(ne), None, None, None, None, None, None)
        n, e = int(nv[0]), int(ne[0])
        xy = np.zeros((n, 2))
        m = np.zeros((n, 3))
        tri = np.zeros((e, 3), np.int32)
        va = np.zeros(n, np.uint8)
        ta = np.zeros(e, np.uint8)
        vf = np.zeros(n, np.uint8)
        L.or_get_raw(self.h, _i(nv), _i(ne), _d(xy), _d(m), _i(tri), _u(va), _u(ta), _u(vf))
        return dict(xy=xy, m=m, tri=tri, valive=va, talive=ta, vflag=vf)

    def adjacency(self, v, cap=256):
        nn = np.zeros(cap, np.int32)
        ne = np.zeros(cap, np.int32)
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        lib().or_adjacency(self.h, v, _i(nn), _i(a), _i(ne), _i(b), cap)
        return nn[: a[0]].copy(), ne[: b[0]].copy()

    def quality_elems(self):
        raw_ne = self.get_raw()["tri"].shape[0]
        q = np.zeros(raw_ne)
        lib().or_quality_elems(self.h, _d(q))
        return q

    def quality(self, grad=True):
        qs = np.zeros(1)
        n = self.get_raw()["xy"].shape[0]
        if not grad:
            lib().or_quality(self.h, _d(qs), None, None)
            return float(qs[0])
        dxy = np.zeros((n, 2))
        dm = np.zeros((n, 3))
        lib().or_quality(self.h, _d(qs), _d(dxy), _d(dm))
        return float(qs[0]), dxy, dm

    def independent_set(self, cand, seed, r, by_colour=False):
        """0/1 per vertex slot: the round-r set of the candidates `cand`
        (by_colour: colour classes of the mesh's last colouring)."""
        cand = np.ascontiguousarray(cand, dtype=np.uint8)
        out = np.zeros(cand.shape[0], np.uint8)
        lib().or_independent_set(self.h, _u(cand), seed & 0xFFFFFFFF, r & 0xFFFFFFFF,
                                 1 if by_colour else 0, _u(out))
        return out

    def colour(self, seed, r):
        """(colour of every vertex slot, -1 when dead; number of colours) as a
        pass whose first round counter is r colours the vertex graph."""
        nv = np.zeros(1, np.int32)
        ne = np.zeros(1, np.int32)
        lib().or_get_raw(self.h, _i(nv), _i(ne), None, None, None, None, None, None)
        col = np.zeros(int(nv[0]), np.int32)
        n = int(lib().or_colour(self.h, seed & 0xFFFFFFFF, r & 0xFFFFFFFF, _i(col)))
        return col, n

    def coarsen_target(self, v, p):
        return int(lib().or_coarsen_target(self.h, v, C.byref(p)))

    def swap_target(self, v, p):
        cd = np.zeros(2, np.int32)
        w = int(lib().or_swap_target(self.h, v, C.byref(p), _i(cd)))
        return w, int(cd[0]), int(cd[1])


def tri_quality(ids, xy, m):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    return float(lib().or_tri_quality(_i(ids), _d(xy), _d(m)))


def tri_quality_grad(ids, xy, m):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    g = np.zeros(15)
    q = float(lib().or_tri_quality_grad(_i(ids), _d(xy), _d(m), _d(g)))
    return q, g.reshape(3, 5)


def edge_length(xa, ma, xb, mb):
    xa, ma, xb, mb = (np.ascontiguousarray(a, dtype=np.float64) for a in (xa, ma, xb, mb))
    return float(lib().or_edge_length(_d(xa), _d(ma), _d(xb), _d(mb)))


def fmix32(h):
    return int(lib().or_fmix32(h & 0xFFFFFFFF))


def prio(v, seed, r):
    return int(lib().or_prio(v & 0xFFFFFFFF, seed & 0xFFFFFFFF, r & 0xFFFFFFFF))


def orient_sign(p, q, r):
    """Exact sign of the orientation of points p, q, r (the oracle's predicate)."""
    pts = np.ascontiguousarray([p[0], p[1], q[0], q[1], r[0], r[1]], dtype=np.float64)
    return int(lib().or_orient_sign(_d(pts)))
