"""Independent mesh checks written for the tests (exact rational geometry).

Nothing here shares code with the oracle or the CUDA library: orientation is
evaluated exactly with fractions, adjacency is rebuilt from the element list.
"""
from fractions import Fraction

import numpy as np


def exact_orient(p, q, r):
    px, py = Fraction(float(p[0])), Fraction(float(p[1]))
    qx, qy = Fraction(float(q[0])), Fraction(float(q[1]))
    rx, ry = Fraction(float(r[0])), Fraction(float(r[1]))
    return (qx - px) * (ry - py) - (qy - py) * (rx - px)


def adjacency(tris, nv):
    NN = [set() for _ in range(nv)]
    NE = [set() for _ in range(nv)]
    for k, t in enumerate(tris):
        for i in range(3):
            NE[t[i]].add(k)
            NN[t[i]].add(t[(i + 1) % 3])
            NN[t[i]].add(t[(i + 2) % 3])
    return NN, NE


def directed_edges(tris):
    out = {}
    for t in tris:
        for i in range(3):
            e = (t[i], t[(i + 1) % 3])
            out[e] = out.get(e, 0) + 1
    return out


def boundary_edges(tris):
    de = directed_edges(tris)
    return {e for e in de if (e[1], e[0]) not in de}


def on_square_side(p, q):
    for k in (0, 1):
        for val in (0.0, 1.0):
            if p[k] == val and q[k] == val:
                return True
    return False


def valid_triangulation(xy, tris, exact=True):
    """Conformity + orientation + vertex manifoldness + disk topology.
    Returns (ok, reason)."""
    used = sorted({v for t in tris for v in t})
    de = directed_edges(tris)
    if any(c > 1 for c in de.values()):
        return False, "duplicate directed edge"
    if len({frozenset(t) for t in tris}) != len(tris):
        return False, "duplicate element"
    for t in tris:
        o = exact_orient(xy[t[0]], xy[t[1]], xy[t[2]]) if exact else None
        if exact and not o > 0:
            return False, "non-positive orientation"
    NN, NE = adjacency(tris, xy.shape[0])
    for v in used:
        d = len(NN[v]) - len(NE[v])
        if d not in (0, 1):
            return False, f"non-manifold vertex {v}"
    undirected = {frozenset(e) for e in de}
    V, E, F = len(used), len(undirected), len(tris)
    if V - E + F != 1:
        return False, f"Euler characteristic {V - E + F}"
    return True, ""


def total_area_exact(xy, tris):
    s = Fraction(0)
    for t in tris:
        s += exact_orient(xy[t[0]], xy[t[1]], xy[t[2]])
    return s / 2


def unit_square_ok(xy, tris, tol=1e-12):
    """Output mesh covers the unit square: area 1, boundary edges on its sides,
    four corners present.  Returns (ok, reason)."""
    p = xy[tris]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    if (area <= 0).any():
        return False, "inverted element"
    if abs(area.sum() - 1.0) > tol:
        return False, f"area {area.sum()!r}"
    t = np.asarray(tris, dtype=np.int64)
    nv = xy.shape[0]
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = e[:, 0] * nv + e[:, 1]
    rkey = e[:, 1] * nv + e[:, 0]
    bnd = e[~np.isin(key, rkey)]
    pa, pb = xy[bnd[:, 0]], xy[bnd[:, 1]]
    side = np.zeros(bnd.shape[0], bool)
    for k in (0, 1):
        for val in (0.0, 1.0):
            side |= (pa[:, k] == val) & (pb[:, k] == val)
    if not side.all():
        i = int(np.nonzero(~side)[0][0])
        return False, f"boundary edge off the square {bnd[i]}"
    corners = {(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (1.0, 1.0)}
    have = {(float(x), float(y)) for x, y in xy}
    if not corners <= have:
        return False, "corner missing"
    return True, ""


def fast_conformity(tris, nv):
    """Vectorised conformity for large meshes: every directed edge at most
    once; every vertex referenced; V - E + F == 1."""
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = e[:, 0] * nv + e[:, 1]
    if np.unique(key).size != key.size:
        return False, "duplicate directed edge"
    und = np.unique(np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1]))
    used = np.unique(t)
    if used.size != nv:
        return False, "unreferenced vertex"
    if nv - und.size + t.shape[0] != 1:
        return False, "Euler characteristic"
    return True, ""
