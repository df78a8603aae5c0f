"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test names what it pins: closed forms of the quality functional and the
metric length (Sec. 2.2), published hash test vectors, brute force for the
independent set (Sec. 3.2) and for the collapse/flip rules (Sec. 2.4), the
hand-derived uniform-grid result, round-equals-sequential (Sec. 3.2-3.3) and
mesh invariants.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04694_gb300 import inputs
from tests import meshcheck as MC

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ulps(a, b):
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


# --- hash (Sec. 3.2 priorities) ----------------------------------------------

def test_fmix32_published_vectors():
    # MurmurHash3_x86_32 of the empty input is fmix32(seed); published test
    # vectors: seed 0 -> 0, seed 1 -> 0x514E28B7, seed 0xFFFFFFFF -> 0x81F16F39.
    assert O.fmix32(0) == 0
    assert O.fmix32(1) == 0x514E28B7
    assert O.fmix32(0xFFFFFFFF) == 0x81F16F39


def test_fmix32_no_collisions_sample():
    vals = {O.fmix32(i * 2654435761 & 0xFFFFFFFF) for i in range(20000)}
    assert len(vals) == 20000


# --- metric length and quality closed forms (Sec. 2.2) ----------------------

def iso(h):
    return np.array([1.0 / h ** 2, 0.0, 1.0 / h ** 2])


def test_edge_length_isotropic_and_symmetric():
    h = 0.02
    a, b = np.array([0.1, 0.2]), np.array([0.13, 0.24])
    L = O.edge_length(a, iso(h), b, iso(h))
    assert abs(L - 0.05 / h) <= 4 * math.ulp(L)
    ma, mb = np.array([3.0, 0.5, 2.0]), np.array([1.0, -0.2, 4.0])
    assert O.edge_length(a, ma, b, mb) == O.edge_length(b, mb, a, ma)  # bitwise


def test_edge_length_anisotropic_axis():
    # M = diag(1/h1^2, 1/h2^2): an x-edge of length d has metric length d/h1.
    h1, h2 = 0.01, 0.3
    m = np.array([1 / h1 ** 2, 0.0, 1 / h2 ** 2])
    assert abs(O.edge_length(np.zeros(2), m, np.array([0.02, 0.0]), m) - 2.0) < 1e-14
    assert abs(O.edge_length(np.zeros(2), m, np.array([0.0, 0.6]), m) - 2.0) < 1e-14


def test_edge_length_rotated_anisotropic_closed_form():
    """End metrics R diag(a_i, b_i) R^T sharing the rotation R: their mean is
    R diag((a1+a2)/2, (b1+b2)/2) R^T, so an edge alpha u1 + beta u2 (u1, u2
    the columns of R) has metric length sqrt(((a1+a2)/2) alpha^2 +
    ((b1+b2)/2) beta^2)."""
    rng = np.random.default_rng(11)

    def rotated(th, a, b):
        c, s = math.cos(th), math.sin(th)
        return np.array([a * c * c + b * s * s, (a - b) * c * s, a * s * s + b * c * c])

    for _ in range(200):
        th = rng.uniform(0.0, math.pi)
        a1, b1, a2, b2 = 10.0 ** rng.uniform(-1.0, 4.0, 4)
        al, be = rng.normal(size=2)
        u1 = np.array([math.cos(th), math.sin(th)])
        u2 = np.array([-math.sin(th), math.cos(th)])
        xa = rng.uniform(0.0, 1.0, 2)
        xb = xa + al * u1 + be * u2
        L = O.edge_length(xa, rotated(th, a1, b1), xb, rotated(th, a2, b2))
        ref = math.sqrt(0.5 * (a1 + a2) * al * al + 0.5 * (b1 + b2) * be * be)
        assert abs(L - ref) <= 1e-11 * ref


def equilateral(h, x0=0.3, y0=0.1, rot=0.0):
    pts = []
    for k in range(3):
        a = rot + 2 * math.pi * k / 3
        pts.append([x0 + h / math.sqrt(3) * math.cos(a), y0 + h / math.sqrt(3) * math.sin(a)])
    return np.array(pts)


@pytest.mark.parametrize("rot", [0.0, 0.3, 1.1, 2.5])
def test_quality_equilateral_unit_metric_is_one(rot):
    h = 0.02
    xy = equilateral(h, rot=rot)
    m = np.tile(iso(h), (3, 1))
    for ids in ([0, 1, 2], [5, 9, 7], [11, 3, 8]):
        q = O.tri_quality(ids, xy, m)
        assert abs(q - 1.0) < 1e-13


def test_quality_equilateral_under_anisotropic_metric():
    # Map an equilateral unit-metric triangle by A; metric A^-T M A^-1 keeps q = 1.
    rng = np.random.default_rng(0)
    for _ in range(20):
        A = rng.normal(size=(2, 2)) + 3 * np.eye(2)
        if np.linalg.det(A) <= 0:
            A[:, 0] *= -1
        xy0 = equilateral(1.0)
        xy = xy0 @ A.T
        Ai = np.linalg.inv(A)
        M = Ai.T @ np.eye(2) @ Ai
        m = np.tile([M[0, 0], M[0, 1], M[1, 1]], (3, 1))
        assert abs(O.tri_quality([0, 1, 2], xy, m) - 1.0) < 1e-12


def test_quality_right_isosceles_closed_form():
    # legs a, hypotenuse a*sqrt2, unit metric: P = a(2+sqrt2), area a^2/2,
    # q = 12 sqrt3 (a^2/2) / P^2 * F(P/3).
    for a in (0.5, 3.0 / (2 + math.sqrt(2)), 1.3):
        xy = np.array([[0.0, 0.0], [a, 0.0], [0.0, a]])
        m = np.tile([1.0, 0.0, 1.0], (3, 1))
        P = a * (2 + math.sqrt(2))
        x = P / 3
        s = min(x, 1 / x)
        F = (s * (2 - s)) ** 3
        expect = 12 * math.sqrt(3) * (a * a / 2) / P ** 2 * F
        assert abs(O.tri_quality([0, 1, 2], xy, m) - expect) < 1e-14
    # at unit perimeter the value is 6 sqrt3 / (2 + sqrt2)^2
    a = 3.0 / (2 + math.sqrt(2))
    xy = np.array([[0.0, 0.0], [a, 0.0], [0.0, a]])
    q = O.tri_quality([0, 1, 2], xy, np.tile([1.0, 0.0, 1.0], (3, 1)))
    assert abs(q - 6 * math.sqrt(3) / (2 + math.sqrt(2)) ** 2) < 1e-14


def test_quality_affine_invariance():
    rng = np.random.default_rng(1)
    for _ in range(50):
        xy = rng.uniform(0, 1, size=(3, 2))
        if MC.exact_orient(*xy) <= 0:
            xy = xy[[0, 2, 1]]
        Ms = []
        for _k in range(3):
            B = rng.normal(size=(2, 2))
            Ms.append(B @ B.T + 0.5 * np.eye(2))
        m = np.array([[M[0, 0], M[0, 1], M[1, 1]] for M in Ms])
        A = rng.normal(size=(2, 2)) + 2 * np.eye(2)
        if np.linalg.det(A) <= 0:
            A[:, 1] *= -1
        Ai = np.linalg.inv(A)
        m2 = []
        for M in Ms:
            N = Ai.T @ M @ Ai
            m2.append([N[0, 0], N[0, 1], N[1, 1]])
        q1 = O.tri_quality([0, 1, 2], xy, m)
        q2 = O.tri_quality([0, 1, 2], xy @ A.T, np.array(m2))
        assert abs(q1 - q2) <= 1e-12 * abs(q1)


def test_quality_rotation_of_storage_does_not_matter():
    rng = np.random.default_rng(2)
    xy = np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.9]])
    m = np.array([[2.0, 0.3, 1.0], [1.5, -0.1, 2.0], [1.0, 0.0, 1.0]])
    ids = np.array([4, 9, 2])
    q = O.tri_quality(ids, xy, m)
    for s in (1, 2):
        perm = [(s + i) % 3 for i in range(3)]
        assert O.tri_quality(ids[perm], xy[perm], m[perm]) == q  # bitwise
    del rng


# --- gradient (quality functional derivative) --------------------------------

def random_triangle(rng):
    xy = rng.uniform(0, 1, size=(3, 2))
    if MC.exact_orient(*xy) <= 0:
        xy = xy[[0, 2, 1]]
    m = []
    for _ in range(3):
        B = rng.normal(size=(2, 2))
        M = B @ B.T + 0.3 * np.eye(2)
        m.append([M[0, 0], M[0, 1], M[1, 1]])
    return xy, np.array(m) * rng.uniform(1, 50)


def test_gradient_central_differences():
    rng = np.random.default_rng(3)
    ids = np.array([7, 3, 5])
    worst = 0.0
    for _ in range(40):
        xy, m = random_triangle(rng)
        q, g = O.tri_quality_grad(ids, xy, m)
        assert q == O.tri_quality(ids, xy, m)
        fd = np.zeros((3, 5))
        for v in range(3):
            for j in range(5):
                base = xy[v, j] if j < 2 else m[v, j - 2]
                h = 1e-6 * max(abs(base), 1e-3)
                xp, mp = xy.copy(), m.copy()
                xm, mm = xy.copy(), m.copy()
                if j < 2:
                    xp[v, j] += h
                    xm[v, j] -= h
                else:
                    mp[v, j - 2] += h
                    mm[v, j - 2] -= h
                fd[v, j] = (O.tri_quality(ids, xp, mp) - O.tri_quality(ids, xm, mm)) / (2 * h)
        # compare per component class (coordinates / metric) in relative norm
        for sl in (slice(0, 2), slice(2, 5)):
            err = np.linalg.norm(g[:, sl] - fd[:, sl]) / max(np.linalg.norm(fd[:, sl]), 1e-300)
            worst = max(worst, err)
    assert worst < 1e-6


def test_gradient_matches_autodiff():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    ids = [2, 0, 1]  # canonical rotation starts at stored slot 1

    def q_torch(xy, m):
        order = [1, 2, 0]
        p, mm = xy[order], m[order]
        k = (mm[0] + mm[1] + mm[2]) / 3.0
        P = 0
        for a, b in ((0, 1), (1, 2), (2, 0)):
            d = p[b] - p[a]
            P = P + torch.sqrt(k[0] * d[0] * d[0] + 2 * k[1] * d[0] * d[1] + k[2] * d[1] * d[1])
        o = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[1, 1] - p[0, 1]) * (p[2, 0] - p[0, 0])
        AM = torch.sqrt(k[0] * k[2] - k[1] * k[1]) * 0.5 * o
        x = P / 3.0
        s = torch.where(x <= 1.0, x, 1.0 / x)
        F = (s * (2.0 - s)) ** 3
        return 12.0 * math.sqrt(3.0) * AM / (P * P) * F

    for _ in range(40):
        xy, m = random_triangle(rng)
        q, g = O.tri_quality_grad(np.array(ids), xy, m)
        txy = torch.tensor(xy, dtype=torch.float64, requires_grad=True)
        tm = torch.tensor(m, dtype=torch.float64, requires_grad=True)
        tq = q_torch(txy, tm)
        tq.backward()
        ref = np.concatenate([txy.grad.numpy(), tm.grad.numpy()], axis=1)
        assert abs(float(tq.detach()) - q) <= 1e-13 * abs(q)
        assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)


# --- independent set (Sec. 3.2) -----------------------------------------------

def test_independent_set_brute_force():
    w = inputs.psi_workload(9, 300, True, 7)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    nv = w.xy.shape[0]
    NN, _ = MC.adjacency([tuple(t) for t in w.tri], nv)
    rng = np.random.default_rng(5)
    for trial in range(30):
        cand = (rng.uniform(size=nv) < rng.uniform(0.2, 1.0)).astype(np.uint8)
        seed, r = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 1000))
        S = om.independent_set(cand, seed, r)
        pr = [O.prio(v, seed, r) for v in range(nv)]
        for v in range(nv):
            local_max = bool(cand[v]) and all(not cand[u] or pr[u] < pr[v] for u in NN[v])
            assert bool(S[v]) == local_max
            if S[v]:
                assert not any(S[u] for u in NN[v])  # independence
        if cand.any():
            assert S.any()  # the global maximum candidate is always selected


@pytest.mark.parametrize("seed", [12345, 2 ** 32 - 7])
def test_first_collapse_round_uses_round_zero_priorities(seed):
    """S5: r counts a call's rounds from 0, so the first round ranks vertices
    by fmix32(v ^ seed) (fmix32 pinned by the published vectors).  The
    vertices that die in a one-round collapse call are exactly the local
    maxima of that priority among the vertices with a valid collapse."""
    w = inputs.psi_workload(17, 1000, True, 3)  # coarser target: many collapses
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    nv = w.xy.shape[0]
    NN, _ = MC.adjacency([tuple(int(a) for a in t) for t in w.tri], nv)
    p = O.make_params(seed=seed)
    cand = {v for v in range(nv) if om.coarsen_target(v, p) >= 0}
    pr = {v: O.fmix32(v ^ seed) for v in cand}
    S = {v for v in cand if all(u not in cand or pr[u] < pr[v] for u in NN[v])}
    assert len(S) > 8
    st = om.coarsen(O.make_params(seed=seed, max_rounds=1))
    assert st["collapses"] == len(S)
    dead = set(np.nonzero(om.get_raw()["valive"] == 0)[0].tolist())
    assert dead == S


# --- small uniform case: hand-derived result ---------------------------------

def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = v.strip()
    return vals


def test_small_uniform_exact_result():
    g = read_golden("small_uniform_counts.txt")
    w = inputs.small_uniform()
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    st = om.adapt(O.make_params())
    xy, tri, m = om.get_mesh()
    assert xy.shape[0] == int(g["vertices"])
    assert tri.shape[0] == int(g["triangles"])
    assert st["splits"] == int(g["splits"])
    assert st["collapses"] == int(g["collapses"]) and st["flips"] == int(g["flips"])
    assert st["moves"] == int(g["moves"]) and st["converged"] == 1
    ok, why = MC.unit_square_ok(xy, tri)
    assert ok, why
    assert MC.fast_conformity(tri, xy.shape[0])[0]


# --- refinement templates (Sec. 2.4.2) ---------------------------------------

def _single_triangle_refine(xy, m, L_up):
    om = O.OracleMesh(xy, np.array([[0, 1, 2]])).set_metric(m)
    om.refine(O.make_params(L_low=1e-9, L_up=L_up, max_rounds=1))
    return om.get_mesh()


def test_refine_three_splits_gives_four_equal_children():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.25, 0.75]])
    m = np.tile([1.0, 0.0, 1.0], (3, 1))
    oxy, tri, om_ = _single_triangle_refine(xy, m, 0.5)
    assert tri.shape[0] == 4 and oxy.shape[0] == 6
    p = oxy[tri]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert np.all(area == 0.375 / 4)  # dyadic coordinates: exact
    mids = {tuple(r) for r in oxy[3:]}
    assert mids == {(0.5, 0.0), (0.625, 0.375), (0.125, 0.375)}


def test_refine_one_and_two_splits():
    # anisotropic metric makes only x-extended edges long
    m = np.tile([100.0, 0.0, 0.01], (3, 1))
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    oxy, tri, _ = _single_triangle_refine(xy, m, 5.0)  # edges with |dx| = 1 exceed
    # edges (0,1) and (1,2) have |dx| = 1 -> two splits -> three children
    assert tri.shape[0] == 3 and oxy.shape[0] == 5
    assert MC.valid_triangulation(oxy, [tuple(t) for t in tri])[0]
    m2 = np.tile([100.0, 0.0, 0.01], (3, 1))
    xy2 = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0]])
    oxy2, tri2, _ = _single_triangle_refine(xy2, m2, 5.0)  # only (0,1),(2,0) have |dx|=1
    assert tri2.shape[0] == 3
    m3 = np.tile([1.0, 0.0, 100.0], (3, 1))
    oxy3, tri3, _ = _single_triangle_refine(xy2, m3, 5.0)  # only (1,2) has |dy| = 1 ... and (2,0)
    assert tri3.shape[0] == 3
    xy4 = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 0.05]])
    oxy4, tri4, _ = _single_triangle_refine(xy4, m3, 5.0)  # no |dy| = 1 edge
    assert tri4.shape[0] == 1
    xy5 = np.array([[0.0, 0.0], [0.05, 0.0], [0.05, 1.0]])
    oxy5, tri5, _ = _single_triangle_refine(xy5, m3, 5.0)  # (1,2),(2,0) long
    assert tri5.shape[0] == 3
    xy6 = np.array([[0.0, 0.0], [0.05, 0.5], [0.0, 1.0]])
    oxy6, tri6, _ = _single_triangle_refine(xy6, m3, 7.5)  # only (2,0) has |dy| = 1
    assert tri6.shape[0] == 2 and oxy6.shape[0] == 4


def test_refine_two_splits_cut_along_the_metric_shorter_diagonal():
    """S11: with two edges split, the trapezoid beside the corner child is cut
    along its diagonal that is shorter in the metric, which need not be the
    Euclidean shorter one."""
    pts = {"A": (0.0, 0.0), "B": (4.0, 0.0), "C": (0.0, 1.5), "mAB": (2.0, 0.0),
           "mBC": (2.0, 0.75)}
    xy = np.array([pts["A"], pts["B"], pts["C"]])  # AB and BC too long, CA not
    u = np.array([2.0, 0.75]) / math.hypot(2.0, 0.75)
    M_dir = np.outer(u, u) + 0.1 * np.eye(2)  # lengths along A -> mBC count most
    # Euclidean: |A mBC| = 2.14 < |mAB C| = 2.5; in M_dir: 2.24 > 1.56
    for M, want, other in ((np.eye(2), ("A", "mBC"), ("mAB", "C")),
                           (M_dir, ("mAB", "C"), ("A", "mBC"))):
        m = np.tile([M[0, 0], M[0, 1], M[1, 1]], (3, 1))
        oxy, tri, _ = _single_triangle_refine(xy, m, 2.0)
        assert tri.shape[0] == 3 and oxy.shape[0] == 5
        idx = {k: int(np.nonzero((oxy == np.array(v)).all(axis=1))[0][0]) for k, v in pts.items()}
        edges = {frozenset((int(t[i]), int(t[(i + 1) % 3]))) for t in tri for i in range(3)}
        assert frozenset((idx[want[0]], idx[want[1]])) in edges
        assert frozenset((idx[other[0]], idx[other[1]])) not in edges


def test_refine_midpoints_reproduce_a_linear_metric_field():
    """A new vertex takes the mean of its edge's end metrics (S11): a metric
    field linear in (x, y) is reproduced exactly at every midpoint (dyadic
    coordinates and coefficients keep the arithmetic exact)."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.25, 0.75]])
    m0, mx, my = np.array([4.0, 0.5, 3.0]), np.array([2.0, -0.25, 1.0]), np.array([-1.0, 0.75, 2.0])
    m = np.array([m0 + p[0] * mx + p[1] * my for p in xy])
    oxy, tri, om_ = _single_triangle_refine(xy, m, 0.5)
    assert oxy.shape[0] == 6
    for p, mm in zip(oxy, om_):
        np.testing.assert_array_equal(mm, m0 + p[0] * mx + p[1] * my)


# --- brute force for the collapse and flip rules (Sec. 2.4.1, 2.4.3) ---------

def tiny_meshes():
    out = []
    for n, seed in ((5, 11), (6, 12), (6, 13), (7, 14)):
        xy, tri = inputs.grid_mesh(n)
        xy = inputs.jitter_interior(xy, n, 0.3 / (n - 1), seed)
        rng = np.random.default_rng(seed)
        m = []
        for _ in range(xy.shape[0]):
            th = rng.uniform(0, math.pi)
            h1 = (1.0 / (n - 1)) * rng.uniform(1.0, 4.0)
            h2 = h1 * rng.uniform(1.0, 3.0)
            c, s = math.cos(th), math.sin(th)
            a, b = 1 / h1 ** 2, 1 / h2 ** 2
            m.append([a * c * c + b * s * s, (a - b) * c * s, a * s * s + b * c * c])
        out.append((xy, tri, np.array(m)))
    return out


def grid_random_diagonals(n, seed):
    """Unjittered n x n grid of the unit square (n - 1 a power of two, so the
    coordinates are exact), each square cut along a random diagonal, with
    random anisotropic metrics as in tiny_meshes: many exactly collinear
    vertex triples, so some collapses would leave a zero-area element."""
    rng = np.random.default_rng(seed)
    g = np.arange(n) / (n - 1)
    xy = np.array([[x, y] for y in g for x in g])
    tri = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            tri += [(a, b, c), (a, c, d)] if rng.random() < 0.5 else [(a, b, d), (b, c, d)]
    m = []
    for _ in range(xy.shape[0]):
        th = rng.uniform(0, math.pi)
        h1 = (1.0 / (n - 1)) * rng.uniform(1.0, 4.0)
        h2 = h1 * rng.uniform(1.0, 3.0)
        c_, s_ = math.cos(th), math.sin(th)
        a_, b_ = 1 / h1 ** 2, 1 / h2 ** 2
        m.append([a_ * c_ * c_ + b_ * s_ * s_, (a_ - b_) * c_ * s_, a_ * s_ * s_ + b_ * c_ * c_])
    return xy, np.array(tri, dtype=np.int32), np.array(m)


def brute_collapse_valid(xy, tris, corner, v, w, L_up, elen, flat_ok=False):
    """Collapse of v onto w checked on the triangulation it would leave, in
    exact arithmetic; flat_ok accepts elements of zero area (for counting the
    cases where that requirement decides)."""
    NN, NE = MC.adjacency(tris, xy.shape[0])
    bedges = MC.boundary_edges(tris)
    bverts = {a for e in bedges for a in e}
    is_bedge = (v, w) in bedges or (w, v) in bedges
    if corner[v]:
        return False
    if v in bverts and not is_bedge:
        return False
    new = []
    for t in tris:
        if v in t and w in t:
            continue
        new.append(tuple(w if a == v else a for a in t))
    if flat_ok:
        if any(MC.exact_orient(xy[t[0]], xy[t[1]], xy[t[2]]) < 0 for t in new):
            return False
        ok, _ = MC.valid_triangulation(xy, new, exact=False)
    else:
        ok, _ = MC.valid_triangulation(xy, new)
    if not ok:
        return False
    if MC.total_area_exact(xy, new) != MC.total_area_exact(xy, tris):
        return False
    nb = MC.boundary_edges(new)
    for a, b in nb:
        if not MC.on_square_side(xy[a], xy[b]):
            return False
    for x in NN[v]:
        if x != w and x not in NN[w] and elen(w, x) > L_up:
            return False
    return True


# L_up = 1.3 makes rule (iii) (no new edge longer than L_up) decide cases too;
# L_low = 0.5 makes the candidate bound decide cases: vertices with no valid
# collapse below L_low but a valid one below 2 L_low (counted); with the first
# bounds, unjittered grids make rule (ii)'s strict orientation decide cases:
# vertices whose target would change if a zero-area element were allowed
# (counted)
@pytest.mark.parametrize("L_low,L_up", [(1.0, 2.5), (1.0, 1.3), (0.5, 2.5)])
def test_collapse_rule_brute_force(L_low, L_up):
    checked = 0
    by_iii = 0  # candidates rejected by rule (iii) alone
    by_low = 0  # vertices whose only valid collapses lie in [L_low, 2 L_low)
    by_flat = 0  # vertices whose target a zero-area element would change
    grids = L_low == 1.0 and L_up == 2.5  # the unjittered grids: once
    meshes = tiny_meshes() + ([grid_random_diagonals(9, s) for s in range(41, 47)] if grids else [])
    for xy, tri, m in meshes:
        om = O.OracleMesh(xy, tri).set_metric(m)
        tris = [tuple(int(a) for a in t) for t in tri]
        raw = om.get_raw()
        corner = (raw["vflag"] & 2) > 0
        NN, _ = MC.adjacency(tris, xy.shape[0])
        bedges = MC.boundary_edges(tris)
        bverts = {a for e in bedges for a in e}
        p = O.make_params(L_low=L_low, L_up=L_up)

        def elen(a, b):
            return O.edge_length(xy[a], m[a], xy[b], m[b])

        for v in range(xy.shape[0]):
            cands, near = [], []
            for w in sorted(NN[v]):
                if v in bverts and not ((v, w) in bedges or (w, v) in bedges):
                    continue
                L = elen(v, w)
                if L < p.L_low:
                    cands.append((L, w))
                elif L < 2.0 * p.L_low:
                    near.append(w)
            cands.sort()
            expect = -1
            if not corner[v]:
                for L, w in cands:
                    if brute_collapse_valid(xy, tris, corner, v, w, p.L_up, elen):
                        expect = w
                        break
                    by_iii += brute_collapse_valid(xy, tris, corner, v, w, math.inf, elen)
                if expect < 0:
                    by_low += any(brute_collapse_valid(xy, tris, corner, v, w, p.L_up, elen)
                                  for w in near)
                flat = next((w for L, w in cands if brute_collapse_valid(
                    xy, tris, corner, v, w, p.L_up, elen, flat_ok=True)), -1)
                by_flat += flat != expect
            assert om.coarsen_target(v, p) == expect, (v, cands)
            checked += len(cands)
    assert checked > 50
    if grids:
        assert by_flat > 5, by_flat
    if L_up < 2.0:
        assert by_iii > 5
    if L_low < 1.0:
        assert by_low > 5, by_low


def test_flip_needs_a_strict_gain():
    """Sec. 2.4.3: an edge is flipped only when the flip raises the minimum
    quality.  On unjittered grids under a uniform metric every element is a
    right isosceles triangle and a flip of a square's diagonal gives two
    congruent ones (gain zero, up to the summation order of the perimeter):
    with every edge listed, no flip is made."""
    for n, seed in ((5, 41), (9, 42), (17, 43)):
        xy, tri, _ = grid_random_diagonals(n, seed)
        m = np.tile([float((n - 1) ** 2), 0.0, float((n - 1) ** 2)], (xy.shape[0], 1))
        om = O.OracleMesh(xy, tri).set_metric(m)
        st = om.swap(O.make_params(q_thresh=1.01, max_rounds=500))
        assert st["flips"] == 0, (n, st)
        np.testing.assert_array_equal(om.get_raw()["tri"], tri)


# q_thresh = 1 lists every edge; on these meshes the improving flips have old
# qualities from 0.03 to 0.67 (median 0.14), so 0.15 lets the threshold decide
@pytest.mark.parametrize("q_thresh", [1.0, 0.15])
def test_flip_rule_brute_force(q_thresh):
    n_flip = 0
    by_thresh = 0  # flips with a positive gain that the threshold rules out
    for xy, tri, m in tiny_meshes():
        om = O.OracleMesh(xy, tri).set_metric(m)
        tris = [tuple(int(a) for a in t) for t in tri]
        NN, NE = MC.adjacency(tris, xy.shape[0])
        p = O.make_params(q_thresh=q_thresh)

        def q_of(t):
            return O.tri_quality(np.array(t), xy[list(t)], m[list(t)])

        for v in range(xy.shape[0]):
            best, bw = None, -1
            for w in sorted(NN[v]):
                K1 = [t for t in tris if any(t[i] == v and t[(i + 1) % 3] == w for i in range(3))]
                K2 = [t for t in tris if any(t[i] == w and t[(i + 1) % 3] == v for i in range(3))]
                if not K1 or not K2:
                    continue
                c = [a for a in K1[0] if a not in (v, w)][0]
                d = [a for a in K2[0] if a not in (v, w)][0]
                if c in NN[d]:
                    continue
                T1, T2 = (v, d, c), (d, w, c)
                if not (MC.exact_orient(xy[v], xy[d], xy[c]) > 0
                        and MC.exact_orient(xy[d], xy[w], xy[c]) > 0):
                    continue
                qold = min(q_of(K1[0]), q_of(K2[0]))
                if not qold < p.q_thresh:
                    by_thresh += min(q_of(T1), q_of(T2)) - qold > 0
                    continue
                gain = min(q_of(T1), q_of(T2)) - qold
                if gain > 0 and (best is None or gain > best):
                    best, bw = gain, w
            got, c, d = om.swap_target(v, p)
            assert got == bw, v
            n_flip += got >= 0
    assert n_flip > 20
    if q_thresh < 1.0:
        assert by_thresh > 5


def test_flip_never_recreates_an_existing_edge():
    """S10: a flip at a degree-3 vertex would join its two opposite vertices a
    second time (and, the quad being non-convex, invert an element).  A point
    P near corner A of triangle ABC, joined to the corners, has three poor
    elements (q_thresh = 1 lists every edge); no flip is taken."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.08, 0.07]])  # A, B, C, P
    tri = np.array([[0, 1, 3], [1, 2, 3], [2, 0, 3]])
    m = np.tile([1.0, 0.0, 1.0], (4, 1))
    om = O.OracleMesh(xy, tri).set_metric(m)
    p = O.make_params(q_thresh=1.0)
    for v in range(4):
        assert om.swap_target(v, p)[0] == -1, v


@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (25, 8000, 22)])
def test_passes_end_with_nothing_left_to_do(n, T, seed):
    """Propagation (Sec. 2.4.5): a collapse or flip pass loops until nothing
    changes, so when it returns no live vertex has a valid collapse, or an
    improving flip, left.  A change whose neighbours were not marked for
    re-evaluation leaves one behind."""
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    p = O.make_params(seed=seed)
    om.refine(p)
    assert om.coarsen(p)["collapses"] > 100
    alive = np.nonzero(om.get_raw()["valive"])[0]
    assert all(om.coarsen_target(int(v), p) < 0 for v in alive)
    assert om.swap(p)["flips"] > 100
    alive = np.nonzero(om.get_raw()["valive"])[0]
    assert all(om.swap_target(int(v), p)[0] < 0 for v in alive)


@pytest.mark.parametrize("n,T,seed", [(9, 4000, 5), (17, 20000, 21)])
def test_refinement_ends_with_no_edge_too_long(n, T, seed):
    """Refinement (Sec. 2.4.2) splits every edge longer than L_up and repeats
    until none is left: when it returns, every edge is at most L_up."""
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    p = O.make_params(seed=seed)
    st = om.refine(p)
    assert st["rounds"] > 2
    raw = om.get_raw()
    xy, m = raw["xy"], raw["m"]
    edges = {tuple(sorted((int(t[i]), int(t[(i + 1) % 3]))))
             for t, a in zip(raw["tri"], raw["talive"]) if a for i in range(3)}
    longest = max(O.edge_length(xy[a], m[a], xy[b], m[b]) for a, b in edges)
    assert longest <= p.L_up


# --- round-equals-sequential and invariants ---------------------------------

@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (25, 8000, 22), (33, 20000, 2)])
def test_round_equals_sequential_and_invariants(n, T, seed):
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    om.set_check_sequential(True)
    st = om.adapt(O.make_params(seed=seed))
    assert not om.seq_failed()
    assert om.check() == 0
    xy, tri, m = om.get_mesh()
    ok, why = MC.unit_square_ok(xy, tri)
    assert ok, why
    assert MC.fast_conformity(tri, xy.shape[0])[0]
    assert st["collapses"] > 0 and st["flips"] > 0 and st["splits"] > 0 and st["moves"] > 0


@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (25, 8000, 22)])
def test_adapt_is_algorithm_1(n, T, seed):
    """Algorithm 1 (Sec. 2.3) written out with the single-operator calls:
    repeat {coarsen; swap; refine} (renumbering after each iteration) until
    an iteration changes nothing or max_iter, then smooth.  Each call starts
    its round counter at 0, and seed_r = seed + 0x9E3779B9 r, so a call given
    seed + 0x9E3779B9 r0 continues a counter that stood at r0.  The mesh and
    the counters equal those of one adapt call."""
    w = inputs.psi_workload(n, T, True, seed)
    a = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    sa = a.adapt(O.make_params(seed=seed))
    b = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    r0 = 0
    tot = dict(collapses=0, flips=0, splits=0, moves=0)
    iters = 0

    def run(op, key):
        nonlocal r0
        st = op(O.make_params(seed=(seed + 0x9E3779B9 * r0) & 0xFFFFFFFF))
        r0 += st["rounds"]
        tot[key] += st[key]
        return st[key]

    for _ in range(O.make_params().max_iter):
        iters += 1
        changed = run(b.coarsen, "collapses") + run(b.swap, "flips") + run(b.refine, "splits")
        b.renumber()
        if changed == 0:
            break
    run(b.smooth, "moves")
    assert iters >= 2
    for x, y in zip(a.get_mesh(), b.get_mesh()):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))
    for k, v in tot.items():
        assert sa[k] == v, (k, sa[k], v)
    assert sa["rounds"] == r0


def test_operators_keep_invariants_round_by_round():
    w = inputs.psi_workload(21, 6000, True, 9)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    om.set_check_sequential(True)
    for op in ("refine", "coarsen", "swap", "refine", "coarsen", "swap", "smooth"):
        for _ in range(3):
            getattr(om, op)(O.make_params(seed=9, max_rounds=2))
            assert om.check() == 0, op
    assert not om.seq_failed()


# --- smoothing (Sec. 2.4.4) ---------------------------------------------------

def hex_patch(offset):
    """Centre vertex 0 with a regular hexagon ring 1..6 (radius 1)."""
    ring = [[math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)] for k in range(6)]
    xy = np.array([[offset[0], offset[1]]] + ring)
    tri = np.array([[0, 1 + k, 1 + (k + 1) % 6] for k in range(6)])
    return xy, tri


def test_laplacian_smoothing_moves_to_centroid_uniform_metric():
    xy, tri = hex_patch((0.21, -0.13))
    m = np.tile([1.0, 0.0, 1.0], (7, 1))
    om = O.OracleMesh(xy, tri).set_metric(m)
    q_before = om.quality_elems().min()
    st = om.smooth(O.make_params(q_thresh=1.01, max_smooth_sweeps=1))
    raw = om.get_raw()
    assert st["moves"] == 1
    assert np.abs(raw["xy"][0]).max() < 1e-15  # centroid of the ring is the origin
    np.testing.assert_array_equal(raw["m"][0], [1.0, 0.0, 1.0])
    assert om.quality_elems().min() > q_before


def test_laplacian_smoothing_metric_weighted_target():
    # Ring metric is uniform (A); the centre carries metric B.  With every edge
    # metric W = (A + B)/2 identical, the weighted mean is the plain centroid.
    xy, tri = hex_patch((0.1, 0.05))
    m = np.tile([2.0, 0.5, 3.0], (7, 1))
    m[0] = [1.0, -0.2, 1.5]
    om = O.OracleMesh(xy, tri).set_metric(m)
    om.smooth(O.make_params(q_thresh=1.01, max_smooth_sweeps=1))
    raw = om.get_raw()
    if raw["xy"][0].any():
        assert np.abs(raw["xy"][0]).max() < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_smoothing_target_moves_with_the_patch(seed):
    """The metric-weighted Laplacian target (S12) is covariant: translating the
    patch translates the new position, and rotating points and metrics
    together (M -> R M R^T) rotates it.  Varying metrics keep the weighted
    mean away from the plain centroid."""
    rng = np.random.default_rng(seed)
    m = np.array([[1.0 + rng.uniform(-0.3, 0.3), rng.uniform(-0.2, 0.2), 1.0 + rng.uniform(-0.3, 0.3)]
                  for _ in range(7)])
    xy, tri = hex_patch((0.3, -0.2))
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])

    def rotated(mm):
        Mr = R @ np.array([[mm[0], mm[1]], [mm[1], mm[2]]]) @ R.T
        return [Mr[0, 0], Mr[0, 1], Mr[1, 1]]

    def new_centre(pts, mets):
        om = O.OracleMesh(pts, tri).set_metric(mets)
        assert om.smooth(O.make_params(q_thresh=1.01, max_smooth_sweeps=1))["moves"] == 1
        return om.get_raw()["xy"][0]

    X = new_centre(xy, m)
    assert np.linalg.norm(X - xy[0]) > 0.1
    t = np.array([0.25, -0.125])
    np.testing.assert_allclose(new_centre(xy + t, m) - t, X, atol=1e-14)
    np.testing.assert_allclose(R.T @ new_centre(xy @ R.T, np.array([rotated(r) for r in m])), X,
                               atol=1e-14)


def test_smoothing_interpolates_a_linear_metric_field_exactly():
    """Barycentric interpolation (S12) reproduces a field that is linear in
    (x, y): the moved vertex's new metric is the field at its new place."""
    m0, mx, my = np.array([4.0, 0.3, 5.0]), np.array([0.5, 0.1, -0.4]), np.array([-0.3, 0.2, 0.6])

    def field(p):
        return m0 + p[0] * mx + p[1] * my

    for off in ((0.21, -0.13), (-0.3, 0.17), (0.05, 0.33)):
        xy, tri = hex_patch(off)
        m = np.array([field(p) for p in xy])
        om = O.OracleMesh(xy, tri).set_metric(m)
        st = om.smooth(O.make_params(q_thresh=1.01, max_smooth_sweeps=1))
        assert st["moves"] == 1, off
        raw = om.get_raw()
        x_new = raw["xy"][0]
        assert np.abs(x_new - np.array(off)).max() > 1e-3  # it moved
        np.testing.assert_allclose(raw["m"][0], field(x_new), rtol=1e-13, atol=1e-13)
        # the ring keeps its metric
        np.testing.assert_array_equal(raw["m"][1:], m[1:])


def test_smoothing_moves_only_for_a_strict_gain():
    """A vertex already at its Laplacian target would gain nothing by moving:
    no move is made (smoothing must raise the local quality, Sec. 2.4.4).
    The centre of the diamond (+-1, 0), (0, +-1) under a uniform metric is
    its neighbours' mean exactly, so the evaluated move goes nowhere and its
    ball keeps every quality bit for bit."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, -1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 4], [0, 4, 1]])
    m = np.tile([1.0, 0.0, 1.0], (5, 1))
    om = O.OracleMesh(xy, tri).set_metric(m)
    st = om.smooth(O.make_params(q_thresh=1.01, max_smooth_sweeps=3))
    assert st["moves"] == 0
    np.testing.assert_array_equal(om.get_raw()["xy"], xy)


@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (21, 6000, 9)])
def test_smoothing_sweeps_leave_only_moved_vertices_movable(n, T, seed):
    """S12 propagation: a vertex is evaluated again in the next sweep when a
    neighbour moved, and sweeps stop when one moves nothing.  After such a
    call every vertex that did not move has failed an evaluation made after
    its last neighbour move, so the first round of a fresh call can only move
    vertices the call moved (a moved vertex's own metric changed, so it may
    gain again)."""
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    p = O.make_params(seed=seed)
    om.refine(p)
    om.coarsen(p)
    om.swap(p)
    xy0 = om.get_raw()["xy"].copy()
    st = om.smooth(O.make_params(seed=seed, max_smooth_sweeps=1000))
    xy1 = om.get_raw()["xy"].copy()
    moved1 = set(np.nonzero((xy1 != xy0).any(axis=1))[0].tolist())
    assert st["moves"] > 100
    om.smooth(O.make_params(seed=seed + 1, max_smooth_sweeps=1, max_rounds=1))
    moved2 = set(np.nonzero((om.get_raw()["xy"] != xy1).any(axis=1))[0].tolist())
    assert moved2 and moved2 <= moved1


def test_smoothing_candidates_lie_below_the_quality_threshold():
    """S12 and S14: only a vertex whose ball holds an element of quality below
    q_thresh is smoothed.  A round at q_thresh = 0.5 moves no vertex whose
    ball minimum was at least 0.5; the same round at q_thresh = 1.01 moves
    some of them, so the threshold decides cases (counted)."""
    w = inputs.psi_workload(25, 8000, True, 4)
    counts = {}
    for thresh in (0.5, 1.01):
        om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        p = O.make_params(seed=4)
        om.refine(p)
        om.swap(p)
        raw0 = om.get_raw()
        q = om.quality_elems()
        qmin = np.full(raw0["xy"].shape[0], np.inf)
        for t, alive, qk in zip(raw0["tri"], raw0["talive"], q):
            if alive:
                for a in t:
                    qmin[a] = min(qmin[a], qk)
        om.smooth(O.make_params(seed=4, q_thresh=thresh, max_smooth_sweeps=1, max_rounds=1))
        moved = np.nonzero((om.get_raw()["xy"] != raw0["xy"]).any(axis=1))[0]
        assert moved.size > 0
        counts[thresh] = int((qmin[moved] >= 0.5).sum())
    assert counts[0.5] == 0
    assert counts[1.01] > 5, counts


def test_smoothing_never_lowers_ball_min_quality():
    w = inputs.psi_workload(25, 8000, True, 4)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    p = O.make_params(seed=4)
    om.refine(p)
    om.swap(p)
    q0 = om.quality_elems()
    st = om.smooth(p)
    q1 = om.quality_elems()
    assert st["moves"] > 0
    assert np.nanmin(q1) >= np.nanmin(q0)
    assert om.check() == 0


def test_opt_smoothing_follows_its_step_rule():
    """G2, checked through independent quantities: in one round every moved
    vertex went along the gradient of the quality sum (pinned by finite
    differences), by 0.1 x its shortest incident Euclidean edge x 2^-k,
    k <= 5; its ball's minimum quality did not drop and the sum rose."""
    w = inputs.psi_workload(25, 8000, True, 6)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    om.refine(O.make_params(seed=6))
    raw0 = om.get_raw()
    _, dxy, _ = om.quality(grad=True)
    om.opt_smooth(O.make_params(seed=6, opt_smooth_rounds=1, max_rounds=1))
    raw1 = om.get_raw()
    xy0, xy1 = raw0["xy"], raw1["xy"]
    moved = np.nonzero((xy1 != xy0).any(axis=1))[0]
    assert moved.size > 100
    live = [tuple(int(a) for a in t) for t, a in zip(raw0["tri"], raw0["talive"]) if a]
    ball = {}
    for t in live:
        for a in t:
            ball.setdefault(a, []).append(t)
    ks = set()
    for v in moved:
        d, g = xy1[v] - xy0[v], dxy[v]
        assert abs(d[0] * g[1] - d[1] * g[0]) <= 1e-9 * np.linalg.norm(d) * np.linalg.norm(g)
        assert d @ g > 0
        lmin = min(math.hypot(*(xy0[u] - xy0[v])) for t in ball[v] for u in t if u != v)
        k = -math.log2(np.linalg.norm(d) / (0.1 * lmin))
        assert abs(k - round(k)) < 1e-9 and 0 <= round(k) <= 5, k
        ks.add(round(k))
        q0 = [O.tri_quality(np.array(t), xy0[list(t)], raw0["m"][list(t)]) for t in ball[v]]
        q1 = [O.tri_quality(np.array(t), xy1[list(t)], raw1["m"][list(t)]) for t in ball[v]]
        assert min(q1) >= min(q0) and sum(q1) > sum(q0)
    assert 0 in ks and len(ks) > 2


def test_opt_smoothing_increases_quality_sum():
    w = inputs.psi_workload(25, 8000, True, 6)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    p = O.make_params(seed=6, opt_smooth_rounds=20)
    om.refine(p)
    s0 = om.quality(grad=False)
    qmin0 = np.nanmin(om.quality_elems())
    st = om.opt_smooth(p)
    assert st["moves"] > 0
    assert om.quality(grad=False) > s0
    assert np.nanmin(om.quality_elems()) >= qmin0
    assert om.check() == 0


# --- mesh-level gradient -------------------------------------------------------

def test_mesh_gradient_central_differences():
    w = inputs.psi_workload(9, 300, True, 8)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    qs, dxy, dm = om.quality()
    rng = np.random.default_rng(8)
    for v in rng.choice(w.xy.shape[0], 10, replace=False):
        for j in range(5):
            xy, m = w.xy.copy(), w.m.copy()
            # step relative to the local scale: the shortest incident edge for
            # coordinates, the metric's largest diagonal entry for metric entries
            nbr = np.unique(w.tri[(w.tri == v).any(axis=1)])
            nbr = nbr[nbr != v]
            lmin = np.min(np.hypot(*(w.xy[nbr] - w.xy[v]).T))
            h = 1e-6 * (lmin if j < 2 else max(m[v, 0], m[v, 2]))
            vals = []
            for sgn in (1, -1):
                xy2, m2 = xy.copy(), m.copy()
                if j < 2:
                    xy2[v, j] += sgn * h
                else:
                    m2[v, j - 2] += sgn * h
                o2 = O.OracleMesh(xy2, w.tri).set_metric(m2)
                vals.append(o2.quality(grad=False))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = dxy[v, j] if j < 2 else dm[v, j - 2]
            assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-6)


# --- input generator -----------------------------------------------------------

@pytest.mark.parametrize("step", [0, 7, 31])
def test_psi_hessian_matches_differences(step):
    """The time-dependent field of Sec. 4 at t = step T / 50."""
    phase = inputs.psi_phase(step)
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, 400)
    y = rng.uniform(0, 1, 400)
    D = np.sin(5 * y + phase) - 2 * x
    keep = np.abs(D) > 0.05
    x, y = x[keep], y[keep]
    h = 1e-4
    hxx, hxy, hyy = inputs.psi_hessian(x, y, phase)

    def f(a, b):
        return inputs.psi(a, b, phase)

    fxx = (f(x + h, y) - 2 * f(x, y) + f(x - h, y)) / h ** 2
    fyy = (f(x, y + h) - 2 * f(x, y) + f(x, y - h)) / h ** 2
    fxy = (f(x + h, y + h) - f(x + h, y - h) - f(x - h, y + h) + f(x - h, y - h)) / (4 * h * h)
    for a, b in ((hxx, fxx), (hxy, fxy), (hyy, fyy)):
        assert np.all(np.abs(a - b) <= 1e-3 * (1 + np.abs(a)))


def test_psi_time_steps_are_periodic_and_start_at_the_static_field():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 200)
    y = rng.uniform(0, 1, 200)
    # phase 0 is the time-independent field bit for bit
    assert np.array_equal(inputs.psi(x, y, inputs.psi_phase(0)), inputs.psi(x, y))
    # 50 steps make one period
    assert np.allclose(inputs.psi(x, y, inputs.psi_phase(50)), inputs.psi(x, y), atol=1e-9)
    assert not np.allclose(inputs.psi(x, y, inputs.psi_phase(25)), inputs.psi(x, y), atol=1e-3)


def test_psi_metric_hits_target_estimate():
    w = inputs.psi_workload(65, 1.0e5, True, 2)
    n = inputs.estimated_elements(w.xy, w.tri, w.m)
    assert abs(n / 1.0e5 - 1) < 1e-6
    det = w.m[:, 0] * w.m[:, 2] - w.m[:, 1] ** 2
    assert (w.m[:, 0] > 0).all() and (det > 0).all()


# --- exact orientation signs (reading S3 with robust predicates) -------------

def _exact_orient(p, q, r):
    from fractions import Fraction as F

    px, py, qx, qy, rx, ry = (F(float(v)) for v in (*p, *q, *r))
    d = (qx - px) * (ry - py) - (qy - py) * (rx - px)
    return (d > 0) - (d < 0)


def _orient_cases(n, seed):
    """Nearly collinear triples (r on the line through p and q, rounded, then a
    few units in the last place off it), some far from the origin where the
    differences themselves round; general triples; exactly collinear ones."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        scale = 10.0 ** float(rng.integers(-3, 3))
        offset = (10.0 ** float(rng.integers(0, 9))) * rng.uniform(-1, 1, 2) * rng.integers(0, 2)
        p = rng.uniform(-1, 1, 2) * scale + offset
        q = rng.uniform(-1, 1, 2) * scale + offset
        r = p + rng.uniform(-2, 2) * (q - p)
        for k in range(2):
            for _ in range(int(rng.integers(0, 3))):
                r[k] = np.nextafter(r[k], np.inf if rng.integers(0, 2) else -np.inf)
        out.append((p, q, r))
    for _ in range(n // 4):
        out.append(tuple(rng.uniform(-1, 1, (3, 2))))
    out += [((0.0, 0.0), (1.0, 1.0), (2.0, 2.0)), ((0.1, 0.3), (0.2, 0.3), (0.7, 0.3)),
            ((0.25, 0.5), (0.25, 0.75), (0.25, 0.125)), ((1.0, 2.0), (1.0, 2.0), (3.0, 5.0))]
    return out


def test_orient_sign_exact():
    """The oracle's orientation sign equals the sign of the exact determinant
    of the doubles (rational arithmetic), is invariant under rotation and
    flips under a swap; the sample holds many triples whose rounded formula
    gives the wrong sign, and exactly collinear ones (sign 0)."""
    wrong, zeros = 0, 0
    for p, q, r in _orient_cases(3000, 77):
        e = _exact_orient(p, q, r)
        assert O.orient_sign(p, q, r) == e, (p, q, r)
        assert O.orient_sign(q, r, p) == e and O.orient_sign(r, p, q) == e
        assert O.orient_sign(q, p, r) == -e
        naive = float((q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0]))
        wrong += int((naive > 0) - (naive < 0) != e)
        zeros += e == 0
    assert wrong > 50, wrong
    assert zeros >= 4, zeros


# --- colouring and colour-class sets (Sec. 3.2) --------------------------------

@pytest.mark.parametrize("n,T,seed", [(9, 300, 7), (17, 3000, 8)])
def test_colouring_proper_complete_smallest_free(n, T, seed):
    """The colouring of the vertex graph is proper and complete, every colour
    below a vertex's own is held by one of its neighbours (each vertex takes
    the smallest colour its neighbours coloured before it leave free, and
    those keep their colours), and the local maxima of the priority take
    colour 0 (in the first round every vertex proposes 0 and exactly the
    local maxima keep it)."""
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    nv = w.xy.shape[0]
    NN, _ = MC.adjacency([tuple(int(a) for a in t) for t in w.tri], nv)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        s, r = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 1000))
        col, ncol = om.colour(s, r)
        assert (col >= 0).all() and ncol == col.max() + 1
        pr = [O.prio(v, s, r) for v in range(nv)]
        for v in range(nv):
            assert all(col[u] != col[v] for u in NN[v])
            assert set(range(col[v])) <= {int(col[u]) for u in NN[v]}
            if all(pr[u] < pr[v] for u in NN[v]):
                assert col[v] == 0
        assert ncol <= max(len(a) for a in NN) + 1
        col2, _ = om.colour(s, r)
        assert np.array_equal(col, col2)


def test_colour_class_first_round_collapses_colour_zero_candidates():
    """With colour-class sets the first round of a collapse call takes class
    r mod ncol = 0; a proper class is independent, so every candidate of
    colour 0 collapses and no other vertex does."""
    w = inputs.psi_workload(17, 1000, True, 3)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    nv = w.xy.shape[0]
    seed = 4242
    p = O.make_params(seed=seed, select_mode=1)
    col, _ = om.colour(seed, 0)
    cand = {v for v in range(nv) if om.coarsen_target(v, p) >= 0}
    S = {v for v in cand if col[v] == 0}
    assert len(S) >= 5
    st = om.coarsen(O.make_params(seed=seed, max_rounds=1, select_mode=1))
    assert st["collapses"] == len(S)
    assert set(np.nonzero(om.get_raw()["valive"] == 0)[0].tolist()) == S


def test_colour_class_round_takes_the_whole_class():
    """Sec. 3.2: the classes of a proper colouring are independent sets, so
    the round with counter r takes every candidate of colour r mod ncol and
    nothing else, whatever their priorities against candidates of other
    classes (which the hash rule alone would make lose: counted)."""
    w = inputs.psi_workload(17, 1000, True, 3)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    seed = 4242
    col, ncol = om.colour(seed, 0)
    assert ncol >= 3
    rng = np.random.default_rng(0)
    lose = 0
    for r in range(2 * ncol):
        cand = (rng.random(col.shape[0]) < 0.7).astype(np.uint8)
        cand[col < 0] = 0
        S = om.independent_set(cand, seed, r, by_colour=True).astype(bool)
        expect = (cand == 1) & (col == r % ncol)
        assert np.array_equal(S, expect), r
        lose += int((expect & ~om.independent_set(cand, seed, r).astype(bool)).sum())
    assert lose > 10, lose


@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (25, 8000, 22)])
def test_colour_class_adaptation_round_equals_sequential(n, T, seed):
    w = inputs.psi_workload(n, T, True, seed)
    om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    om.set_check_sequential(True)
    st = om.adapt(O.make_params(seed=seed, select_mode=1))
    assert not om.seq_failed()
    assert om.check() == 0
    xy, tri, m = om.get_mesh()
    ok, why = MC.unit_square_ok(xy, tri)
    assert ok, why
    assert st["collapses"] > 0 and st["flips"] > 0 and st["moves"] > 0
