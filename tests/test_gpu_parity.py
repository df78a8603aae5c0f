"""GPU (CUDA library through the C interface) against the CPU oracle.

Topology and coordinates must match bit for bit (Sec. 3.2-3.3 round
semantics, FP64 without contraction on both sides); the quality sum and
gradient to a relative 1e-12 (different summation order of the mesh total).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04694_gb300 import inputs

pytestmark = pytest.mark.gpu

pm = pytest.importorskip("paper_1505_04694_gb300.pm")


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def assert_same_mesh(g, o, what=""):
    gxy, gtri, gm = g
    oxy, otri, om = o
    assert gtri.shape == otri.shape and gxy.shape == oxy.shape, (what, gtri.shape, otri.shape)
    bad = np.nonzero((gtri != otri).any(axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} triangles differ, first {bad[:5]}"
    bx = np.nonzero((bits(gxy) != bits(oxy)).any(axis=1))[0]
    assert bx.size == 0, f"{what}: {bx.size} vertices differ in coordinates, first {bx[:5]}"
    bm = np.nonzero((bits(gm) != bits(om)).any(axis=1))[0]
    assert bm.size == 0, f"{what}: {bm.size} vertices differ in metric, first {bm[:5]}"


def assert_same_raw(g, o, what=""):
    for k in ("valive", "talive", "vflag", "tri"):
        assert np.array_equal(g[k], o[k]), f"{what}: raw {k} differs"
    alive = g["valive"] > 0
    assert np.array_equal(bits(g["xy"][alive]), bits(o["xy"][alive])), f"{what}: xy"
    assert np.array_equal(bits(g["m"][alive]), bits(o["m"][alive])), f"{what}: metric"


def assert_same_adjacency(gm, om, raw):
    for v in np.nonzero(raw["valive"])[0]:
        a = gm.adjacency(int(v))
        b = om.adjacency(int(v))
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), f"row of vertex {v}"


def both(w, seed):
    g = pm.Mesh.from_host(w.xy, w.tri, device=0)
    g.set_metric(w.m)
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    return g, o


def gp(seed, **kw):
    return pm.Params(seed=seed, **kw)


def op(seed, **kw):
    return O.make_params(seed=seed, **kw)


STAT_KEYS = ("rounds", "collapses", "splits", "flips", "moves", "converged")


def test_small_uniform_adapt_bit_exact():
    w = inputs.small_uniform()
    g, o = both(w, 1)
    sg = g.adapt(gp(1))
    so = o.adapt(op(1))
    assert_same_mesh(g.get_mesh(), o.get_mesh(), "small uniform")
    for k in STAT_KEYS:
        assert sg[k] == so[k], k
    assert g.sizes() == (3281, 6400)


def test_get_mesh_into_pinned_buffers():
    """get_mesh(out=...) into larger page-locked arrays returns the same mesh
    as get_mesh() into fresh arrays, as views of the buffers' first rows."""
    torch = pytest.importorskip("torch")
    w = inputs.psi_workload(17, 3000, True, 21)
    g = pm.Mesh.from_host(w.xy, w.tri, device=0)
    g.set_metric(w.m)
    g.adapt(gp(21))
    ref = g.get_mesh()
    cap = 2 * ref[1].shape[0] + 7
    out = (torch.empty((cap, 2), dtype=torch.float64).pin_memory().numpy(),
           torch.empty((cap, 3), dtype=torch.int32).pin_memory().numpy(),
           torch.empty((cap, 3), dtype=torch.float64).pin_memory().numpy())
    got = g.get_mesh(out=out)
    assert_same_mesh(got, ref, "pinned output")
    assert got[0].ctypes.data == out[0].ctypes.data and got[1].ctypes.data == out[1].ctypes.data
    with pytest.raises(ValueError):
        g.get_mesh(out=(out[0][:3], out[1], out[2]))


# (65, 1500, 3) coarsens most of the mesh in its first iteration: the
# renumbering after it compacts the slots, the later ones keep them in place
@pytest.mark.parametrize("n,T,seed", [(9, 400, 5), (17, 3000, 21), (25, 8000, 22), (33, 20000, 2),
                                      (65, 100000, 2), (65, 1500, 3)])
def test_psi_adapt_bit_exact(n, T, seed):
    w = inputs.psi_workload(n, T, True, seed)
    g, o = both(w, seed)
    sg = g.adapt(gp(seed))
    so = o.adapt(op(seed))
    assert_same_mesh(g.get_mesh(), o.get_mesh(), f"psi {n}")
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])


def test_time_dependent_psi_readapt_bit_exact():
    """Sec. 4's time-dependent benchmark: every time step re-adapts the last
    step's mesh to the metric of psi(x, y, t_k), t_k = k T / 50, evaluated at
    that mesh's vertices."""
    seed = 6
    w = inputs.psi_workload(21, 4000, True, seed)
    g, o = both(w, seed)
    g.adapt(gp(seed))
    o.adapt(op(seed))
    for k in range(1, 4):
        gm, om = g.get_mesh(), o.get_mesh()
        assert_same_mesh(gm, om, f"time step {k - 1}")
        m = inputs.psi_metric(gm[0], gm[1], 4000, phase=inputs.psi_phase(k))
        g.set_metric(m)
        o.set_metric(m)
        sg = g.adapt(gp(seed))
        so = o.adapt(op(seed))
        for key in STAT_KEYS:
            assert sg[key] == so[key], (k, key, sg[key], so[key])
        assert sg["collapses"] + sg["splits"] + sg["flips"] > 0  # the field moved
    assert_same_mesh(g.get_mesh(), o.get_mesh(), "time step 3")


@pytest.mark.parametrize("opname", ["coarsen", "swap", "refine", "smooth", "opt_smooth"])
def test_single_operator_raw_state_and_rows(opname):
    w = inputs.psi_workload(21, 6000, True, 9)
    g, o = both(w, 9)
    # bring the mesh into a state where every operator has work
    for name in ("refine", "coarsen"):
        getattr(g, name)(gp(9))
        getattr(o, name)(op(9))
    kw = dict(opt_smooth_rounds=5) if opname == "opt_smooth" else {}
    sg = getattr(g, opname)(gp(9, **kw))
    so = getattr(o, opname)(op(9, **kw))
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    rg, ro = g.get_raw(), o.get_raw()
    assert_same_raw(rg, ro, opname)
    assert_same_adjacency(g, o, rg)


def test_round_by_round():
    w = inputs.psi_workload(25, 8000, True, 12)
    g, o = both(w, 12)
    for opname in ("refine", "coarsen", "swap", "smooth"):
        for _ in range(4):
            sg = getattr(g, opname)(gp(12, max_rounds=1))
            so = getattr(o, opname)(op(12, max_rounds=1))
            assert sg["rounds"] == so["rounds"]
            rg, ro = g.get_raw(), o.get_raw()
            assert_same_raw(rg, ro, opname)
        assert_same_adjacency(g, o, rg)


def test_quality_and_gradient_against_oracle():
    w = inputs.psi_workload(33, 20000, True, 3)
    g, o = both(w, 3)
    g.refine(gp(3))
    o.refine(op(3))
    qg, dg, mg = g.quality()
    qo, do, mo = o.quality()
    assert abs(qg - qo) <= 1e-12 * abs(qo)
    # the per-vertex sums use the same order on both sides
    assert np.array_equal(bits(dg), bits(do))
    assert np.array_equal(bits(mg), bits(mo))


def test_quality_arrays_and_autograd():
    torch = pytest.importorskip("torch")
    from paper_1505_04694_gb300.autograd import quality

    w = inputs.psi_workload(17, 3000, True, 4)
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    qo, do, mo = o.quality()
    dev = torch.device("cuda:0")
    xy = torch.tensor(w.xy, dtype=torch.float64, device=dev, requires_grad=True)
    m = torch.tensor(w.m, dtype=torch.float64, device=dev, requires_grad=True)
    tri = torch.tensor(w.tri, dtype=torch.int32, device=dev)
    q = quality(xy, m, tri)
    q.backward()
    assert abs(float(q) - qo) <= 1e-12 * abs(qo)
    gx = xy.grad.cpu().numpy()
    gm = m.grad.cpu().numpy()
    assert np.linalg.norm(gx - do) <= 1e-12 * np.linalg.norm(do)
    assert np.linalg.norm(gm - mo) <= 1e-12 * np.linalg.norm(mo)


def test_autograd_gradcheck_small():
    torch = pytest.importorskip("torch")
    from paper_1505_04694_gb300.autograd import QualityFunction

    xy0, tri0 = inputs.grid_mesh(3)  # 8 triangles
    xy0 = inputs.jitter_interior(xy0, 3, 0.1, 7)
    m0 = inputs.uniform_metric(xy0.shape[0], 0.4)
    dev = torch.device("cuda:0")
    xy = torch.tensor(xy0, dtype=torch.float64, device=dev, requires_grad=True)
    m = torch.tensor(m0, dtype=torch.float64, device=dev, requires_grad=True)
    tri = torch.tensor(tri0, dtype=torch.int32, device=dev)
    assert torch.autograd.gradcheck(lambda a, b: QualityFunction.apply(a, b, tri), (xy, m),
                                    eps=1e-7, atol=1e-7, rtol=1e-6)


def test_batch_equals_single_runs():
    ws = [inputs.psi_workload(n, T, True, s) for n, T, s in ((9, 400, 31), (17, 3000, 32),
                                                             (13, 1500, 33))]
    ws.append(inputs.small_uniform())
    meshes = []
    params = []
    for i, w in enumerate(ws):
        g = pm.Mesh.from_host(w.xy, w.tri, device=0)
        g.set_metric(w.m)
        meshes.append(g)
        params.append(gp(w.params.seed))
    stats = pm.adapt_batch(meshes, params)
    for w, g, st in zip(ws, meshes, stats):
        o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        so = o.adapt(op(w.params.seed))
        assert_same_mesh(g.get_mesh(), o.get_mesh(), w.name)
        for k in STAT_KEYS:
            assert st[k] == so[k], (w.name, k, st[k], so[k])


def _small_batch():
    ws = [inputs.psi_workload(n, T, True, s) for n, T, s in ((9, 400, 31), (17, 3000, 32),
                                                             (13, 1500, 33))]
    ws.append(inputs.small_uniform())
    ws += inputs.batch_workloads(count=6, seed=9, tmin=200, tmax=3000)
    return ws


def test_batch_handle_equals_oracle_mesh_by_mesh():
    """One pm_batch_create handle for ten meshes (psi-Hessian, uniform and
    constant anisotropic metrics, each with its own seed): pm_batch_adapt's
    per-mesh results and counters are those of the oracle adapting each mesh
    alone (Sec. 3.2: a round's set over the union of disjoint vertex graphs)."""
    ws = _small_batch()
    b = pm.Batch.from_host([(w.xy, w.tri) for w in ws], device=0)
    assert b.count() == len(ws)
    b.set_metric(np.concatenate([w.m for w in ws]))
    stats = b.adapt([gp(w.params.seed) for w in ws])
    got = b.get_meshes()
    for w, g, st in zip(ws, got, stats):
        o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        so = o.adapt(op(w.params.seed))
        assert_same_mesh(g, o.get_mesh(), w.name)
        for k in STAT_KEYS:
            assert st[k] == so[k], (w.name, k, st[k], so[k])
    # one-mesh calls on a batch handle are refused
    a, c = np.zeros(1, np.int32), np.zeros(1, np.int32)
    assert pm.lib.pm_get_mesh(b.h, pm._i(a), pm._i(c), None, None, None) == 1


@pytest.mark.parametrize("n,T,seed", [(17, 3000, 21), (65, 100000, 2)])
def test_colour_class_adapt_bit_exact(n, T, seed):
    """Colour-class sets (pm_params.select = PM_SELECT_COLOUR): the vertex
    graph coloured at the start of every collapse, flip and smoothing pass,
    one class per round.  Mesh and counters equal the oracle's in the same
    mode, on a mesh that runs in persistent rounds and on one whose first
    rounds take the one-kernel-per-phase path."""
    w = inputs.psi_workload(n, T, True, seed)
    g = pm.Mesh.from_host(w.xy, w.tri, device=0)
    g.set_metric(w.m)
    sg = g.adapt(gp(seed, select=pm.SELECT_COLOUR))
    gm = g.get_mesh()
    g.close()
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    so = o.adapt(op(seed, select_mode=1))
    assert_same_mesh(gm, o.get_mesh(), f"colour classes {n}")
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    # the same mesh with hash-priority sets takes other rounds
    oh = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    assert oh.adapt(op(seed))["rounds"] != so["rounds"]


def test_colour_class_batch_mixed_modes_bit_exact():
    """A batch in which every other mesh uses colour-class sets: each mesh's
    result and counters equal the oracle's in its own mode."""
    ws = _small_batch()
    modes = [i % 2 for i in range(len(ws))]
    b = pm.Batch.from_host([(w.xy, w.tri) for w in ws], device=0)
    b.set_metric(np.concatenate([w.m for w in ws]))
    stats = b.adapt([gp(w.params.seed, select=md) for w, md in zip(ws, modes)])
    got = b.get_meshes()
    b.close()
    for w, g, st, md in zip(ws, got, stats, modes):
        o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        so = o.adapt(op(w.params.seed, select_mode=md))
        assert_same_mesh(g, o.get_mesh(), f"{w.name} mode {md}")
        for k in STAT_KEYS:
            assert st[k] == so[k], (w.name, md, k, st[k], so[k])


def _edge_case_meshes():
    """Small and degenerate inputs: one triangle (three corners), two
    triangles, a strip of slivers 1e-7 high (orientation determinants of
    order 1e-9, where the exact sign stages decide), and a grid whose metric
    it already satisfies (nothing to do)."""
    out = []
    one = (np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 2]], np.int32))
    out.append(("one triangle", one[0], one[1], inputs.uniform_metric(3, 0.3)))
    xy, tri = inputs.grid_mesh(2)
    out.append(("two triangles", xy, tri, inputs.uniform_metric(4, 0.4)))
    xy, tri = inputs.grid_mesh(17)
    xs = xy.copy()
    xs[:, 1] *= 1e-7
    out.append(("sliver strip", xs, tri, inputs.uniform_metric(xs.shape[0], 0.05)))
    xy, tri = inputs.grid_mesh(9)
    out.append(("already adapted", xy, tri, inputs.uniform_metric(xy.shape[0], 0.13)))
    return out


@pytest.mark.parametrize("select", [0, 1])
def test_edge_cases_alone_and_in_a_ragged_batch(select):
    """Each edge case adapted alone and inside one batch with a regular mesh
    (sizes 1 to 3,000 triangles): mesh and counters equal the oracle's."""
    cases = _edge_case_meshes()
    w = inputs.psi_workload(17, 3000, True, 5)
    cases.append(("psi", w.xy, w.tri, w.m))
    want = []
    for name, xy, tri, m in cases:
        o = O.OracleMesh(xy, tri).set_metric(m)
        so = o.adapt(op(7, select_mode=select))
        want.append((name, o.get_mesh(), so))
        g = pm.Mesh.from_host(xy, tri, device=0)
        g.set_metric(m)
        sg = g.adapt(gp(7, select=select))
        assert_same_mesh(g.get_mesh(), o.get_mesh(), name)
        g.close()
        for k in STAT_KEYS:
            assert sg[k] == so[k], (name, k, sg[k], so[k])
    by = {name: so for name, _, so in want}
    assert by["already adapted"]["collapses"] == by["already adapted"]["splits"] == 0
    assert by["already adapted"]["converged"] == 1
    b = pm.Batch.from_host([(xy, tri) for _, xy, tri, _ in cases], device=0)
    b.set_metric(np.concatenate([m for _, _, _, m in cases]))
    stats = b.adapt([gp(7, select=select)] * len(cases))
    got = b.get_meshes()
    b.close()
    for (name, om, so), g, st in zip(want, got, stats):
        assert_same_mesh(g, om, f"{name} in the batch")
        for k in STAT_KEYS:
            assert st[k] == so[k], (name, k, st[k], so[k])


def test_batch_handle_device_arrays():
    """pm_batch_create_dev + pm_set_metric_dev + pm_batch_get_mesh_dev give the
    host path's meshes; a second adaptation of the same handle continues from
    the adapted meshes (the metric re-set in their new numbering)."""
    torch = pytest.importorskip("torch")
    ws = _small_batch()
    dev = torch.device("cuda:0")
    nv = np.array([w.xy.shape[0] for w in ws], np.int32)
    ne = np.array([w.tri.shape[0] for w in ws], np.int32)
    xy = torch.tensor(np.concatenate([w.xy for w in ws]), device=dev)
    tri = torch.tensor(np.concatenate([w.tri for w in ws]), dtype=torch.int32, device=dev)
    m = torch.tensor(np.concatenate([w.m for w in ws]), device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    b = pm.Batch.from_device(xy, nv, tri, ne, stream=stream)
    b.set_metric_dev(m)
    b.adapt([gp(w.params.seed) for w in ws])
    cap = 200_000
    oxy = torch.empty((cap, 2), dtype=torch.float64, device=dev)
    otri = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    om = torch.empty((cap, 3), dtype=torch.float64, device=dev)
    a, c = b.get_mesh_dev(oxy, otri, om)
    torch.cuda.synchronize(dev)
    ref = pm.Batch.from_host([(w.xy, w.tri) for w in ws])
    ref.set_metric(np.concatenate([w.m for w in ws]))
    ref.adapt([gp(w.params.seed) for w in ws])
    host = ref.get_meshes()
    va, vc = 0, 0
    for i, (hxy, htri, hm) in enumerate(host):
        assert (a[i], c[i]) == (hxy.shape[0], htri.shape[0])
        g = (oxy[va:va + a[i]].cpu().numpy(), otri[vc:vc + c[i]].cpu().numpy(),
             om[va:va + a[i]].cpu().numpy())
        assert_same_mesh(g, (hxy, htri, hm), ws[i].name)
        va += a[i]
        vc += c[i]
    # both continue with a coarser metric in the adapted numbering, against
    # the oracle continuing in the same way
    w0 = ws[1]
    o = O.OracleMesh(w0.xy, w0.tri).set_metric(w0.m)
    o.adapt(op(w0.params.seed))
    ref.set_metric(np.concatenate([mm * 0.5 for _, _, mm in host]))
    st = ref.adapt([gp(w.params.seed) for w in ws])
    o.set_metric(o.get_mesh()[2] * 0.5)
    so = o.adapt(op(w0.params.seed))
    assert_same_mesh(ref.get_meshes()[1], o.get_mesh(), "re-adapted mesh 1")
    for k in STAT_KEYS:
        assert st[1][k] == so[k], (k, st[1][k], so[k])
    assert so["collapses"] > 0


def _wheel(nb):
    """The unit square as a wheel: a centre vertex joined to nb vertices spaced
    evenly along the boundary (the four corners among them), so the centre's
    degree is nb."""
    per_side = nb // 4
    pts = []
    for side in range(4):
        for k in range(per_side):
            t = k / per_side
            pts.append([(t, 0.0), (1.0, t), (1.0 - t, 1.0), (0.0, 1.0 - t)][side])
    xy = np.array([[0.5, 0.5]] + pts)
    tri = np.array([[0, 1 + i, 1 + (i + 1) % nb] for i in range(nb)], np.int32)
    return xy, tri


def test_vertex_of_degree_84_adapts_bit_exact():
    """Rows longer than 64 entries: a wheel whose centre has 84 neighbours,
    adapted in full against the oracle (which has no row limit)."""
    xy, tri = _wheel(84)
    m = inputs.uniform_metric(xy.shape[0], 0.05)
    g = pm.Mesh.from_host(xy, tri, device=0)
    assert g.adjacency(0)[0].shape[0] == 84
    g.set_metric(m)
    o = O.OracleMesh(xy, tri).set_metric(m)
    sg = g.adapt(gp(17))
    so = o.adapt(op(17))
    assert_same_mesh(g.get_mesh(), o.get_mesh(), "wheel of 84")
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    assert sg["splits"] > 0 and sg["collapses"] + sg["flips"] > 0
    # beyond the supported row length (128 entries) the mesh is refused
    xy2, tri2 = _wheel(140)
    with pytest.raises(pm.PmError) as e:
        pm.Mesh.from_host(xy2, tri2, device=0)
    assert e.value.status == 4


def test_bounded_barrier_wait_times_out_and_device_stays_usable():
    """A grid barrier that no arrival completes gives up after its limit and
    reports PM_ERR_TIMEOUT (6) through the status word; the next call works."""
    status, ms = pm.selftest_wait_timeout(50.0)
    assert status == 6
    assert 50.0 <= ms < 1000.0
    with pytest.raises(pm.PmError):
        pm.selftest_wait_timeout(0.0)
    w = inputs.small_uniform()
    g, o = both(w, 1)
    g.adapt(gp(1))
    o.adapt(op(1))
    assert_same_mesh(g.get_mesh(), o.get_mesh(), "after a timed-out wait")


def test_rejects_invalid_input():
    xy, tri = inputs.grid_mesh(5)
    bad = tri.copy()
    bad[3] = bad[3][[0, 2, 1]]  # clockwise element
    with pytest.raises(pm.PmError) as e:
        pm.Mesh.from_host(xy, bad, device=0)
    assert e.value.status == 2
    # a vertex id out of range, alone and as the second mesh of a batch
    # (checked on the device before any adjacency is built)
    bad = tri.copy()
    bad[5, 1] = xy.shape[0] + 7
    with pytest.raises(pm.PmError) as e:
        pm.Mesh.from_host(xy, bad, device=0)
    assert e.value.status == 2
    with pytest.raises(pm.PmError) as e:
        pm.Batch.from_host([(xy, tri), (xy, bad)], device=0)
    assert e.value.status == 2
    # a non-finite coordinate
    nan = xy.copy()
    nan[6, 0] = np.nan
    for make in (lambda: pm.Mesh.from_host(nan, tri, device=0),
                 lambda: pm.Batch.from_host([(xy, tri), (nan, tri)], device=0)):
        with pytest.raises(pm.PmError) as e:
            make()
        assert e.value.status == 1
    g = pm.Mesh.from_host(xy, tri, device=0)
    m = inputs.uniform_metric(xy.shape[0], 0.1)
    m[4, 2] = -1.0
    with pytest.raises(pm.PmError) as e:
        g.set_metric(m)
    assert e.value.status == 1
    with pytest.raises(pm.PmError) as e:
        g.adapt(pm.Params(L_low=2.0, L_up=1.0))
    assert e.value.status == 1
    with pytest.raises(pm.PmError) as e:
        g.adapt(pm.Params(select=2))
    assert e.value.status == 1


# --- full-size workloads ------------------------------------------------------------

_ORACLE_2M = {}


def oracle_2m():
    """The oracle's adaptation of the 2M workload (stats, compacted mesh),
    computed once for the tests that need it."""
    if not _ORACLE_2M:
        w = inputs.anisotropic_2m()
        o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        _ORACLE_2M["stats"] = o.adapt(op(w.params.seed))
        _ORACLE_2M["mesh"] = o.get_mesh()
    return _ORACLE_2M["stats"], _ORACLE_2M["mesh"]


@pytest.mark.slow
def test_anisotropic_2m_full_adapt_bit_exact():
    """The single-mesh anisotropic workload at full size (2.1M output triangles)."""
    w = inputs.anisotropic_2m()
    g = pm.Mesh.from_host(w.xy, w.tri, device=0)
    g.set_metric(w.m)
    sg = g.adapt(gp(w.params.seed))
    so, omesh = oracle_2m()
    gm = g.get_mesh()
    assert_same_mesh(gm, omesh, "anisotropic 2M")
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    assert gm[1].shape[0] > 2_000_000


@pytest.mark.slow
def test_anisotropic_20m_full_adapt_bit_exact():
    """The large workload at full size (1025^2 grid, 2.1M triangles in, about
    20M out, within the 10% the size reading allows): the whole adaptation
    against the oracle's, bit for bit."""
    w = inputs.anisotropic_20m()
    seed = w.params.seed
    g = pm.Mesh.from_host(w.xy, w.tri, device=0)
    g.set_metric(w.m)
    sg = g.adapt(gp(seed))
    gmesh = g.get_mesh()
    g.close()
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    so = o.adapt(op(seed))
    assert_same_mesh(gmesh, o.get_mesh(), "anisotropic 20M")
    for k in STAT_KEYS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    assert 18_000_000 <= gmesh[1].shape[0] <= 22_000_000


@pytest.mark.slow
def test_batch_recipe_all_512_meshes_bit_exact():
    """All 512 meshes of the batch recipe adapted in one pm_batch_adapt,
    against the oracle adapting each alone (one spawned oracle process per
    host core)."""
    import os

    from tests import oracle_pool

    ws = inputs.batch_workloads()
    cores = len(os.sched_getaffinity(0))
    order = sorted(range(len(ws)), key=lambda i: -ws[i].tri.shape[0])  # largest first
    with oracle_pool.pool(cores) as p:
        pending = p.map_async(oracle_pool.batch_mesh, order, chunksize=1)
        b = pm.Batch.from_host([(w.xy, w.tri) for w in ws])
        b.set_metric(np.concatenate([w.m for w in ws]))
        stats = b.adapt([gp(w.params.seed) for w in ws])
        got = b.get_meshes()
        b.close()
        res = {r[0]: r[1:] for r in pending.get()}
    for i, w in enumerate(ws):
        oxy, otri, om, so = res[i]
        assert_same_mesh(got[i], (oxy, otri, om), w.name)
        for k in STAT_KEYS:
            assert stats[i][k] == so[k], (w.name, k, stats[i][k], so[k])


@pytest.mark.slow
def test_gradient_workload_reference_fd_and_opt_smoothing():
    """The adapted mesh of the 2M workload (~1M vertices), produced by the
    oracle itself: GPU quality gradient against the oracle's (1e-12) and
    against central differences at 1,000 vertices (1e-6); then 20 rounds of
    optimisation-based smoothing, bit-exact."""
    torch = pytest.importorskip("torch")
    from paper_1505_04694_gb300.autograd import quality

    xy0, tri0, m0 = oracle_2m()[1]
    assert xy0.shape[0] > 1_000_000
    o2 = O.OracleMesh(xy0, tri0).set_metric(m0)
    qo, do, mo = o2.quality()
    dev = torch.device("cuda:0")
    xy = torch.tensor(xy0, device=dev, requires_grad=True)
    m = torch.tensor(m0, device=dev, requires_grad=True)
    tri = torch.tensor(tri0, dtype=torch.int32, device=dev)
    q = quality(xy, m, tri)
    q.backward()
    gx, gm = xy.grad.cpu().numpy(), m.grad.cpu().numpy()
    assert abs(float(q.detach()) - qo) <= 1e-12 * abs(qo)
    assert np.linalg.norm(gx - do) <= 1e-12 * np.linalg.norm(do)
    assert np.linalg.norm(gm - mo) <= 1e-12 * np.linalg.norm(mo)
    # central differences of the ball quality sum at 1,000 seeded vertices
    rng = np.random.default_rng(4)
    vs = rng.choice(xy0.shape[0], 1000, replace=False)
    order = np.argsort(tri0.ravel() // 1, kind="stable")
    corners = tri0.ravel()[order]
    starts = np.searchsorted(corners, np.arange(xy0.shape[0] + 1))
    elems = order // 3
    def perimeter_third(t):
        k = m0[t].mean(axis=0)
        p = xy0[t]
        d = p[[1, 2, 0]] - p
        L = np.sqrt(k[0] * d[:, 0] ** 2 + 2 * k[1] * d[:, 0] * d[:, 1] + k[2] * d[:, 1] ** 2)
        return L.sum() / 3.0

    # error over all sampled vertices at once (one norm per component class:
    # coordinates and metric entries have different units); after smoothing
    # many vertices sit at a local optimum whose tiny gradient is below the
    # differences' roundoff, so a per-vertex ratio would measure noise
    acc = {"xy": [0.0, 0.0], "m": [0.0, 0.0]}
    skipped = 0
    for v in vs:
        ball = tri0[elems[starts[v]:starts[v + 1]]]
        # F(x) has a jump in its second derivative at x = 1: differences across
        # it lose an order of accuracy, so such balls are left out and counted
        if any(abs(perimeter_third(t) - 1.0) < 1e-4 for t in ball):
            skipped += 1
            continue
        nb = np.unique(ball)
        lmin = np.min(np.hypot(*(xy0[nb[nb != v]] - xy0[v]).T))

        def ball_sum(xy_v, m_v):
            s = 0.0
            for t in ball:
                pxy = xy0[t].copy()
                pm_ = m0[t].copy()
                pxy[t == v] = xy_v
                pm_[t == v] = m_v
                s += O.tri_quality(t, pxy, pm_)
            return s

        an = np.concatenate([gx[v], gm[v]])
        fd = np.zeros(5)
        for j in range(5):
            h = 1e-6 * (lmin if j < 2 else max(m0[v, 0], m0[v, 2]))
            xp, mp = xy0[v].copy(), m0[v].copy()
            xm, mm = xy0[v].copy(), m0[v].copy()
            if j < 2:
                xp[j] += h
                xm[j] -= h
            else:
                mp[j - 2] += h
                mm[j - 2] -= h
            fd[j] = (ball_sum(xp, mp) - ball_sum(xm, mm)) / (2 * h)
        for key, sl in (("xy", slice(0, 2)), ("m", slice(2, 5))):
            acc[key][0] += float(np.sum((an[sl] - fd[sl]) ** 2))
            acc[key][1] += float(np.sum(fd[sl] ** 2))
    for key, (num, den) in acc.items():
        assert (num / den) ** 0.5 <= 1e-6, (key, (num / den) ** 0.5)
    assert skipped < 100, skipped
    # 20 rounds of optimisation-based smoothing, GPU against the oracle
    g = pm.Mesh.from_host(xy0, tri0, device=0)
    g.set_metric(m0)
    sg = g.opt_smooth(gp(4, opt_smooth_rounds=20))
    so = o2.opt_smooth(op(4, opt_smooth_rounds=20))
    assert sg["moves"] == so["moves"] and sg["moves"] > 0
    assert_same_raw(g.get_raw(), o2.get_raw(), "opt smoothing")
