"""Every pin of the oracle must catch a plausible mistake.

Each case compiles the oracle with one planted change (a dropped factor, a
swapped index, a flipped comparison, a relaxed bound) into a private library
and runs the pins named for it against that library in a child process: they
must fail.  The oracle source itself is never modified.  CPU only.

Changes that cannot alter any result on a valid mesh are not listed: dropping
the duplicate-edge test of a flip (such a flip always inverts an element, so
the orientation test rejects it first) and dropping the second orientation
test of a flip (an inverted element has negative quality, so the gain test
rejects it).  Nor is leaving a flip's two opposite vertices unmarked: a flip
they would enable is found from its other end, and on the test meshes every
pass still ends with nothing left to do.  Nor is dropping one of the two
tests that keep a boundary vertex on boundary edges: the candidate list and
the collapse validity test each enforce it.  Nor is allowing a zero-area
element after a smoothing move: its quality is 0, so the move has no strict
gain.
"""
import os
import subprocess
import sys
import textwrap
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle.build import FLAGS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pm_oracle.cpp")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what, text in the oracle, planted text, pins that must fail)
MUTATIONS = [
    ("colouring: the lower priority keeps its proposal",
     "        if (m.col[u] < 0 && prop[u] == prop[v] && prio((uint32_t)u, seed, rc) > pv) keep = false;",
     "        if (m.col[u] < 0 && prop[u] == prop[v] && prio((uint32_t)u, seed, rc) < pv) keep = false;",
     "colouring_proper_complete_smallest_free"),
    ("colouring: proposals ignore coloured neighbours",
     "        if (m.col[u] >= 0 && m.col[u] < (int)used.size()) used[m.col[u]] = 1;",
     "        if (m.col[u] >= 0 && m.col[u] < 0) used[m.col[u]] = 1;",
     "colouring_proper_complete_smallest_free"),
    ("colour classes: a round takes the next class",
     "  const int cls = by_colour ? (int)(m.r % (uint32_t)m.ncol) : -1;",
     "  const int cls = by_colour ? (int)((m.r + 1u) % (uint32_t)m.ncol) : -1;",
     "colour_class_first_round"),
    ("colour classes: candidates of every class compete",
     "    if (by_colour && m.col[v] != cls) continue;",
     "    if (false && by_colour && m.col[v] != cls) continue;",
     "colour_class_first_round"),
    ("colour classes: neighbours of other classes compete",
     "if (inC[u] && (!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) > pv) {",
     "if (inC[u] && prio((uint32_t)u, seed, m.r) > pv) {",
     "colour_class_round_takes_the_whole_class"),
    ("orientation sign: the rounded formula decides every case",
     "const double ORIENT_FILTER = 8.0 * 1.1102230246251565e-16;  // 8 eps",
     "const double ORIENT_FILTER = 0.0;  // 8 eps",
     "orient_sign_exact"),
    ("orientation sign: product errors left out of the exact sum",
     "      n = grow_expansion(e, n, std::fma(a[i], b[j], -pr));",
     "      n = grow_expansion(e, n, 0.0);",
     "orient_sign_exact"),
    ("orientation sign: difference errors left out of the exact sum",
     "  two_diff(q.x, p.x, a[0], a[1]);",
     "  two_diff(q.x, p.x, a[0], a[1]);\n  a[1] = 0.0;",
     "orient_sign_exact"),
    ("metric length: off-diagonal term not doubled",
     "double L2 = ((e00 * dx) * dx + ((2.0 * e01) * dx) * dy) + (e11 * dy) * dy;",
     "double L2 = ((e00 * dx) * dx + (e01 * dx) * dy) + (e11 * dy) * dy;",
     "rotated_anisotropic"),
    ("metric length: the edge metric from one end only",
     "  double e00 = 0.5 * (a.m00 + b.m00);\n  double e01 = 0.5 * (a.m01 + b.m01);\n  double e11 = 0.5 * (a.m11 + b.m11);\n  double dx = b.x - a.x;",
     "  double e00 = a.m00;\n  double e01 = a.m01;\n  double e11 = a.m11;\n  double dx = b.x - a.x;",
     "edge_length"),
    ("quality: the shape factor without the reciprocal above the ideal perimeter",
     "  double s = (xx <= 1.0) ? xx : 1.0 / xx;",
     "  double s = xx;",
     "quality_right_isosceles"),
    ("orientation: wrong vertex in the second product",
     "return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);",
     "return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - q.x);",
     "quality_equilateral_unit"),
    ("quality: wrong shape factor",
     "double f = s * (2.0 - s);",
     "double f = s * (2.0 - s * s);",
     "quality_right_isosceles"),
    ("quality: determinant of the element metric with the wrong sign",
     "  double AM = std::sqrt(k00 * k11 - k01 * k01) * area;\n  double xx = P / 3.0;",
     "  double AM = std::sqrt(k00 * k11 + k01 * k01) * area;\n  double xx = P / 3.0;",
     "quality_affine_invariance"),
    ("quality: ideal perimeter taken as two",
     "  double AM = std::sqrt(k00 * k11 - k01 * k01) * area;\n  double xx = P / 3.0;",
     "  double AM = std::sqrt(k00 * k11 - k01 * k01) * area;\n  double xx = P / 2.0;",
     "quality_equilateral_unit"),
    ("hash priority: wrong multiplier",
     "h *= 0x85ebca6bu;",
     "h *= 0x85ebca6du;",
     "fmix32_published"),
    ("independent set: round counter starts at 1",
     "  uint32_t sr = seed + 0x9E3779B9u * r;",
     "  uint32_t sr = seed + 0x9E3779B9u * (r + 1u);",
     "round_zero"),
    ("independent set: non-candidate neighbours compete",
     "if (inC[u] && (!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) > pv) {",
     "if ((!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) > pv) {",
     "independent_set_brute_force"),
    ("independent set: the lower priority wins",
     "if (inC[u] && (!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) > pv) {",
     "if (inC[u] && (!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) < pv) {",
     "independent_set_brute_force"),
    ("collapse: candidates below twice L_low",
     "    if (L < P.L_low) cand.push_back({L, w});",
     "    if (L < 2.0 * P.L_low) cand.push_back({L, w});",
     "collapse_rule_brute_force"),
    ("refinement: edges split above half of L_up",
     "      if (!(metric_len(m.vd(a), m.vd(b)) > P.L_up)) continue;",
     "      if (!(metric_len(m.vd(a), m.vd(b)) > 0.5 * P.L_up)) continue;",
     "small_uniform_exact_result"),
    ("collapse: a degenerate element allowed",
     "    if (orient_sign(d[0], d[1], d[2]) <= 0) return false;\n  }\n  for (int x : m.NN[v]) {",
     "    if (orient_sign(d[0], d[1], d[2]) < 0) return false;\n  }\n  for (int x : m.NN[v]) {",
     "collapse_rule_brute_force"),
    ("smoothing: candidates up to twice the quality threshold",
     "  if (!(qold < P.q_thresh)) return false;\n  double a00 = 0.0",
     "  if (!(qold < 2.0 * P.q_thresh)) return false;\n  double a00 = 0.0",
     "below_the_quality_threshold"),
    ("collapse: boundary edges need two common neighbours",
     "if (common != (bedge ? 1 : 2)) return false;",
     "if (common != (bedge ? 2 : 2)) return false;",
     "collapse_rule_brute_force"),
    ("collapse: candidates tried longest first",
     "  std::sort(cand.begin(), cand.end());\n  for (const auto& c : cand)",
     "  std::sort(cand.rbegin(), cand.rend());\n  for (const auto& c : cand)",
     "collapse_rule_brute_force"),
    ("collapse: new-edge bound relaxed",
     "if (metric_len(dw, m.vd(x)) > P.L_up) return false;",
     "if (metric_len(dw, m.vd(x)) > 2.0 * P.L_up) return false;",
     "collapse_rule_brute_force"),
    ("flip: gain from the larger new quality",
     "double qnew = (n1 < n2) ? n1 : n2;",
     "double qnew = (n1 < n2) ? n2 : n1;",
     "flip_rule_brute_force"),
    ("flip: quality threshold doubled",
     "double qold = (q1 < q2) ? q1 : q2;\n  if (!(qold < P.q_thresh)) return false;",
     "double qold = (q1 < q2) ? q1 : q2;\n  if (!(qold < 2.0 * P.q_thresh)) return false;",
     "flip_rule_brute_force"),
    ("flip: a flip without gain taken",
     "  if (!(gain > 0.0)) return false;",
     "  if (!(gain >= 0.0)) return false;",
     "flip_needs_a_strict_gain"),
    ("flip: the smallest gain wins",
     "    if (!found || op.gain > best.gain) {",
     "    if (!found || op.gain < best.gain) {",
     "flip_rule_brute_force"),
    ("flip: the second new element clockwise",
     "  m.tri[op.K2] = {op.d, op.w, op.c};",
     "  m.tri[op.K2] = {op.w, op.d, op.c};",
     "operators_keep_invariants_round_by_round"),
    ("flip: the new edge missing from one end's row",
     "  recs.push_back({op.d, NN_ADD, op.c});\n",
     "",
     "operators_keep_invariants_round_by_round"),
    ("collapse: the surviving end keeps the removed vertex in its row",
     "  recs.push_back({w, NN_DEL, v});\n  m.valive[v] = 0;",
     "  m.valive[v] = 0;",
     "operators_keep_invariants_round_by_round"),
    ("refinement: the centre child of a three-split clockwise",
     "      emit(K, false, m0, m1, m2);",
     "      emit(K, false, m0, m2, m1);",
     "operators_keep_invariants_round_by_round"),
    ("refinement: a one-split child on the wrong end",
     "      emit(K, false, mm, b, o);",
     "      emit(K, false, mm, a, o);",
     "operators_keep_invariants_round_by_round"),
    ("refinement: a midpoint's x from one end",
     "      m.x.push_back(0.5 * (da.x + db.x));",
     "      m.x.push_back(0.5 * (da.x + da.x));",
     "operators_keep_invariants_round_by_round"),
    ("refinement: the longer diagonal",
     "if (d1 <= d2) {",
     "if (d1 > d2) {",
     "shorter_diagonal"),
    ("smoothing: Laplacian weight transposed",
     "b0 = b0 + (w00 * m.x[j] + w01 * m.y[j]);",
     "b0 = b0 + (w00 * m.x[j] + w11 * m.y[j]);",
     "laplacian_smoothing"),
    ("smoothing: barycentric weights swapped",
     "mv.m00 = (l0 * d[0].m00 + l1 * d[1].m00) + l2 * d[2].m00;",
     "mv.m00 = (l1 * d[0].m00 + l0 * d[1].m00) + l2 * d[2].m00;",
     "linear_metric"),
    ("smoothing: sign error in the 2x2 solve",
     "  double X = (a11 * b0 - a01 * b1) / det;",
     "  double X = (a11 * b0 + a01 * b1) / det;",
     "moves_with_the_patch"),
    ("smoothing: second right-hand side with swapped weights",
     "    b1 = b1 + (w01 * m.x[j] + w11 * m.y[j]);",
     "    b1 = b1 + (w11 * m.x[j] + w01 * m.y[j]);",
     "moves_with_the_patch"),
    ("smoothing: a move that gains nothing is taken",
     "  return qmin > qold;\n}",
     "  return qmin >= qold;\n}",
     "strict_gain"),
    ("refinement: the midpoint of a boundary edge is not a boundary vertex",
     "      m.vbnd.push_back(edge_elements(m, a, b) == 1 ? 1 : 0);",
     "      m.vbnd.push_back(0);",
     "round_equals_sequential_and_invariants"),
    ("refinement: a midpoint takes one end's metric",
     "      m.m00.push_back(0.5 * (da.m00 + db.m00));",
     "      m.m00.push_back(0.5 * (da.m00 + da.m00));",
     "linear_metric_field"),
    ("smoothing: neighbours of a moved vertex not pending for the next sweep",
     "          if (m.valive[j] && !m.vbnd[j]) next[j] = 1;",
     "          if (false && m.valive[j] && !m.vbnd[j]) next[j] = 1;",
     "only_moved_vertices"),
    ("smoothing: one sweep only",
     "    if (moved_sweep == 0) break;",
     "    break;",
     "only_moved_vertices"),
    ("collapse: neighbours not marked for re-evaluation",
     "      for (int x : m.NN[v]) dirty[x] = 1;",
     "      for (int x : m.NN[v]) dirty[x] = dirty[x];",
     "nothing_left"),
    ("refinement: stops after three rounds",
     "    int64_t n = refine_round(m, P, st);\n    if (n == 0) break;",
     "    int64_t n = refine_round(m, P, st);\n    if (n == 0 || rounds == 3) break;",
     "no_edge_too_long"),
    ("Algorithm 1: refinement first",
     "    int64_t n = op_coarsen(*m, *P, local);\n    n += op_swap(*m, *P, local);\n    n += op_refine(*m, *P, local);",
     "    int64_t n = op_refine(*m, *P, local);\n    n += op_coarsen(*m, *P, local);\n    n += op_swap(*m, *P, local);",
     "algorithm_1"),
    ("Algorithm 1: no renumbering between iterations",
     "    renumber(*m);\n    if (n == 0) {\n      local.converged = 1;",
     "    if (n == 0) {\n      local.converged = 1;",
     "algorithm_1"),
    ("independent set: seeds of later rounds by exclusive or",
     "  uint32_t sr = seed + 0x9E3779B9u * r;",
     "  uint32_t sr = seed ^ (0x9E3779B9u * r);",
     "algorithm_1"),
    ("smoothing: the plain centroid as the target",
     "    double w00 = 0.5 * (m.m00[v] + m.m00[j]);\n    double w01 = 0.5 * (m.m01[v] + m.m01[j]);\n    double w11 = 0.5 * (m.m11[v] + m.m11[j]);",
     "    double w00 = 1.0;\n    double w01 = 0.0;\n    double w11 = 1.0;",
     "smoothing"),
    ("Algorithm 1: stops after one iteration",
     "    if (n == 0) {\n      local.converged = 1;",
     "    if (n >= 0) {\n      local.converged = 1;",
     "round_equals_sequential"),
    ("quality gradient: sign lost past the ideal perimeter",
     "  double gxx = left ? gs : -(gs / (xx * xx));",
     "  double gxx = left ? gs : (gs / (xx * xx));",
     "gradient_central_differences"),
    ("quality gradient: off-diagonal determinant partial halved",
     "  double gk01 = -(2.0 * k01) * gdet;",
     "  double gk01 = -(k01) * gdet;",
     "gradient_central_differences"),
    ("quality gradient: canonical slots not mapped back",
     "    for (int j = 0; j < 5; ++j) g[(s + k) % 3][j] = cg[k][j];",
     "    for (int j = 0; j < 5; ++j) g[k][j] = cg[k][j];",
     "gradient_central_differences"),
    ("optimisation smoothing: first step doubled",
     "  double alpha = (0.1 * lmin) / gn;",
     "  double alpha = (0.2 * lmin) / gn;",
     "step_rule"),
    ("optimisation smoothing: a step kept without a rising quality sum",
     "      if (ball_after_move(m, v, cand, qmin, qsum) && qmin >= qmin_old && qsum > qsum_old) {",
     "      if (ball_after_move(m, v, cand, qmin, qsum) && qmin >= qmin_old) {",
     "step_rule"),
    ("optimisation smoothing: a step kept that lowers the minimum quality",
     "      if (ball_after_move(m, v, cand, qmin, qsum) && qmin >= qmin_old && qsum > qsum_old) {",
     "      if (ball_after_move(m, v, cand, qmin, qsum) && qsum > qsum_old) {",
     "step_rule"),
    ("optimisation smoothing: seven step sizes tried",
     "  for (int k = 0; k < 6; ++k) {\n    double X = m.x[v] + alpha * gx;",
     "  for (int k = 0; k < 7; ++k) {\n    double X = m.x[v] + alpha * gx;",
     "step_rule"),
    ("optimisation smoothing: step along a swapped gradient component",
     "    double X = m.x[v] + alpha * gx;",
     "    double X = m.x[v] + alpha * gy;",
     "step_rule"),
    ("boundary: corner test inverted",
     "m->vcorner[v] = orient_sign(m->vd(lo), m->vd(v), m->vd(hi)) != 0 ? 1 : 0;",
     "m->vcorner[v] = orient_sign(m->vd(lo), m->vd(v), m->vd(hi)) == 0 ? 1 : 0;",
     "collapse_rule_brute_force"),
]

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    from oracle import build
    build.build = lambda force=False: {lib!r}
    import pytest
    sys.exit(pytest.main(["-q", "-p", "no:cacheprovider", {pins!r}, "-k", {sel!r}]))
""")


def read_source():
    with open(SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    """The unchanged oracle and every mutant whose site occurs once, compiled
    with the oracle's own flags, all at once (one g++ per core); maps a
    mutation's name (None: unchanged) to its library."""
    src = read_source()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {None: src}
    for what, old, new, _ in MUTATIONS:
        if src.count(old) == 1:
            jobs[what] = src.replace(old, new)
    out = {}
    for i, (what, text) in enumerate(jobs.items()):
        (d / f"m{i}.cpp").write_text(text)
        out[what] = d / f"m{i}.so"

    def compile_one(i):
        subprocess.check_call(["g++", *FLAGS, str(d / f"m{i}.cpp"), "-o", str(d / f"m{i}.so")])

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(compile_one, range(len(jobs))))
    return out


def run_pins(lib, sel):
    """Run the pins `sel` against the oracle library `lib` in a child
    process; returns pytest's exit status and output."""
    code = CHILD.format(root=ROOT, lib=str(lib), pins=PINS, sel=sel)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout


def test_selected_pins_pass_on_the_unchanged_oracle(libs):
    sel = " or ".join(sorted({m[3] for m in MUTATIONS}))
    status, out = run_pins(libs[None], sel)
    assert status == 0, out[-3000:]


@pytest.mark.parametrize("what,old,new,sel", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(libs, what, old, new, sel):
    assert read_source().count(old) == 1, f"{what}: the planted site must occur once"
    status, out = run_pins(libs[what], sel)
    # pytest's exit status 1: tests ran and some failed (5 would mean none ran)
    assert status == 1, f"{what}: pins {sel!r} did not fail\n{out[-3000:]}"
