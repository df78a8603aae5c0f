// Sequential CPU oracle for round-based independent-set 2D anisotropic mesh
// adaptation (Rokos, Gorman, Jensen, Kelly: "Thread Parallelism for Highly
// Irregular Computation in Anisotropic Mesh Adaptation").
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA library is checked against.  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it.  It shares no code, header or
// constant table with the CUDA path; both sides are written from the same
// readings of the paper (listed in the design notes) and use IEEE-754 binary64
// with no contraction (built with -ffp-contract=off), evaluated in the order
// written here.
//
// What it follows:
//  * Algorithm 1 (Sec. 2.3): repeat {coarsen; swap; refine} until no change or
//    the iteration limit, then smooth.
//  * Sec. 2.4: the four kernels (collapse, split + templates, flip, smoothing)
//    and propagation (operators sweep until nothing changes).
//  * Sec. 3.2: every operator runs in rounds; each round processes one
//    independent set of the vertex graph.  By default the set is the local
//    maxima of a hash priority among the round's candidates; with
//    select_mode 1 the vertex graph is coloured at the start of each
//    collapse, flip and smoothing pass and round r takes the candidates of
//    colour r mod (number of colours), the paper's own scheme.
//  * Sec. 2.4 validity tests (an element counter-clockwise, a point in the
//    closed element, a corner): the sign of the exact orientation
//    determinant (a floating-point filter, else an exact expansion).
//  * Sec. 3.3: deferred update.  While a round applies its operations, every
//    adjacency change is queued as a record addressed to the vertex whose list
//    changes; the queue is committed only after the whole set was processed.
//  * Sec. 3.4: worklists.  The sequential oracle simply walks vertex ids in
//    ascending order; the set semantics do not depend on the order.
//
// Parity status of each function is stated at its definition; those marked
// "convention" are readings of passages the paper leaves open (the choice of
// collapse target, flip edge, refinement diagonal, smoothing target,
// optimisation step); each is pinned through quantities the tests compute
// independently (brute force, closed forms, the gradient), besides
// round-equals-sequential and the invariants.

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

// Status codes mirror the public library's meaning (kept as plain ints here).
enum { OK = 0, ERR_INVALID_ARG = 1, ERR_INVALID_MESH = 2, ERR_INVARIANT = 7 };

struct Params {
  double L_low, L_up, q_thresh;
  int32_t max_iter, max_smooth_sweeps;
  uint32_t seed;
  int32_t opt_smooth_rounds;
  int32_t max_rounds;   // cap on rounds per operator call; 0 = none
  int32_t select_mode;  // 0: hash-priority sets; 1: colour classes (Sec. 3.2)
};

struct Stats {
  int64_t rounds, collapses, splits, flips, moves;
  int32_t converged;
  double ms;
};

// One vertex's data as the arithmetic sees it.
struct VD {
  double x, y, m00, m01, m11;
};

struct OMesh {
  std::vector<double> x, y, m00, m01, m11;
  std::vector<uint8_t> valive, vbnd, vcorner;
  std::vector<std::array<int, 3>> tri;
  std::vector<uint8_t> talive;
  std::vector<std::vector<int>> NN, NE;  // sorted sets
  uint32_t r = 0;                        // round counter of the current call
  std::vector<int> col;                  // colour of each vertex (colour-class sets)
  int ncol = 1;                          // colours in use
  bool check_seq = false;                // round-equals-sequential self check
  int seq_fail = 0;
  int64_t euler0 = 1;                    // V - E + F at creation (1 for a disk)

  int nv() const { return (int)x.size(); }
  int ne() const { return (int)tri.size(); }
  VD vd(int v) const { return VD{x[v], y[v], m00[v], m01[v], m11[v]}; }
};

int check_invariants(const OMesh& m);

// ---------------------------------------------------------------------------
// Arithmetic (Sec. 2.2: quality functional of Vasilevskii et al.; unit edge
// length in metric space).
// ---------------------------------------------------------------------------

// Metric length of edge (a,b): the edge metric is the component-wise mean of
// the end-point metrics, L^2 = d^T E d.  Bitwise symmetric in (a,b).
double metric_len(const VD& a, const VD& b) {
  double e00 = 0.5 * (a.m00 + b.m00);
  double e01 = 0.5 * (a.m01 + b.m01);
  double e11 = 0.5 * (a.m11 + b.m11);
  double dx = b.x - a.x;
  double dy = b.y - a.y;
  double L2 = ((e00 * dx) * dx + ((2.0 * e01) * dx) * dy) + (e11 * dy) * dy;
  return std::sqrt(L2);
}

// Twice the signed area of (p,q,r); > 0 for counter-clockwise.
double orient3(const VD& p, const VD& q, const VD& r) {
  return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);
}

// Canonical rotation of a triangle: the smallest vertex id goes first, the
// cyclic order is kept.  Orientation values (areas, barycentric weights) and
// qualities are taken in this rotation so that they do not depend on how a
// triangle happens to be stored; orientation signs are exact (below) and so
// independent of the rotation anyway.
void canon(int ids[3], VD d[3]) {
  int s = 0;
  if (ids[1] < ids[s]) s = 1;
  if (ids[2] < ids[s]) s = 2;
  if (s == 0) return;
  int i2[3] = {ids[s], ids[(s + 1) % 3], ids[(s + 2) % 3]};
  VD d2[3] = {d[s], d[(s + 1) % 3], d[(s + 2) % 3]};
  for (int k = 0; k < 3; ++k) {
    ids[k] = i2[k];
    d[k] = d2[k];
  }
}

// ---------------------------------------------------------------------------
// Exact orientation sign (reading S3 with robust predicates).  Every validity
// decision (an element counter-clockwise, a point in the closed element, a
// corner) takes the sign of
//   det = (q.x - p.x)(r.y - p.y) - (q.y - p.y)(r.x - p.x)
// of the real numbers the doubles stand for, so it does not depend on the
// rounding of the formula or on the rotation it is evaluated in.
//   - Filter: when |det| computed in floating point exceeds 8 eps (|t1| +
//     |t2|), eps = 2^-53, its sign is the exact one (a bound on the rounding
//     error of this form is (3 + 16 eps) eps (|t1| + |t2|): J. R. Shewchuk,
//     "Adaptive precision floating-point arithmetic and fast robust
//     geometric predicates", 1997).
//   - Otherwise det is summed exactly: each difference is a two-term
//     expansion (its rounded value and rounding error), each of the eight
//     partial products is exact as a product and its error (fma), and the
//     sixteen terms are grown into a non-overlapping expansion by exact
//     two-sums; the sign of such an expansion is that of its largest term.
// Exact as long as no product or error underflows or overflows (coordinates
// zero or of magnitude between 1e-140 and 1e140).  Parity: pinned against
// rational arithmetic.
void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

void two_diff(double a, double b, double& s, double& e) {
  s = a - b;
  double bv = a - s;
  e = (a - (s + bv)) + (bv - b);
}

// Adds b to the non-overlapping expansion e[0..n) (increasing magnitude),
// dropping zero terms; returns the new length.
int grow_expansion(double* e, int n, double b) {
  double q = b;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    double sum, err;
    two_sum(q, e[i], sum, err);
    if (err != 0.0) e[m++] = err;
    q = sum;
  }
  if (q != 0.0) e[m++] = q;
  return m;
}

int orient_exact(const VD& p, const VD& q, const VD& r) {
  double a[2], b[2], c[2], d[2];  // {rounded difference, its error}
  two_diff(q.x, p.x, a[0], a[1]);
  two_diff(r.y, p.y, b[0], b[1]);
  two_diff(q.y, p.y, c[0], c[1]);
  two_diff(r.x, p.x, d[0], d[1]);
  double e[32];
  int n = 0;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double pr = a[i] * b[j];
      n = grow_expansion(e, n, pr);
      n = grow_expansion(e, n, std::fma(a[i], b[j], -pr));
      double ps = c[i] * d[j];
      n = grow_expansion(e, n, -ps);
      n = grow_expansion(e, n, -std::fma(c[i], d[j], -ps));
    }
  if (n == 0) return 0;
  return e[n - 1] > 0.0 ? 1 : -1;
}

const double ORIENT_FILTER = 8.0 * 1.1102230246251565e-16;  // 8 eps

int orient_sign(const VD& p, const VD& q, const VD& r) {
  double t1 = (q.x - p.x) * (r.y - p.y);
  double t2 = (q.y - p.y) * (r.x - p.x);
  double det = t1 - t2;
  double bound = ORIENT_FILTER * (std::fabs(t1) + std::fabs(t2));
  if (det > bound) return 1;
  if (-det > bound) return -1;
  return orient_exact(p, q, r);
}

const double QC = 12.0 * 1.7320508075688772;  // 12 sqrt(3)

// Length of (q - p) under the fixed metric k.
double len_under(double k00, double k01, double k11, const VD& p, const VD& q) {
  double dx = q.x - p.x;
  double dy = q.y - p.y;
  double L2 = ((k00 * dx) * dx + ((2.0 * k01) * dx) * dy) + (k11 * dy) * dy;
  return std::sqrt(L2);
}

// Vasilevskii-Lipnikov quality of a triangle in the element-mean metric:
//   q = 12 sqrt(3) |K|_M / P_M^2 * F(P_M / 3),  F(x) = (min(x,1/x)(2 - min(x,1/x)))^3
// which is 1 for an equilateral triangle with unit metric edges.  Parity:
// pinned by closed forms (equilateral, right isosceles, affine invariance).
double quality_c(int i0, int i1, int i2, VD a, VD b, VD c) {
  int ids[3] = {i0, i1, i2};
  VD d[3] = {a, b, c};
  canon(ids, d);
  double k00 = ((d[0].m00 + d[1].m00) + d[2].m00) / 3.0;
  double k01 = ((d[0].m01 + d[1].m01) + d[2].m01) / 3.0;
  double k11 = ((d[0].m11 + d[1].m11) + d[2].m11) / 3.0;
  double l0 = len_under(k00, k01, k11, d[0], d[1]);
  double l1 = len_under(k00, k01, k11, d[1], d[2]);
  double l2 = len_under(k00, k01, k11, d[2], d[0]);
  double P = (l0 + l1) + l2;
  double area = 0.5 * orient3(d[0], d[1], d[2]);
  double AM = std::sqrt(k00 * k11 - k01 * k01) * area;
  double xx = P / 3.0;
  double s = (xx <= 1.0) ? xx : 1.0 / xx;
  double f = s * (2.0 - s);
  double F = (f * f) * f;
  return ((QC * AM) / (P * P)) * F;
}

// Reverse-mode derivative of quality_c.  Writes dq/d(x,y,m00,m01,m11) of the
// three vertices in the caller's (stored) order.  Parity: pinned against
// central finite differences of quality_c and against automatic
// differentiation of the same formula.
double quality_grad_c(int i0, int i1, int i2, VD a, VD b, VD c, double g[3][5]) {
  int ids[3] = {i0, i1, i2};
  VD d[3] = {a, b, c};
  int s = 0;
  if (ids[1] < ids[s]) s = 1;
  if (ids[2] < ids[s]) s = 2;
  canon(ids, d);
  const VD &p0 = d[0], &p1 = d[1], &p2 = d[2];
  double k00 = ((p0.m00 + p1.m00) + p2.m00) / 3.0;
  double k01 = ((p0.m01 + p1.m01) + p2.m01) / 3.0;
  double k11 = ((p0.m11 + p1.m11) + p2.m11) / 3.0;
  double dx[3] = {p1.x - p0.x, p2.x - p1.x, p0.x - p2.x};
  double dy[3] = {p1.y - p0.y, p2.y - p1.y, p0.y - p2.y};
  double l[3];
  for (int e = 0; e < 3; ++e) {
    double L2 = ((k00 * dx[e]) * dx[e] + ((2.0 * k01) * dx[e]) * dy[e]) + (k11 * dy[e]) * dy[e];
    l[e] = std::sqrt(L2);
  }
  double P = (l[0] + l[1]) + l[2];
  double area = 0.5 * orient3(p0, p1, p2);
  double sd = std::sqrt(k00 * k11 - k01 * k01);
  double AM = sd * area;
  double xx = P / 3.0;
  bool left = (xx <= 1.0);
  double sv = left ? xx : 1.0 / xx;
  double f = sv * (2.0 - sv);
  double F = (f * f) * f;
  double t = (QC * AM) / (P * P);
  double q = t * F;

  // backward, seed dq = 1
  double gF = t;
  double gt = F;
  double gAM = (gt * QC) / (P * P);
  double gP = -((2.0 * t) / P) * gt;
  double gf = (3.0 * (f * f)) * gF;
  double gs = (2.0 - 2.0 * sv) * gf;
  double gxx = left ? gs : -(gs / (xx * xx));
  gP = gP + gxx / 3.0;
  double gsd = area * gAM;
  double garea = sd * gAM;
  double gdet = gsd / (2.0 * sd);
  double gk00 = k11 * gdet;
  double gk11 = k00 * gdet;
  double gk01 = -(2.0 * k01) * gdet;
  double go = 0.5 * garea;
  double gdx[3], gdy[3];
  for (int e = 0; e < 3; ++e) {
    double gL2 = gP / (2.0 * l[e]);
    gk00 = gk00 + (dx[e] * dx[e]) * gL2;
    gk01 = gk01 + (2.0 * (dx[e] * dy[e])) * gL2;
    gk11 = gk11 + (dy[e] * dy[e]) * gL2;
    gdx[e] = ((2.0 * k00) * dx[e] + (2.0 * k01) * dy[e]) * gL2;
    gdy[e] = ((2.0 * k01) * dx[e] + (2.0 * k11) * dy[e]) * gL2;
  }
  double cg[3][5];
  cg[0][0] = (go * (p1.y - p2.y) - gdx[0]) + gdx[2];
  cg[1][0] = (go * (p2.y - p0.y) + gdx[0]) - gdx[1];
  cg[2][0] = (go * (p0.y - p1.y) + gdx[1]) - gdx[2];
  cg[0][1] = (go * (p2.x - p1.x) - gdy[0]) + gdy[2];
  cg[1][1] = (go * (p0.x - p2.x) + gdy[0]) - gdy[1];
  cg[2][1] = (go * (p1.x - p0.x) + gdy[1]) - gdy[2];
  for (int k = 0; k < 3; ++k) {
    cg[k][2] = gk00 / 3.0;
    cg[k][3] = gk01 / 3.0;
    cg[k][4] = gk11 / 3.0;
  }
  // canonical slot k holds stored vertex (s + k) % 3
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 5; ++j) g[(s + k) % 3][j] = cg[k][j];
  return q;
}

// ---------------------------------------------------------------------------
// Independent sets (Sec. 3.2).  Priority = MurmurHash3 fmix32 finaliser of the
// vertex id xor a per-round seed; a vertex joins the set when its priority is
// larger than that of every candidate neighbour (fmix32 is a bijection, so
// ties cannot occur).  Parity: fmix32 pinned by the published MurmurHash3
// test vectors; the set pinned by brute force (independence, local maxima).
// ---------------------------------------------------------------------------

uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

uint32_t prio(uint32_t v, uint32_t seed, uint32_t r) {
  uint32_t sr = seed + 0x9E3779B9u * r;
  return fmix32(v ^ sr);
}

// S = { v in C : prio(v) > prio(u) for every u in NN(v) that is also in C }.
// With colour classes (by_colour): only the candidates of class m.r mod
// ncol compete, and among them the same rule (a collapse or flip may have
// joined two vertices of one class since the colouring).
std::vector<int> independent_set(const OMesh& m, const std::vector<uint8_t>& inC,
                                 const std::vector<int>& C, uint32_t seed,
                                 bool by_colour = false) {
  std::vector<int> S;
  const int cls = by_colour ? (int)(m.r % (uint32_t)m.ncol) : -1;
  for (int v : C) {
    if (by_colour && m.col[v] != cls) continue;
    uint32_t pv = prio((uint32_t)v, seed, m.r);
    bool best = true;
    for (int u : m.NN[v]) {
      if (inC[u] && (!by_colour || m.col[u] == cls) && prio((uint32_t)u, seed, m.r) > pv) {
        best = false;
        break;
      }
    }
    if (best) S.push_back(v);
  }
  return S;
}

// ---------------------------------------------------------------------------
// Colouring of the vertex graph (Sec. 3.2: independent sets as colour
// classes, re-coloured after the topology changes; here once per operator
// pass).  Speculative rounds on a snapshot: every uncoloured live vertex
// proposes the smallest colour that no coloured neighbour holds; of two
// uncoloured neighbours proposing the same colour the one of lower priority
// (prio with the pass's first round counter) withdraws; every other
// proposal is kept.  The vertex of highest priority among the uncoloured
// always keeps its proposal, so the rounds end.  Parity: pinned by the
// colouring's properness, completeness and the smallest-free-colour rule
// checked by brute force.
// ---------------------------------------------------------------------------

void colour_vertices(OMesh& m, uint32_t seed) {
  const int nv = m.nv();
  const uint32_t rc = m.r;
  m.col.assign(nv, -1);
  std::vector<int> prop(nv, -1);
  for (;;) {
    bool open = false;
    for (int v = 0; v < nv; ++v) {
      if (!m.valive[v] || m.col[v] >= 0) continue;
      open = true;
      std::vector<uint8_t> used(m.NN[v].size() + 1, 0);
      for (int u : m.NN[v])
        if (m.col[u] >= 0 && m.col[u] < (int)used.size()) used[m.col[u]] = 1;
      int c = 0;
      while (used[c]) ++c;
      prop[v] = c;
    }
    if (!open) break;
    std::vector<int> next = m.col;
    for (int v = 0; v < nv; ++v) {
      if (!m.valive[v] || m.col[v] >= 0) continue;
      bool keep = true;
      const uint32_t pv = prio((uint32_t)v, seed, rc);
      for (int u : m.NN[v])
        if (m.col[u] < 0 && prop[u] == prop[v] && prio((uint32_t)u, seed, rc) > pv) keep = false;
      if (keep) next[v] = prop[v];
    }
    m.col.swap(next);
  }
  m.ncol = 1;
  for (int v = 0; v < nv; ++v)
    if (m.valive[v] && m.col[v] + 1 > m.ncol) m.ncol = m.col[v] + 1;
}

// ---------------------------------------------------------------------------
// Adjacency (Sec. 3.1 "adjacency list of a vertex"): NN = vertex neighbours,
// NE = incident elements, both kept as sorted sets and fully determined by the
// live element list.  rebuild_adjacency is the definition; the per-round
// deferred update (commit) must reproduce it, which check_invariants verifies.
// ---------------------------------------------------------------------------

void sorted_insert(std::vector<int>& row, int val) {
  auto it = std::lower_bound(row.begin(), row.end(), val);
  if (it == row.end() || *it != val) row.insert(it, val);
}

void sorted_erase(std::vector<int>& row, int val) {
  auto it = std::lower_bound(row.begin(), row.end(), val);
  if (it != row.end() && *it == val) row.erase(it);
}

bool sorted_has(const std::vector<int>& row, int val) {
  return std::binary_search(row.begin(), row.end(), val);
}

void rebuild_adjacency(OMesh& m) {
  int nv = m.nv();
  m.NN.assign(nv, {});
  m.NE.assign(nv, {});
  for (int K = 0; K < m.ne(); ++K) {
    if (!m.talive[K]) continue;
    for (int i = 0; i < 3; ++i) {
      int v = m.tri[K][i];
      m.NE[v].push_back(K);
      m.NN[v].push_back(m.tri[K][(i + 1) % 3]);
      m.NN[v].push_back(m.tri[K][(i + 2) % 3]);
    }
  }
  for (int v = 0; v < nv; ++v) {
    std::sort(m.NE[v].begin(), m.NE[v].end());
    std::sort(m.NN[v].begin(), m.NN[v].end());
    m.NN[v].erase(std::unique(m.NN[v].begin(), m.NN[v].end()), m.NN[v].end());
  }
}

// An edge is on the boundary when exactly one live element contains it.
int edge_elements(const OMesh& m, int v, int w) {
  int n = 0;
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    if (t[0] == w || t[1] == w || t[2] == w) ++n;
  }
  return n;
}

bool tri_has(const std::array<int, 3>& t, int v) { return t[0] == v || t[1] == v || t[2] == v; }

// Deferred-update record: "row `kind` of vertex `target` gains/loses `val`".
enum RecKind { NN_ADD, NN_DEL, NE_ADD, NE_DEL };
struct Rec {
  int target;
  int kind;
  int val;
};

// Commit phase of the deferred update (Sec. 3.3): every record is applied to
// the one list it names, after the whole independent set was processed.
// Rows are sets, so the order of records does not matter.
void commit(OMesh& m, const std::vector<Rec>& recs) {
  for (const Rec& rc : recs) {
    switch (rc.kind) {
      case NN_ADD: sorted_insert(m.NN[rc.target], rc.val); break;
      case NN_DEL: sorted_erase(m.NN[rc.target], rc.val); break;
      case NE_ADD: sorted_insert(m.NE[rc.target], rc.val); break;
      case NE_DEL: sorted_erase(m.NE[rc.target], rc.val); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Coarsening (Sec. 2.4.1): collapse a short edge v->w, removing the elements
// that contain it.  Convention (paper defers to Li et al.): candidate targets
// are neighbours with metric length < L_low, tried by (length, id); the first
// that keeps the mesh valid wins:
//   (i) link condition: |NN(v) & NN(w)| is 2 (interior edge) or 1 (boundary);
//  (ii) every element of v's ball not containing w stays counter-clockwise
//       with v moved onto w;
// (iii) no new edge (w,x) is longer than L_up.
// Corners never collapse; a boundary vertex collapses only along a boundary
// edge.  Parity: convention, pinned by brute-force enumeration.
// ---------------------------------------------------------------------------

bool collapse_valid(const OMesh& m, int v, int w, const Params& P) {
  bool bedge = edge_elements(m, v, w) == 1;
  if (m.vbnd[v] && !bedge) return false;
  int common = 0;
  for (int x : m.NN[v])
    if (sorted_has(m.NN[w], x)) ++common;
  if (common != (bedge ? 1 : 2)) return false;
  VD dw = m.vd(w);
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    if (tri_has(t, w)) continue;
    int id[3];
    VD d[3];
    for (int i = 0; i < 3; ++i) {
      id[i] = (t[i] == v) ? w : t[i];
      d[i] = (t[i] == v) ? dw : m.vd(t[i]);
    }
    if (orient_sign(d[0], d[1], d[2]) <= 0) return false;
  }
  for (int x : m.NN[v]) {
    if (x == w || sorted_has(m.NN[w], x)) continue;
    if (metric_len(dw, m.vd(x)) > P.L_up) return false;
  }
  return true;
}

int coarsen_target(const OMesh& m, int v, const Params& P) {
  if (!m.valive[v] || m.vcorner[v]) return -1;
  std::vector<std::pair<double, int>> cand;
  for (int w : m.NN[v]) {
    if (m.vbnd[v] && edge_elements(m, v, w) != 1) continue;
    double L = metric_len(m.vd(v), m.vd(w));
    if (L < P.L_low) cand.push_back({L, w});
  }
  std::sort(cand.begin(), cand.end());
  for (const auto& c : cand)
    if (collapse_valid(m, v, c.second, P)) return c.second;
  return -1;
}

void apply_collapse(OMesh& m, int v, int w, std::vector<Rec>& recs) {
  for (int K : m.NE[v]) {
    auto& t = m.tri[K];
    if (tri_has(t, w)) {
      m.talive[K] = 0;
      for (int i = 0; i < 3; ++i)
        if (t[i] != v) recs.push_back({t[i], NE_DEL, K});
    } else {
      for (int i = 0; i < 3; ++i)
        if (t[i] == v) t[i] = w;
      recs.push_back({w, NE_ADD, K});
    }
  }
  for (int x : m.NN[v]) {
    if (x == w) continue;
    recs.push_back({x, NN_DEL, v});
    recs.push_back({x, NN_ADD, w});
    recs.push_back({w, NN_ADD, x});
  }
  recs.push_back({w, NN_DEL, v});
  m.valive[v] = 0;
}

// ---------------------------------------------------------------------------
// Swapping (Sec. 2.4.3): flip an interior edge when the minimum quality of the
// two elements improves.  Convention: a set member v looks at its interior
// edges (v,w) whose two elements have min quality below q_thresh, skips flips
// that would duplicate an edge or fold an element, and takes the largest
// strictly positive gain (ties: smallest w).  K1=(v,w,c) becomes (v,d,c) and
// K2=(w,v,d) becomes (d,w,c).  Parity: convention, pinned by brute force and
// the monotone-min-quality property.
// ---------------------------------------------------------------------------

struct SwapOp {
  int w, c, d, K1, K2;
  double gain;
};

double quality_of(const OMesh& m, int K) {
  const auto& t = m.tri[K];
  return quality_c(t[0], t[1], t[2], m.vd(t[0]), m.vd(t[1]), m.vd(t[2]));
}

bool flip_candidate(const OMesh& m, int v, int w, const Params& P, SwapOp& op) {
  int K1 = -1, K2 = -1, c = -1, d = -1;
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    int i = (t[0] == v) ? 0 : (t[1] == v) ? 1 : 2;
    if (t[(i + 1) % 3] == w) {
      K1 = K;
      c = t[(i + 2) % 3];
    }
    if (t[(i + 2) % 3] == w) {
      K2 = K;
      d = t[(i + 1) % 3];
    }
  }
  if (K1 < 0 || K2 < 0) return false;
  if (sorted_has(m.NN[d], c)) return false;
  double q1 = quality_of(m, K1), q2 = quality_of(m, K2);
  double qold = (q1 < q2) ? q1 : q2;
  if (!(qold < P.q_thresh)) return false;
  VD dv = m.vd(v), dw = m.vd(w), dc = m.vd(c), dd = m.vd(d);
  if (orient_sign(dv, dd, dc) <= 0) return false;
  if (orient_sign(dd, dw, dc) <= 0) return false;
  double n1 = quality_c(v, d, c, dv, dd, dc);
  double n2 = quality_c(d, w, c, dd, dw, dc);
  double qnew = (n1 < n2) ? n1 : n2;
  double gain = qnew - qold;
  if (!(gain > 0.0)) return false;
  op = SwapOp{w, c, d, K1, K2, gain};
  return true;
}

bool swap_eval(const OMesh& m, int v, const Params& P, SwapOp& best) {
  if (!m.valive[v]) return false;
  bool found = false;
  for (int w : m.NN[v]) {
    SwapOp op;
    if (!flip_candidate(m, v, w, P, op)) continue;
    if (!found || op.gain > best.gain) {
      best = op;
      found = true;
    }
  }
  return found;
}

void apply_flip(OMesh& m, int v, const SwapOp& op, std::vector<Rec>& recs) {
  m.tri[op.K1] = {v, op.d, op.c};
  m.tri[op.K2] = {op.d, op.w, op.c};
  recs.push_back({v, NN_DEL, op.w});
  recs.push_back({op.w, NN_DEL, v});
  recs.push_back({op.c, NN_ADD, op.d});
  recs.push_back({op.d, NN_ADD, op.c});
  recs.push_back({v, NE_DEL, op.K2});
  recs.push_back({op.w, NE_DEL, op.K1});
  recs.push_back({op.c, NE_ADD, op.K2});
  recs.push_back({op.d, NE_ADD, op.K1});
}

// ---------------------------------------------------------------------------
// Smoothing (Sec. 2.4.4): quality-constrained Laplacian.  Convention: the
// target is the metric-weighted mean of the neighbours, x* = A^-1 b with
// A = sum W_j, b = sum W_j x_j, W_j the edge metric; the new metric is the
// barycentric interpolation at x* in the ball element that contains it; the
// move is kept only when every ball element stays counter-clockwise and the
// minimum ball quality strictly increases.  Parity: convention, pinned by the
// closed-form regular-patch cases, exact reproduction of a linear metric
// field, the strict-gain case and the monotone property.
// ---------------------------------------------------------------------------

struct Move {
  double x, y, m00, m01, m11;
};

double ball_min_quality(const OMesh& m, int v, double* qsum = nullptr) {
  double qmin = 0.0, sum = 0.0;
  bool first = true;
  for (int K : m.NE[v]) {
    double q = quality_of(m, K);
    if (first || q < qmin) qmin = q;
    first = false;
    sum = sum + q;
  }
  if (qsum) *qsum = sum;
  return qmin;
}

// Locate point X in v's ball (v at its current position) and interpolate the
// metric there.  Returns false when no ball element contains X.
bool interpolate_in_ball(const OMesh& m, int v, double X, double Y, Move& mv) {
  VD px{X, Y, 0.0, 0.0, 0.0};
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    int ids[3] = {t[0], t[1], t[2]};
    VD d[3] = {m.vd(t[0]), m.vd(t[1]), m.vd(t[2])};
    canon(ids, d);
    // X lies in the closed element when all three sub-triangles (X replacing
    // one vertex) are counter-clockwise or flat (exact signs); its
    // barycentric coordinates are then the sub-triangle orientations over
    // the element's own orientation.
    if (orient_sign(px, d[1], d[2]) >= 0 && orient_sign(d[0], px, d[2]) >= 0 &&
        orient_sign(d[0], d[1], px) >= 0) {
      double o = orient3(d[0], d[1], d[2]);
      double s0 = orient3(px, d[1], d[2]);
      double s1 = orient3(d[0], px, d[2]);
      double s2 = orient3(d[0], d[1], px);
      double l0 = s0 / o, l1 = s1 / o, l2 = s2 / o;
      mv.x = X;
      mv.y = Y;
      mv.m00 = (l0 * d[0].m00 + l1 * d[1].m00) + l2 * d[2].m00;
      mv.m01 = (l0 * d[0].m01 + l1 * d[1].m01) + l2 * d[2].m01;
      mv.m11 = (l0 * d[0].m11 + l1 * d[1].m11) + l2 * d[2].m11;
      return true;
    }
  }
  return false;
}

// Ball check with v relocated to mv: all elements counter-clockwise; returns
// min and sum of the new qualities.
bool ball_after_move(const OMesh& m, int v, const Move& mv, double& qmin, double& qsum) {
  VD nv{mv.x, mv.y, mv.m00, mv.m01, mv.m11};
  bool first = true;
  qmin = 0.0;
  qsum = 0.0;
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    VD d[3];
    for (int i = 0; i < 3; ++i) d[i] = (t[i] == v) ? nv : m.vd(t[i]);
    if (orient_sign(d[0], d[1], d[2]) <= 0) return false;
    double q = quality_c(t[0], t[1], t[2], d[0], d[1], d[2]);
    if (first || q < qmin) qmin = q;
    first = false;
    qsum = qsum + q;
  }
  return true;
}

bool smooth_eval(const OMesh& m, int v, const Params& P, Move& mv) {
  if (!m.valive[v] || m.vbnd[v]) return false;
  double qold = ball_min_quality(m, v);
  if (!(qold < P.q_thresh)) return false;
  double a00 = 0.0, a01 = 0.0, a11 = 0.0, b0 = 0.0, b1 = 0.0;
  for (int j : m.NN[v]) {
    double w00 = 0.5 * (m.m00[v] + m.m00[j]);
    double w01 = 0.5 * (m.m01[v] + m.m01[j]);
    double w11 = 0.5 * (m.m11[v] + m.m11[j]);
    a00 = a00 + w00;
    a01 = a01 + w01;
    a11 = a11 + w11;
    b0 = b0 + (w00 * m.x[j] + w01 * m.y[j]);
    b1 = b1 + (w01 * m.x[j] + w11 * m.y[j]);
  }
  double det = a00 * a11 - a01 * a01;
  if (!(det > 0.0)) return false;
  double X = (a11 * b0 - a01 * b1) / det;
  double Y = (a00 * b1 - a01 * b0) / det;
  if (!interpolate_in_ball(m, v, X, Y, mv)) return false;
  double qmin, qsum;
  if (!ball_after_move(m, v, mv, qmin, qsum)) return false;
  return qmin > qold;
}

// Optimisation-based smoothing (Sec. 2.4.4, the "more expensive" variant),
// in gradient form: ascend the ball's quality sum along its gradient with
// respect to v's coordinates (metric held fixed), step 0.1 * shortest
// incident Euclidean edge / |g|, halved up to five times; a step is kept when
// all elements stay counter-clockwise, the minimum quality does not drop and
// the quality sum increases.  Parity: convention, pinned by the step rule
// checked against the finite-difference-pinned gradient and the Euclidean
// edge lengths, and by the monotone property.
bool opt_eval(const OMesh& m, int v, Move& mv) {
  if (!m.valive[v] || m.vbnd[v]) return false;
  double gx = 0.0, gy = 0.0;
  for (int K : m.NE[v]) {
    const auto& t = m.tri[K];
    double g[3][5];
    quality_grad_c(t[0], t[1], t[2], m.vd(t[0]), m.vd(t[1]), m.vd(t[2]), g);
    int i = (t[0] == v) ? 0 : (t[1] == v) ? 1 : 2;
    gx = gx + g[i][0];
    gy = gy + g[i][1];
  }
  double gn = std::sqrt(gx * gx + gy * gy);
  if (!(gn > 0.0)) return false;
  double lmin = 0.0;
  bool first = true;
  for (int j : m.NN[v]) {
    double dx = m.x[j] - m.x[v];
    double dy = m.y[j] - m.y[v];
    double l = std::sqrt(dx * dx + dy * dy);
    if (first || l < lmin) lmin = l;
    first = false;
  }
  double qsum_old;
  double qmin_old = ball_min_quality(m, v, &qsum_old);
  double alpha = (0.1 * lmin) / gn;
  for (int k = 0; k < 6; ++k) {
    double X = m.x[v] + alpha * gx;
    double Y = m.y[v] + alpha * gy;
    Move cand;
    if (interpolate_in_ball(m, v, X, Y, cand)) {
      double qmin, qsum;
      if (ball_after_move(m, v, cand, qmin, qsum) && qmin >= qmin_old && qsum > qsum_old) {
        mv = cand;
        return true;
      }
    }
    alpha = alpha * 0.5;
  }
  return false;
}

void apply_move(OMesh& m, int v, const Move& mv) {
  m.x[v] = mv.x;
  m.y[v] = mv.y;
  m.m00[v] = mv.m00;
  m.m01[v] = mv.m01;
  m.m11[v] = mv.m11;
}

// ---------------------------------------------------------------------------
// Round-equals-sequential self check (Sec. 3.2 claim that an independent set
// can be processed concurrently): the round's operations, applied one at a
// time in ascending id order to a copy of the pre-round mesh and re-validated
// against that copy's current state, must all stay valid and reach the same
// mesh as the concurrent round.
// ---------------------------------------------------------------------------

bool same_state(const OMesh& a, const OMesh& b) {
  return a.x == b.x && a.y == b.y && a.m00 == b.m00 && a.m01 == b.m01 && a.m11 == b.m11 &&
         a.valive == b.valive && a.tri == b.tri && a.talive == b.talive && a.NN == b.NN &&
         a.NE == b.NE;
}

void clear_dead_rows(OMesh& m) {
  for (int v = 0; v < m.nv(); ++v)
    if (!m.valive[v]) {
      m.NN[v].clear();
      m.NE[v].clear();
    }
}

// ---------------------------------------------------------------------------
// Operators.  Each runs rounds until no candidate is left (propagation,
// Sec. 2.4.5).  Round counter r advances by one for every round that formed a
// non-empty candidate set.
// ---------------------------------------------------------------------------

bool round_cap(const Params& P, int64_t rounds_this_call) {
  return P.max_rounds > 0 && rounds_this_call >= P.max_rounds;
}

int64_t op_coarsen(OMesh& m, const Params& P, Stats& st) {
  int nv = m.nv();
  std::vector<uint8_t> dirty(nv, 0), inC(nv, 0);
  for (int v = 0; v < nv; ++v) dirty[v] = m.valive[v];
  std::vector<int> target(nv, -1);
  int64_t ops = 0, rounds = 0;
  const bool by_colour = P.select_mode == 1;
  if (by_colour) colour_vertices(m, P.seed);
  while (!round_cap(P, rounds)) {
    std::vector<int> C;
    for (int v = 0; v < nv; ++v) {
      inC[v] = 0;
      if (!dirty[v]) continue;
      target[v] = coarsen_target(m, v, P);
      if (target[v] >= 0) {
        C.push_back(v);
        inC[v] = 1;
      } else {
        dirty[v] = 0;
      }
    }
    if (C.empty()) break;
    std::vector<int> S = independent_set(m, inC, C, P.seed, by_colour);
    m.r += 1;
    ++rounds;
    OMesh before;
    if (m.check_seq) before = m;
    std::vector<Rec> recs;
    for (int v : S) {
      dirty[v] = 0;
      for (int x : m.NN[v]) dirty[x] = 1;
      apply_collapse(m, v, target[v], recs);
    }
    commit(m, recs);
    clear_dead_rows(m);
    ops += (int64_t)S.size();
    if (m.check_seq) {
      for (int v : S) {
        if (!collapse_valid(before, v, target[v], P)) m.seq_fail = 1;
        std::vector<Rec> one;
        apply_collapse(before, v, target[v], one);
        commit(before, one);
        clear_dead_rows(before);
      }
      if (!same_state(before, m)) m.seq_fail = 1;
      if (check_invariants(m) != 0) m.seq_fail = 2;
    }
  }
  st.rounds += rounds;
  st.collapses += ops;
  return ops;
}

int64_t op_swap(OMesh& m, const Params& P, Stats& st) {
  int nv = m.nv();
  std::vector<uint8_t> dirty(nv, 0), inC(nv, 0);
  for (int v = 0; v < nv; ++v) dirty[v] = m.valive[v];
  std::vector<SwapOp> ops_of(nv);
  int64_t ops = 0, rounds = 0;
  const bool by_colour = P.select_mode == 1;
  if (by_colour) colour_vertices(m, P.seed);
  while (!round_cap(P, rounds)) {
    std::vector<int> C;
    for (int v = 0; v < nv; ++v) {
      inC[v] = 0;
      if (!dirty[v]) continue;
      if (swap_eval(m, v, P, ops_of[v])) {
        C.push_back(v);
        inC[v] = 1;
      } else {
        dirty[v] = 0;
      }
    }
    if (C.empty()) break;
    std::vector<int> S = independent_set(m, inC, C, P.seed, by_colour);
    m.r += 1;
    ++rounds;
    OMesh before;
    if (m.check_seq) before = m;
    std::vector<Rec> recs;
    for (int v : S) {
      const SwapOp& op = ops_of[v];
      dirty[v] = dirty[op.w] = dirty[op.c] = dirty[op.d] = 1;
      apply_flip(m, v, op, recs);
    }
    commit(m, recs);
    ops += (int64_t)S.size();
    if (m.check_seq) {
      for (int v : S) {
        SwapOp again;
        if (!flip_candidate(before, v, ops_of[v].w, P, again) || again.c != ops_of[v].c ||
            again.d != ops_of[v].d)
          m.seq_fail = 1;
        std::vector<Rec> one;
        apply_flip(before, v, ops_of[v], one);
        commit(before, one);
      }
      if (!same_state(before, m)) m.seq_fail = 1;
      if (check_invariants(m) != 0) m.seq_fail = 2;
    }
  }
  st.rounds += rounds;
  st.flips += ops;
  return ops;
}

// Refinement (Sec. 2.4.2): split every edge whose metric length exceeds L_up
// at its midpoint (coordinates and metric averaged), then divide each element
// by the template for its number of split edges.  New ids follow ascending
// (owner a = smaller end, other end b) for vertices and ascending parent id
// for elements, so they are reproducible.  Convention for the two-split
// template: the trapezoid is cut along its metric-shorter diagonal (tie: the
// one from the first unsplit-edge vertex).  Parity: convention, pinned by the
// closed-form uniform-grid count, a two-split case whose metric-shorter
// diagonal is the Euclidean longer one, linear metric fields at midpoints,
// and invariants.
int64_t refine_round(OMesh& m, const Params& P, Stats& st) {
  int nv0 = m.nv(), ne0 = m.ne();
  // mid[a] = list of (b, new id), b ascending
  std::vector<std::vector<std::pair<int, int>>> mid(nv0);
  int64_t nsplit = 0;
  for (int a = 0; a < nv0; ++a) {
    if (!m.valive[a]) continue;
    for (int b : m.NN[a]) {
      if (b <= a) continue;
      if (!(metric_len(m.vd(a), m.vd(b)) > P.L_up)) continue;
      int id = m.nv();
      mid[a].push_back({b, id});
      ++nsplit;
      VD da = m.vd(a), db = m.vd(b);
      m.x.push_back(0.5 * (da.x + db.x));
      m.y.push_back(0.5 * (da.y + db.y));
      m.m00.push_back(0.5 * (da.m00 + db.m00));
      m.m01.push_back(0.5 * (da.m01 + db.m01));
      m.m11.push_back(0.5 * (da.m11 + db.m11));
      m.valive.push_back(1);
      m.vbnd.push_back(edge_elements(m, a, b) == 1 ? 1 : 0);
      m.vcorner.push_back(0);
    }
  }
  if (nsplit == 0) return 0;
  auto midpoint = [&](int p, int q) -> int {
    int a = p < q ? p : q, b = p < q ? q : p;
    for (const auto& e : mid[a])
      if (e.first == b) return e.second;
    return -1;
  };
  auto emit = [&](int K, bool first, int a, int b, int c) {
    if (first) {
      m.tri[K] = {a, b, c};
    } else {
      m.tri.push_back({a, b, c});
      m.talive.push_back(1);
    }
  };
  for (int K = 0; K < ne0; ++K) {
    if (!m.talive[K]) continue;
    std::array<int, 3> t = m.tri[K];
    int mi[3];
    int ns = 0;
    for (int i = 0; i < 3; ++i) {
      mi[i] = midpoint(t[i], t[(i + 1) % 3]);
      if (mi[i] >= 0) ++ns;
    }
    if (ns == 1) {
      int i = (mi[0] >= 0) ? 0 : (mi[1] >= 0) ? 1 : 2;
      int a = t[i], b = t[(i + 1) % 3], o = t[(i + 2) % 3], mm = mi[i];
      emit(K, true, a, mm, o);
      emit(K, false, mm, b, o);
    } else if (ns == 2) {
      int j = (mi[0] < 0) ? 0 : (mi[1] < 0) ? 1 : 2;  // the unsplit edge
      int s = (j + 1) % 3;
      int u0 = t[s], u1 = t[(s + 1) % 3], u2 = t[(s + 2) % 3];
      int m0 = mi[s], m1 = mi[(s + 1) % 3];
      emit(K, true, m0, u1, m1);
      double d1 = metric_len(m.vd(u0), m.vd(m1));
      double d2 = metric_len(m.vd(m0), m.vd(u2));
      if (d1 <= d2) {
        emit(K, false, u0, m0, m1);
        emit(K, false, u0, m1, u2);
      } else {
        emit(K, false, u0, m0, u2);
        emit(K, false, m0, m1, u2);
      }
    } else if (ns == 3) {
      int v0 = t[0], v1 = t[1], v2 = t[2];
      int m0 = mi[0], m1 = mi[1], m2 = mi[2];
      emit(K, true, v0, m0, m2);
      emit(K, false, m0, v1, m1);
      emit(K, false, m2, m1, v2);
      emit(K, false, m0, m1, m2);
    }
  }
  rebuild_adjacency(m);
  st.splits += nsplit;
  return nsplit;
}

int64_t op_refine(OMesh& m, const Params& P, Stats& st) {
  int64_t total = 0, rounds = 0;
  while (!round_cap(P, rounds)) {
    int64_t n = refine_round(m, P, st);
    if (n == 0) break;
    if (m.check_seq && check_invariants(m) != 0) m.seq_fail = 2;
    m.r += 1;
    ++rounds;
    total += n;
  }
  st.rounds += rounds;
  return total;
}

int64_t op_smooth_laplace(OMesh& m, const Params& P, Stats& st) {
  int nv = m.nv();
  std::vector<uint8_t> pending(nv, 0), next(nv, 0), inC(nv, 0);
  for (int v = 0; v < nv; ++v) pending[v] = m.valive[v] && !m.vbnd[v];
  std::vector<Move> mv(nv);
  int64_t moves = 0, rounds = 0;
  // smoothing changes no topology: one colouring serves every sweep
  const bool by_colour = P.select_mode == 1;
  if (by_colour) colour_vertices(m, P.seed);
  for (int sweep = 0; sweep < P.max_smooth_sweeps; ++sweep) {
    int64_t moved_sweep = 0;
    std::fill(next.begin(), next.end(), 0);
    while (!round_cap(P, rounds)) {
      std::vector<int> C;
      for (int v = 0; v < nv; ++v) {
        inC[v] = 0;
        if (!pending[v]) continue;
        if (smooth_eval(m, v, P, mv[v])) {
          C.push_back(v);
          inC[v] = 1;
        } else {
          pending[v] = 0;
        }
      }
      if (C.empty()) break;
      std::vector<int> S = independent_set(m, inC, C, P.seed, by_colour);
      m.r += 1;
      ++rounds;
      OMesh before;
      if (m.check_seq) before = m;
      for (int v : S) {
        apply_move(m, v, mv[v]);
        pending[v] = 0;
        for (int j : m.NN[v])
          if (m.valive[j] && !m.vbnd[j]) next[j] = 1;
      }
      moved_sweep += (int64_t)S.size();
      if (m.check_seq) {
        for (int v : S) {
          Move again;
          if (!smooth_eval(before, v, P, again) || again.x != mv[v].x || again.y != mv[v].y ||
              again.m00 != mv[v].m00 || again.m01 != mv[v].m01 || again.m11 != mv[v].m11)
            m.seq_fail = 1;
          apply_move(before, v, mv[v]);
        }
        if (!same_state(before, m)) m.seq_fail = 1;
      }
    }
    moves += moved_sweep;
    if (moved_sweep == 0) break;
    pending.swap(next);
  }
  st.rounds += rounds;
  st.moves += moves;
  return moves;
}

int64_t op_smooth_opt(OMesh& m, const Params& P, Stats& st) {
  int nv = m.nv();
  std::vector<uint8_t> inC(nv, 0);
  std::vector<Move> mv(nv);
  int64_t moves = 0, rounds = 0;
  for (int it = 0; it < P.opt_smooth_rounds; ++it) {
    if (round_cap(P, rounds)) break;
    std::vector<int> C;
    for (int v = 0; v < nv; ++v) {
      inC[v] = m.valive[v] && !m.vbnd[v];
      if (inC[v]) C.push_back(v);
    }
    if (C.empty()) break;
    std::vector<int> S = independent_set(m, inC, C, P.seed);
    m.r += 1;
    ++rounds;
    std::vector<int> mover;
    for (int v : S)
      if (opt_eval(m, v, mv[v])) mover.push_back(v);
    for (int v : mover) apply_move(m, v, mv[v]);
    moves += (int64_t)mover.size();
  }
  st.rounds += rounds;
  st.moves += moves;
  return moves;
}

// Renumbering: stable compaction of live vertices and elements (ascending old
// id); adjacency rows stay sorted because the map is monotone.
void renumber(OMesh& m) {
  int nv = m.nv(), ne = m.ne();
  std::vector<int> vmap(nv, -1), emap(ne, -1);
  int k = 0;
  for (int v = 0; v < nv; ++v)
    if (m.valive[v]) vmap[v] = k++;
  int nvn = k;
  k = 0;
  for (int K = 0; K < ne; ++K)
    if (m.talive[K]) emap[K] = k++;
  int nen = k;
  OMesh o;
  o.r = m.r;
  o.check_seq = m.check_seq;
  o.seq_fail = m.seq_fail;
  o.euler0 = m.euler0;
  for (int v = 0; v < nv; ++v) {
    if (vmap[v] < 0) continue;
    o.x.push_back(m.x[v]);
    o.y.push_back(m.y[v]);
    o.m00.push_back(m.m00[v]);
    o.m01.push_back(m.m01[v]);
    o.m11.push_back(m.m11[v]);
    o.valive.push_back(1);
    o.vbnd.push_back(m.vbnd[v]);
    o.vcorner.push_back(m.vcorner[v]);
    std::vector<int> nn, nel;
    for (int u : m.NN[v]) nn.push_back(vmap[u]);
    for (int K : m.NE[v]) nel.push_back(emap[K]);
    o.NN.push_back(nn);
    o.NE.push_back(nel);
  }
  for (int K = 0; K < ne; ++K) {
    if (emap[K] < 0) continue;
    const auto& t = m.tri[K];
    o.tri.push_back({vmap[t[0]], vmap[t[1]], vmap[t[2]]});
    o.talive.push_back(1);
  }
  (void)nvn;
  (void)nen;
  m = std::move(o);
}

// ---------------------------------------------------------------------------
// Invariants (checked after rounds in the tests): conformity, orientation,
// adjacency equal to its definition, boundary flags, Euler characteristic of
// a disk.  Returns 0 when all hold, else a code naming the first failure.
// ---------------------------------------------------------------------------

int64_t euler_characteristic(const OMesh& m);

int check_invariants(const OMesh& m) {
  OMesh ref = m;
  rebuild_adjacency(ref);
  for (int v = 0; v < m.nv(); ++v) {
    if (!m.valive[v]) continue;
    if (ref.NN[v] != m.NN[v]) return 10;
    if (ref.NE[v] != m.NE[v]) return 11;
    if (m.NE[v].empty()) return 12;
    size_t a = m.NN[v].size(), b = m.NE[v].size();
    bool bnd = (a == b + 1);
    if (!(a == b || a == b + 1)) return 13;
    if ((bool)m.vbnd[v] != bnd) return 14;
  }
  // directed edges unique (no overlapping elements), undirected edges in 1 or 2
  std::vector<std::vector<int>> out(m.nv());
  int64_t V = 0, F = 0, E2 = 0, EB = 0;
  for (int K = 0; K < m.ne(); ++K) {
    if (!m.talive[K]) continue;
    ++F;
    const auto& t = m.tri[K];
    for (int i = 0; i < 3; ++i) {
      if (!m.valive[t[i]]) return 15;
      out[t[i]].push_back(t[(i + 1) % 3]);
    }
    VD d0 = m.vd(t[0]), d1 = m.vd(t[1]), d2 = m.vd(t[2]);
    if (orient_sign(d0, d1, d2) <= 0) return 16;
  }
  for (int v = 0; v < m.nv(); ++v) {
    std::vector<int> o = out[v];
    std::sort(o.begin(), o.end());
    if (std::adjacent_find(o.begin(), o.end()) != o.end()) return 17;
    if (m.valive[v]) ++V;
    for (int w : out[v]) {
      // edge v->w; its reverse w->v exists iff interior
      bool rev = std::find(out[w].begin(), out[w].end(), v) != out[w].end();
      if (rev) {
        if (v < w) ++E2;
      } else {
        ++EB;
      }
    }
  }
  int64_t E = E2 + EB;
  if (V - E + F != m.euler0) return 18;
  return 0;
}

int64_t euler_characteristic(const OMesh& m) {
  std::vector<std::vector<int>> nbr(m.nv());
  int64_t V = 0, F = 0, E = 0;
  for (int K = 0; K < m.ne(); ++K) {
    if (!m.talive[K]) continue;
    ++F;
    for (int i = 0; i < 3; ++i) nbr[m.tri[K][i]].push_back(m.tri[K][(i + 1) % 3]);
  }
  for (int v = 0; v < m.nv(); ++v) {
    if (m.valive[v]) ++V;
    for (int w : nbr[v]) {
      bool rev = std::find(nbr[w].begin(), nbr[w].end(), v) != nbr[w].end();
      if (!rev || v < w) ++E;
    }
  }
  return V - E + F;
}

int validate_params(const Params* P) {
  if (!P) return ERR_INVALID_ARG;
  if (!(P->L_low > 0.0) || !(P->L_up > P->L_low) || !std::isfinite(P->L_up)) return ERR_INVALID_ARG;
  if (!(P->q_thresh >= 0.0) || !std::isfinite(P->q_thresh)) return ERR_INVALID_ARG;
  if (P->max_iter < 0 || P->max_smooth_sweeps < 0 || P->opt_smooth_rounds < 0 || P->max_rounds < 0)
    return ERR_INVALID_ARG;
  return OK;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the tests (ctypes).
// ---------------------------------------------------------------------------

extern "C" {

// Exact orientation sign of (p, q, r), pts = {px, py, qx, qy, rx, ry}.
int32_t or_orient_sign(const double* pts) {
  VD p{pts[0], pts[1], 0.0, 0.0, 0.0}, q{pts[2], pts[3], 0.0, 0.0, 0.0},
      r{pts[4], pts[5], 0.0, 0.0, 0.0};
  return orient_sign(p, q, r);
}


typedef struct OMesh or_mesh;

// Copies the input; derives boundary flags from the elements and corners from
// non-collinear boundary neighbours unless `corner` is given.  Returns null and
// sets *status on invalid input.
or_mesh* or_create(const double* xy, int32_t nv, const int32_t* tri, int32_t ne,
                   const uint8_t* corner, int32_t* status) {
  *status = OK;
  if (!xy || !tri || nv < 3 || ne < 1) {
    *status = ERR_INVALID_ARG;
    return nullptr;
  }
  OMesh* m = new OMesh();
  for (int v = 0; v < nv; ++v) {
    m->x.push_back(xy[2 * v]);
    m->y.push_back(xy[2 * v + 1]);
    m->m00.push_back(1.0);
    m->m01.push_back(0.0);
    m->m11.push_back(1.0);
    m->valive.push_back(1);
  }
  for (int K = 0; K < ne; ++K) {
    std::array<int, 3> t = {tri[3 * K], tri[3 * K + 1], tri[3 * K + 2]};
    for (int i = 0; i < 3; ++i)
      if (t[i] < 0 || t[i] >= nv) {
        *status = ERR_INVALID_MESH;
        delete m;
        return nullptr;
      }
    if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) {
      *status = ERR_INVALID_MESH;
      delete m;
      return nullptr;
    }
    m->tri.push_back(t);
    m->talive.push_back(1);
  }
  rebuild_adjacency(*m);
  m->vbnd.assign(nv, 0);
  m->vcorner.assign(nv, 0);
  for (int v = 0; v < nv; ++v) {
    if (m->NE[v].empty()) {
      *status = ERR_INVALID_MESH;
      delete m;
      return nullptr;
    }
    size_t a = m->NN[v].size(), b = m->NE[v].size();
    if (a == b + 1) m->vbnd[v] = 1;
  }
  for (int v = 0; v < nv; ++v) {
    if (corner) {
      m->vcorner[v] = corner[v] ? 1 : 0;
      continue;
    }
    if (!m->vbnd[v]) continue;
    int bn[2], k = 0;
    for (int w : m->NN[v])
      if (edge_elements(*m, v, w) == 1 && k < 2) bn[k++] = w;
    if (k < 2) {
      m->vcorner[v] = 1;
      continue;
    }
    int lo = bn[0] < bn[1] ? bn[0] : bn[1], hi = bn[0] < bn[1] ? bn[1] : bn[0];
    m->vcorner[v] = orient_sign(m->vd(lo), m->vd(v), m->vd(hi)) != 0 ? 1 : 0;
  }
  m->euler0 = euler_characteristic(*m);
  int inv = check_invariants(*m);
  if (inv != 0) {
    *status = ERR_INVALID_MESH;
    delete m;
    return nullptr;
  }
  return m;
}

void or_destroy(or_mesh* m) { delete m; }

int32_t or_set_metric(or_mesh* m, const double* M) {
  if (!m || !M) return ERR_INVALID_ARG;
  for (int v = 0; v < m->nv(); ++v) {
    double a = M[3 * v], b = M[3 * v + 1], c = M[3 * v + 2];
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c) || !(a > 0.0) ||
        !(a * c - b * b > 0.0))
      return ERR_INVALID_ARG;
  }
  for (int v = 0; v < m->nv(); ++v) {
    m->m00[v] = M[3 * v];
    m->m01[v] = M[3 * v + 1];
    m->m11[v] = M[3 * v + 2];
  }
  return OK;
}

void or_set_check_sequential(or_mesh* m, int32_t on) { m->check_seq = on != 0; }
int32_t or_seq_failed(or_mesh* m) { return m->seq_fail; }

#define OR_OP(name, body)                                           \
  int32_t name(or_mesh* m, const Params* P, Stats* st) {            \
    int e = validate_params(P);                                     \
    if (e) return e;                                                \
    Stats local{};                                                  \
    double t0 = now_ms();                                           \
    m->r = 0;                                                       \
    body;                                                           \
    local.ms = now_ms() - t0;                                       \
    if (st) *st = local;                                            \
    return OK;                                                      \
  }

OR_OP(or_coarsen, op_coarsen(*m, *P, local))
OR_OP(or_swap, op_swap(*m, *P, local))
OR_OP(or_refine, op_refine(*m, *P, local))
OR_OP(or_smooth, {
  op_smooth_laplace(*m, *P, local);
  op_smooth_opt(*m, *P, local);
})
OR_OP(or_opt_smooth, op_smooth_opt(*m, *P, local))

// Algorithm 1 (Sec. 2.3) followed by smoothing and renumbering.
OR_OP(or_adapt, {
  local.converged = 0;
  for (int it = 0; it < P->max_iter; ++it) {
    int64_t n = op_coarsen(*m, *P, local);
    n += op_swap(*m, *P, local);
    n += op_refine(*m, *P, local);
    renumber(*m);
    if (n == 0) {
      local.converged = 1;
      break;
    }
  }
  op_smooth_laplace(*m, *P, local);
  op_smooth_opt(*m, *P, local);
  renumber(*m);
})

int32_t or_renumber(or_mesh* m) {
  renumber(*m);
  return OK;
}

// Compacted copy in canonical order: live vertices and elements by ascending
// id, each element rotated so that its smallest vertex id comes first.
// Null arrays: only the sizes are written.
int32_t or_get_mesh(or_mesh* m, int32_t* nv, int32_t* ne, double* xy, int32_t* tri, double* M) {
  OMesh c = *m;
  renumber(c);
  *nv = c.nv();
  *ne = c.ne();
  if (xy)
    for (int v = 0; v < c.nv(); ++v) {
      xy[2 * v] = c.x[v];
      xy[2 * v + 1] = c.y[v];
    }
  if (M)
    for (int v = 0; v < c.nv(); ++v) {
      M[3 * v] = c.m00[v];
      M[3 * v + 1] = c.m01[v];
      M[3 * v + 2] = c.m11[v];
    }
  if (tri)
    for (int K = 0; K < c.ne(); ++K) {
      auto t = c.tri[K];
      int s = 0;
      if (t[1] < t[s]) s = 1;
      if (t[2] < t[s]) s = 2;
      for (int i = 0; i < 3; ++i) tri[3 * K + i] = t[(s + i) % 3];
    }
  return OK;
}

// Raw slot state (dead slots included) for round-level comparisons.
int32_t or_get_raw(or_mesh* m, int32_t* nv, int32_t* ne, double* xy, double* M, int32_t* tri,
                   uint8_t* valive, uint8_t* talive, uint8_t* vflag) {
  *nv = m->nv();
  *ne = m->ne();
  if (!xy) return OK;
  for (int v = 0; v < m->nv(); ++v) {
    xy[2 * v] = m->x[v];
    xy[2 * v + 1] = m->y[v];
    M[3 * v] = m->m00[v];
    M[3 * v + 1] = m->m01[v];
    M[3 * v + 2] = m->m11[v];
    valive[v] = m->valive[v];
    vflag[v] = (uint8_t)((m->vbnd[v] ? 1 : 0) | (m->vcorner[v] ? 2 : 0));
  }
  for (int K = 0; K < m->ne(); ++K) {
    for (int i = 0; i < 3; ++i) tri[3 * K + i] = m->tri[K][i];
    talive[K] = m->talive[K];
  }
  return OK;
}

// Sorted adjacency rows of vertex v (cap entries at most); returns row sizes.
int32_t or_adjacency(or_mesh* m, int32_t v, int32_t* nn, int32_t* nnlen, int32_t* ne,
                     int32_t* nelen, int32_t cap) {
  if (v < 0 || v >= m->nv()) return ERR_INVALID_ARG;
  *nnlen = (int32_t)m->NN[v].size();
  *nelen = (int32_t)m->NE[v].size();
  for (int i = 0; i < *nnlen && i < cap; ++i) nn[i] = m->NN[v][i];
  for (int i = 0; i < *nelen && i < cap; ++i) ne[i] = m->NE[v][i];
  return OK;
}

int32_t or_check(or_mesh* m) { return check_invariants(*m); }

// Per-slot quality (NaN for dead slots).
int32_t or_quality_elems(or_mesh* m, double* q) {
  for (int K = 0; K < m->ne(); ++K) q[K] = m->talive[K] ? quality_of(*m, K) : NAN;
  return OK;
}

// Sum of element qualities over live elements (ascending id) and, if given,
// its gradient: per vertex slot, the sum over incident elements in ascending
// element id of dq/d(x,y) and dq/d(m00,m01,m11).
int32_t or_quality(or_mesh* m, double* qsum, double* dxy, double* dM) {
  double s = 0.0;
  for (int K = 0; K < m->ne(); ++K)
    if (m->talive[K]) s = s + quality_of(*m, K);
  *qsum = s;
  if (!dxy && !dM) return OK;
  for (int v = 0; v < m->nv(); ++v) {
    double acc[5] = {0, 0, 0, 0, 0};
    if (m->valive[v])
      for (int K : m->NE[v]) {
        const auto& t = m->tri[K];
        double g[3][5];
        quality_grad_c(t[0], t[1], t[2], m->vd(t[0]), m->vd(t[1]), m->vd(t[2]), g);
        int i = (t[0] == v) ? 0 : (t[1] == v) ? 1 : 2;
        for (int j = 0; j < 5; ++j) acc[j] = acc[j] + g[i][j];
      }
    if (dxy) {
      dxy[2 * v] = acc[0];
      dxy[2 * v + 1] = acc[1];
    }
    if (dM) {
      dM[3 * v] = acc[2];
      dM[3 * v + 1] = acc[3];
      dM[3 * v + 2] = acc[4];
    }
  }
  return OK;
}

// Single-triangle arithmetic, exposed for the closed-form pins.
double or_tri_quality(const int32_t* ids, const double* xy, const double* M) {
  VD d[3];
  for (int i = 0; i < 3; ++i) d[i] = VD{xy[2 * i], xy[2 * i + 1], M[3 * i], M[3 * i + 1], M[3 * i + 2]};
  return quality_c(ids[0], ids[1], ids[2], d[0], d[1], d[2]);
}

double or_tri_quality_grad(const int32_t* ids, const double* xy, const double* M, double* g15) {
  VD d[3];
  for (int i = 0; i < 3; ++i) d[i] = VD{xy[2 * i], xy[2 * i + 1], M[3 * i], M[3 * i + 1], M[3 * i + 2]};
  double g[3][5];
  double q = quality_grad_c(ids[0], ids[1], ids[2], d[0], d[1], d[2], g);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 5; ++j) g15[5 * i + j] = g[i][j];
  return q;
}

double or_edge_length(const double* xya, const double* Ma, const double* xyb, const double* Mb) {
  VD a{xya[0], xya[1], Ma[0], Ma[1], Ma[2]}, b{xyb[0], xyb[1], Mb[0], Mb[1], Mb[2]};
  return metric_len(a, b);
}

uint32_t or_fmix32(uint32_t h) { return fmix32(h); }
uint32_t or_prio(uint32_t v, uint32_t seed, uint32_t r) { return prio(v, seed, r); }

// Independent set of the given candidate flags on the current vertex graph,
// with round counter r (by_colour: among the candidates of colour r mod the
// number of colours, from the mesh's last colouring).  Writes 0/1 per vertex
// slot.
int32_t or_independent_set(or_mesh* m, const uint8_t* cand, uint32_t seed, uint32_t r,
                           int32_t by_colour, uint8_t* inS) {
  std::vector<uint8_t> inC(cand, cand + m->nv());
  std::vector<int> C;
  for (int v = 0; v < m->nv(); ++v)
    if (inC[v] && m->valive[v]) C.push_back(v);
  uint32_t keep = m->r;
  m->r = r;
  std::vector<int> S = independent_set(*m, inC, C, seed, by_colour != 0);
  m->r = keep;
  std::memset(inS, 0, (size_t)m->nv());
  for (int v : S) inS[v] = 1;
  return OK;
}

// Colours of the vertex graph as a pass with round counter r colours it
// (-1 for dead slots); returns the number of colours.
int32_t or_colour(or_mesh* m, uint32_t seed, uint32_t r, int32_t* col) {
  const uint32_t keep = m->r;
  m->r = r;
  colour_vertices(*m, seed);
  m->r = keep;
  for (int v = 0; v < m->nv(); ++v) col[v] = m->col[v];
  return m->ncol;
}

int32_t or_coarsen_target(or_mesh* m, int32_t v, const Params* P) { return coarsen_target(*m, v, *P); }

int32_t or_swap_target(or_mesh* m, int32_t v, const Params* P, int32_t* cd) {
  SwapOp op;
  if (!swap_eval(*m, v, *P, op)) return -1;
  cd[0] = op.c;
  cd[1] = op.d;
  return op.w;
}

}  // extern "C"
