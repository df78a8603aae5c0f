// Shared device-side definitions of the GB300 mesh-adaptation library.
//
// Arithmetic follows the readings of the paper used throughout the library:
// FP64, no contraction of a*b+c (compiled with -fmad=false), every expression
// evaluated in the order written, IEEE-correct division and square root.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pm.h"

namespace pm {

// ---------------------------------------------------------------------------
// Storage layout (structure of arrays; all meshes of a batch share the arrays,
// each mesh owns the slot ranges [vbase, vbase + vcap) and [ebase, ebase + ecap)).
// Ids stored in EN / NN / NE are LOCAL to the mesh (slot - base).
// ---------------------------------------------------------------------------

enum : uint8_t { VF_ALIVE = 1, VF_BND = 2, VF_CORNER = 4 };

// Per-mesh table (device copy); arrays of length nmesh.
struct MeshTab {
  int* vbase;
  int* vcap;
  int* ebase;
  int* ecap;
  int* nv;      // used vertex slots (alive + dead) of each mesh
  int* ne;      // used element slots
  uint32_t* seed;
  uint32_t* r;  // round counter of the current call
  int* had;     // 1 when the mesh formed candidates this round (2 * nmesh)
  int* active;  // mesh takes part in the current phase
  unsigned long long* ops;       // operations applied in the current call
  unsigned long long* iter_ops;  // operations of the current outer iteration
  double* L_low;                 // per-mesh parameters
  double* L_up;
  double* q_thresh;
  double4* band;                 // (L_low_lo^2, L_low_hi^2, L_up_lo^2, L_up_hi^2)
  // 2 * (nmesh + 1) ints: exclusive prefix sums over the meshes of a vertex
  // count and an element count (pre[0..nmesh] vertices, pre[nmesh+1..]
  // elements); the offsets of each mesh in a concatenated input or output.
  int* pre;
  // Mesh of every vertex slot and every element slot (sets of more than one
  // mesh; filled once per layout).
  int* vmesh;
  int* emesh;
  int* select;  // PM_SELECT_* of each mesh
  int* ncol;    // colours of each mesh's current colouring (colour-class sets)
  int* col;     // colour of every vertex slot (colour-class sets; -1: none)
};

struct Store {
  int nmesh;
  int W;          // row capacity of NN and NE
  int vslots;     // total vertex slots (sum of vcap)
  int eslots;     // total element slots
  int vused;      // every slot in use lies below these bounds
  int eused;
  double2* xy;
  double4* M;     // (m00, m01, m11, 0)
  uint8_t* vflag;
  int4* EN;       // (v0, v1, v2, alive)
  double* qK;     // quality of every live element (kept current by all operators)
  int* NN;        // vslots * W
  int* NNlen;
  int* NE;
  int* NElen;
  // Change stamps: touch[v] is the (odd) round stamp of the last change of
  // v's rows or position; ntouch[v] the stamp of the last change of a vertex
  // that was v's neighbour after that change; evc/evs/evm/evr are the (even)
  // round tags of v's last collapse / flip / smoothing / split evaluation.
  // An evaluation whose inputs (v, its rows, its neighbours' rows and
  // positions) carry no newer stamp would give the same answer again.
  int* touch;
  int* ntouch;
  int* evc;
  int* evs;
  int* evm;
  int* evr;
  // Vertex numbering.  A vertex's id is its slot offset in its mesh's region,
  // except after a renumbering that left the slots in place: lid[v] is then
  // v's id (its rank among the live slots of its mesh at that renumbering,
  // slots appended since counting on from there) and voff[mesh] is the number
  // of dead slots the ids skip.  Null when ids are the slot offsets.
  int* lid;
  int* voff;
  MeshTab tab;
};

// Status words written by kernels (device).
struct DevStatus {
  int err;       // pm_status set by a kernel (first writer wins)
  int overflow;  // an adjacency row would exceed W
  int maxdeg;    // largest row length seen by the last adjacency build
  int pad;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void set_err(DevStatus* st, int code) {
  atomicCAS(&st->err, 0, code);
}

// Mesh of a global vertex / element slot: one load from the layout's slot
// index (a set of one mesh needs none).
__device__ __forceinline__ int mesh_of_vslot(const Store& S, int slot) {
  return S.nmesh == 1 ? 0 : __ldg(S.tab.vmesh + slot);
}

__device__ __forceinline__ int mesh_of_eslot(const Store& S, int slot) {
  return S.nmesh == 1 ? 0 : __ldg(S.tab.emesh + slot);
}

// Segment of position g in a concatenation: the largest i < n with
// pre[i] <= g (pre: n + 1 ascending exclusive prefix sums).
__device__ __forceinline__ int seg_of(const int* pre, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Warp-aggregated append (the GPU form of the atomic-capture worklist of
// Sec. 3.4): one atomic per warp reserves room for every lane with pred set.
// All 32 lanes of the warp must call it.
__device__ __forceinline__ void warp_append(bool pred, int val, int* list, int* count) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// Room for `cnt` items of this lane in a list: one atomic per warp, the
// lanes' ranges in lane order.  Returns the first slot of this lane.  All 32
// lanes of the warp must call it.
__device__ __forceinline__ int warp_reserve(int cnt, int* count) {
  const int lane = threadIdx.x & 31;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(count, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - cnt;
}

// Writes vb + row[k] for every set bit k of `bits`, from slot `pos` on.
__device__ __forceinline__ void write_row_bits(unsigned long long bits, const int* row, int vb,
                                               int* list, int pos) {
  while (bits) {
    int k = __ffsll((long long)bits) - 1;
    bits &= bits - 1ull;
    list[pos++] = vb + row[k];
  }
}

// A set of entries of one adjacency row (rows hold at most 128 entries): one
// bit per entry, in two named words so that it stays in registers.
struct RowMask {
  unsigned long long lo = 0ull, hi = 0ull;
  __device__ __forceinline__ void set(int k) {
    if (k < 64) lo |= 1ull << k;
    else hi |= 1ull << (k - 64);
  }
  __device__ __forceinline__ bool test(int k) const {
    return k < 64 ? ((lo >> k) & 1ull) != 0ull : ((hi >> (k - 64)) & 1ull) != 0ull;
  }
  __device__ __forceinline__ bool any() const { return (lo | hi) != 0ull; }
  __device__ __forceinline__ int count() const { return __popcll(lo) + __popcll(hi); }
  // the lowest entry, removed from the set
  __device__ __forceinline__ int pop() {
    if (lo) {
      int k = __ffsll((long long)lo) - 1;
      lo &= lo - 1ull;
      return k;
    }
    int k = __ffsll((long long)hi) - 1;
    hi &= hi - 1ull;
    return 64 + k;
  }
  // entries of the set below entry k
  __device__ __forceinline__ int below(int k) const {
    return k < 64 ? __popcll(lo & ((1ull << k) - 1ull))
                  : __popcll(lo) + __popcll(hi & ((1ull << (k - 64)) - 1ull));
  }
};

// Writes vb + row[k] for every entry k of `bits`, from slot `pos` on.
__device__ __forceinline__ void write_row_bits(RowMask bits, const int* row, int vb, int* list,
                                               int pos) {
  while (bits.any()) list[pos++] = vb + row[bits.pop()];
}

template <class T>
__device__ __forceinline__ void warp_append_t(bool pred, T val, T* list, int* count) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// Append once per round: the stamp array holds the tag of the last round in
// which the slot was appended.
__device__ __forceinline__ bool stamp_first(int* stamp, int slot, int tag) {
  return atomicExch(stamp + slot, tag) != tag;
}

// Position of val in the first len entries of an adjacency row, or -1.  A
// row starts on a 64-byte boundary (arrays are 256-byte aligned and the row
// width is a power of two of at least 16), so it is read in 16-byte chunks
// whose loads do not wait on one another (no exit that depends on a loaded
// value): one memory round trip for a row of up to 16 entries instead of a
// chain of dependent loads.  Chunks never pass the row's end (len <= width,
// a multiple of 4); entries at len and beyond are not compared.
__device__ __forceinline__ int row_find(const int* row, int len, int val) {
  const int4* r4 = reinterpret_cast<const int4*>(row);
  int at = -1;
#pragma unroll 4
  for (int k = 0; k < len; k += 4) {
    const int4 q = r4[k >> 2];
    at = (q.w == val && k + 3 < len) ? k + 3 : at;
    at = (q.z == val && k + 2 < len) ? k + 2 : at;
    at = (q.y == val && k + 1 < len) ? k + 1 : at;
    at = (q.x == val) ? k : at;
  }
  return at;
}

__device__ __forceinline__ bool row_has(const int* row, int len, int val) {
  return row_find(row, len, val) >= 0;
}

// Position of val in a sorted array a[0..len) (binary search), or -1.
__device__ __forceinline__ int sorted_pos(const int* a, int len, int val) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < val) lo = mid + 1;
    else hi = mid;
  }
  return (lo < len && a[lo] == val) ? lo : -1;
}

// Copies the first len entries of an adjacency row into out (capacity: the
// row width or more) in 16-byte chunks whose loads do not wait on one
// another; entries of the last chunk past len are copied too and ignored.
__device__ __forceinline__ void load_row(const int* row, int len, int* out) {
  const int4* r4 = reinterpret_cast<const int4*>(row);
#pragma unroll 4
  for (int k = 0; k < len; k += 4) {
    const int4 q = r4[k >> 2];
    out[k] = q.x;
    out[k + 1] = q.y;
    out[k + 2] = q.z;
    out[k + 3] = q.w;
  }
}

// Insert into a sorted small buffer without duplicates; returns false when
// the buffer is full.
__device__ __forceinline__ bool sorted_insert(int* buf, int& n, int cap, int val) {
  int k = n;
  while (k > 0 && buf[k - 1] > val) --k;
  if (k > 0 && buf[k - 1] == val) return true;
  if (n >= cap) return false;
  for (int j = n; j > k; --j) buf[j] = buf[j - 1];
  buf[k] = val;
  ++n;
  return true;
}

__device__ __forceinline__ void sorted_erase(int* buf, int& n, int val) {
  int k = 0;
  while (k < n && buf[k] < val) ++k;
  if (k < n && buf[k] == val) {
    for (int j = k; j < n - 1; ++j) buf[j] = buf[j + 1];
    --n;
  }
}

// ---------------------------------------------------------------------------
// Arithmetic (Sec. 2.2).
// ---------------------------------------------------------------------------

struct VD {
  double x, y, m00, m01, m11;
};

__device__ __forceinline__ VD load_vd(const Store& S, int slot) {
  double2 p = S.xy[slot];
  double4 m = S.M[slot];
  return VD{p.x, p.y, m.x, m.y, m.z};
}

// The position alone, read again through L2 (ld.global.cg, never merged
// with an earlier load): for rarely taken branches that need coordinates the
// hot path no longer holds in registers.
__device__ __forceinline__ VD load_xy_again(const Store& S, int slot) {
  const double2 p = __ldcg(&S.xy[slot]);
  return VD{p.x, p.y, 0.0, 0.0, 0.0};
}

// Metric length of edge (a,b) under the mean of the end-point metrics.
__device__ __forceinline__ double metric_len(const VD& a, const VD& b) {
  double e00 = 0.5 * (a.m00 + b.m00);
  double e01 = 0.5 * (a.m01 + b.m01);
  double e11 = 0.5 * (a.m11 + b.m11);
  double dx = b.x - a.x;
  double dy = b.y - a.y;
  double L2 = ((e00 * dx) * dx + ((2.0 * e01) * dx) * dy) + (e11 * dy) * dy;
  return sqrt(L2);
}

// Squared metric length (the radicand of metric_len, same operations).
__device__ __forceinline__ double metric_len2(const VD& a, const VD& b) {
  double e00 = 0.5 * (a.m00 + b.m00);
  double e01 = 0.5 * (a.m01 + b.m01);
  double e11 = 0.5 * (a.m11 + b.m11);
  double dx = b.x - a.x;
  double dy = b.y - a.y;
  return ((e00 * dx) * dx + ((2.0 * e01) * dx) * dy) + (e11 * dy) * dy;
}

// sqrt(L2) > t and sqrt(L2) < t decided exactly without the square root
// outside a band of relative width 1e-9 around t: lo2 <= (t(1-1e-9))^2 and
// hi2 >= (t(1+1e-9))^2, far wider than the rounding of sqrt or of the squares.
// Comparisons decided on the bit patterns of doubles: GB300 issues FP64
// compares on its scarce FP64 pipe, 64-bit integer compares elsewhere.  For
// non-NaN operands they equal the floating-point comparison when the right
// side b satisfies the stated range: every double below +0 (negatives and -0)
// has a negative pattern, and non-negative doubles order as their patterns.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// a > b for b >= +0 (b not -0)
__device__ __forceinline__ bool dgt(double a, double b) { return dbits(a) > dbits(b); }
// a < b for b > 0
__device__ __forceinline__ bool dlt(double a, double b) { return dbits(a) < dbits(b); }
// a >= 0.0 (true for -0 as well)
__device__ __forceinline__ bool dge0(double a) {
  long long x = dbits(a);
  return x >= 0 || x == (long long)0x8000000000000000ull;
}

// Band tests of a squared length against positive squared bounds.
__device__ __forceinline__ bool len_gt(double L2, double lo2, double hi2, double t) {
  if (dgt(L2, hi2)) return true;
  if (dlt(L2, lo2)) return false;
  return sqrt(L2) > t;
}
__device__ __forceinline__ bool len_lt(double L2, double lo2, double hi2, double t) {
  if (dlt(L2, lo2)) return true;
  if (dgt(L2, hi2)) return false;
  return sqrt(L2) < t;
}

__device__ __forceinline__ double orient3(const VD& p, const VD& q, const VD& r) {
  return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);
}

// Rotate (i0,i1,i2) so that the smallest id comes first (cyclic order kept):
// orientation values (areas, barycentric weights) and qualities are taken in
// this rotation, so they do not depend on how an element is stored.
__device__ __forceinline__ void canon(int& i0, int& i1, int& i2, VD& a, VD& b, VD& c) {
  if (i1 < i0 && i1 < i2) {
    int t = i0; i0 = i1; i1 = i2; i2 = t;
    VD u = a; a = b; b = c; c = u;
  } else if (i2 < i0 && i2 < i1) {
    int t = i2; i2 = i1; i1 = i0; i0 = t;
    VD u = c; c = b; b = a; a = u;
  }
}

// ---------------------------------------------------------------------------
// Exact orientation sign.  Every validity decision (an element
// counter-clockwise, a point in the closed element, a corner) takes the sign
// of det = (q.x - p.x)(r.y - p.y) - (q.y - p.y)(r.x - p.x) of the real
// numbers the doubles stand for, so it depends neither on rounding nor on the
// rotation the triangle is taken in.  A floating-point filter decides when
// |det| clearly exceeds 8 eps (|t1| + |t2|) (eps = 2^-53; the rounding error
// of this form is at most (3 + 16 eps) eps (|t1| + |t2|): J. R. Shewchuk,
// "Adaptive precision floating-point arithmetic and fast robust geometric
// predicates", 1997); otherwise det is summed exactly.  Exact while no product or error
// underflows or overflows (coordinates zero or of magnitude 1e-140..1e140).
// ---------------------------------------------------------------------------

// a + b = s + e exactly (Knuth's two-sum; round to nearest, no contraction)
__device__ __forceinline__ void exact_add(double a, double b, double& s, double& e) {
  s = a + b;
  const double bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// det as an exact sum: each difference is its rounded value plus its error
// (two-sum of a and -b), each of the eight partial products is its rounded
// value plus its error (fused multiply-add), and the sixteen terms are added
// one by one into a list of non-overlapping parts of increasing magnitude
// (each addition a chain of two-sums, zero parts dropped); the sign of the
// sum is the sign of its largest part.  Rarely taken, kept out of line.
static __device__ __noinline__ int orient_sign_exact(double px, double py, double qx, double qy,
                                              double rx, double ry) {
  double a[2], b[2], c[2], d[2];
  exact_add(qx, -px, a[0], a[1]);
  exact_add(ry, -py, b[0], b[1]);
  exact_add(qy, -py, c[0], c[1]);
  exact_add(rx, -px, d[0], d[1]);
  double part[32];
  int n = 0;
  for (int k = 0; k < 16; ++k) {
    const int i = (k >> 2) & 1, j = (k >> 1) & 1;
    const bool second = k & 1;  // the product's error rather than its value
    const bool cd = k >= 8;     // the subtracted product c * d
    const double x = cd ? c[i] : a[i], y = cd ? d[j] : b[j];
    const double pr = x * y;
    double term = second ? __fma_rn(x, y, -pr) : pr;
    if (cd) term = -term;
    double q = term;
    int m = 0;
    for (int u = 0; u < n; ++u) {
      double sum, err;
      exact_add(q, part[u], sum, err);
      if (err != 0.0) part[m++] = err;
      q = sum;
    }
    if (q != 0.0) part[m++] = q;
    n = m;
  }
  if (n == 0) return 0;
  return part[n - 1] > 0.0 ? 1 : -1;
}

// Sign of a double on its bit pattern (-0 and +0 give 0): integer ALUs.
__device__ __forceinline__ int dsign(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b << 1) == 0ull ? 0 : ((b >> 63) ? -1 : 1);
}

// Sign of a * b - c * d for exact doubles a, b, c, d: each product is its
// rounded value plus its error (fused multiply-add), so the difference is
// the exact sum p1 + e1 - p2 - e2.  (e1, p1) is already a non-overlapping
// pair of increasing magnitude; -e2 and then -p2 are added by chains of
// two-sums, leaving four non-overlapping parts (zeros allowed among them)
// whose largest non-zero part carries the sign.  All in registers.
__device__ __forceinline__ int sign_of_product_difference(double a, double b, double c, double d) {
  const double p1 = a * b, e1 = __fma_rn(a, b, -p1);
  const double p2 = c * d, e2 = __fma_rn(c, d, -p2);
  double s, h0, h1, h2, h3;
  exact_add(-e2, e1, s, h0);
  exact_add(s, p1, h2, h1);
  exact_add(-p2, h0, s, h0);
  exact_add(s, h1, s, h1);
  exact_add(s, h2, h3, h2);
  const int s3 = dsign(h3), s2 = dsign(h2), s1 = dsign(h1);
  return s3 != 0 ? s3 : (s2 != 0 ? s2 : (s1 != 0 ? s1 : dsign(h0)));
}

// Error of the rounded difference s = RN(a - b): a - b = s + e exactly.
// Dekker's fast two-sum on the operand of larger magnitude first (chosen on
// the bit patterns): two FP64 operations instead of the six of Knuth's form.
__device__ __forceinline__ double diff_error(double a, double b, double s) {
  const bool abig = ((unsigned long long)__double_as_longlong(a) << 1) >=
                    ((unsigned long long)__double_as_longlong(b) << 1);
  const double x = abig ? a : -b, y = abig ? -b : a;
  return y - (s - x);
}

// Biased exponent field of a double (0 for zero and subnormals).
__device__ __forceinline__ int dexp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFull);
}

// The filter: +1 or -1 when the rounded determinant decides the sign, 0 when
// it cannot (then orient_resolve gives the exact sign).  Decided when det is
// normal and its exponent is at least max(exponent(t1), exponent(t2)) - 48:
// then |det| >= 2^(e_det - 1023) >= 2^(e_max - 1071) > 2^-50 * 2 max(|t1|, |t2|)
// >= 8 eps (|t1| + |t2|), beyond the rounding error bound.  Only the seven
// FP64 operations of det itself; the test and the sign use integer ALUs.
__device__ __forceinline__ int orient_filter(const VD& p, const VD& q, const VD& r) {
  const double t1 = (q.x - p.x) * (r.y - p.y);
  const double t2 = (q.y - p.y) * (r.x - p.x);
  const double det = t1 - t2;
  const int ed = dexp(det);
  if (ed > 0 && ed + 48 >= max(dexp(t1), dexp(t2))) return __double_as_longlong(det) < 0 ? -1 : 1;
  return 0;
}

// Exact sign where the filter cannot decide: when the four coordinate
// differences are exact (their two-sum errors zero, the usual case for nearly
// or exactly collinear points close together) the exact sign of the
// two-product difference above, else the full sixteen-term sum.
__device__ __forceinline__ int orient_resolve(const VD& p, const VD& q, const VD& r) {
  const double ax = q.x - p.x, by = r.y - p.y, ay = q.y - p.y, bx = r.x - p.x;
  const unsigned long long tails =
      (unsigned long long)(__double_as_longlong(diff_error(q.x, p.x, ax)) |
                           __double_as_longlong(diff_error(r.y, p.y, by)) |
                           __double_as_longlong(diff_error(q.y, p.y, ay)) |
                           __double_as_longlong(diff_error(r.x, p.x, bx)));
  if ((tails << 1) == 0ull) return sign_of_product_difference(ax, by, ay, bx);
  return orient_sign_exact(p.x, p.y, q.x, q.y, r.x, r.y);
}

// Sign of the exact determinant (-1, 0, +1).
__device__ __forceinline__ int orient_sign(const VD& p, const VD& q, const VD& r) {
  const int f = orient_filter(p, q, r);
  return f != 0 ? f : orient_resolve(p, q, r);
}

constexpr double QC = 12.0 * 1.7320508075688772;  // 12 sqrt(3)
// x / 3.0, bit for bit the IEEE quotient (round to nearest), in one multiply
// and two fused multiply-adds instead of the division sequence.  With
// R = RN(1/3), q = RN(x R) lies within one ulp of x/3; the remainder
// r = x - 3q is exact in one fma; RN(q + r R) is then the correctly rounded
// quotient (Markstein's correction theorem: P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990; J.-M. Muller et al., Handbook of Floating-Point
// Arithmetic, ch. 4).  A zero remainder keeps q (so -0 stays -0); a
// non-finite x (r is NaN) keeps q as well (x/3 = x for infinities and NaN).
__device__ __forceinline__ double div3(double x) {
  constexpr double R = 1.0 / 3.0;
  double q = x * R;
  double r = __fma_rn(-3.0, q, x);
  long long rb = __double_as_longlong(r);
  bool keep = ((unsigned long long)rb << 1) == 0ull || ((rb >> 52) & 0x7ff) == 0x7ff;
  return keep ? q : __fma_rn(r, R, q);
}

__device__ __forceinline__ double len_under(double k00, double k01, double k11, const VD& p,
                                            const VD& q) {
  double dx = q.x - p.x;
  double dy = q.y - p.y;
  double L2 = ((k00 * dx) * dx + ((2.0 * k01) * dx) * dy) + (k11 * dy) * dy;
  return sqrt(L2);
}

// Vasilevskii-Lipnikov quality in the element-mean metric, canonical rotation.
__device__ __forceinline__ double quality_c(int i0, int i1, int i2, VD a, VD b, VD c) {
  canon(i0, i1, i2, a, b, c);
  double k00 = div3((a.m00 + b.m00) + c.m00);
  double k01 = div3((a.m01 + b.m01) + c.m01);
  double k11 = div3((a.m11 + b.m11) + c.m11);
  double l0 = len_under(k00, k01, k11, a, b);
  double l1 = len_under(k00, k01, k11, b, c);
  double l2 = len_under(k00, k01, k11, c, a);
  double P = (l0 + l1) + l2;
  double area = 0.5 * orient3(a, b, c);
  double AM = sqrt(k00 * k11 - k01 * k01) * area;
  double xx = div3(P);
  double s = !dgt(xx, 1.0) ? xx : 1.0 / xx;  // xx <= 1
  double f = s * (2.0 - s);
  double F = (f * f) * f;
  return ((QC * AM) / (P * P)) * F;
}

// Reverse-mode derivative of quality_c; g[k][0..4] = dq/d(x,y,m00,m01,m11) of
// the k-th vertex in the caller's order.  Same operation order as the
// definition of the derivative used by the optimisation-based smoother.
__device__ __forceinline__ double quality_grad_c(int i0, int i1, int i2, VD a, VD b, VD c,
                                                 double g[3][5]) {
  int s = 0;
  if (i1 < i0 && i1 < i2) s = 1;
  else if (i2 < i0 && i2 < i1) s = 2;
  canon(i0, i1, i2, a, b, c);
  double k00 = div3((a.m00 + b.m00) + c.m00);
  double k01 = div3((a.m01 + b.m01) + c.m01);
  double k11 = div3((a.m11 + b.m11) + c.m11);
  double dx[3] = {b.x - a.x, c.x - b.x, a.x - c.x};
  double dy[3] = {b.y - a.y, c.y - b.y, a.y - c.y};
  double l[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    double L2 = ((k00 * dx[e]) * dx[e] + ((2.0 * k01) * dx[e]) * dy[e]) + (k11 * dy[e]) * dy[e];
    l[e] = sqrt(L2);
  }
  double P = (l[0] + l[1]) + l[2];
  double area = 0.5 * orient3(a, b, c);
  double sd = sqrt(k00 * k11 - k01 * k01);
  double AM = sd * area;
  double xx = div3(P);
  bool left = (xx <= 1.0);
  double sv = left ? xx : 1.0 / xx;
  double f = sv * (2.0 - sv);
  double F = (f * f) * f;
  double t = (QC * AM) / (P * P);
  double q = t * F;
  double gF = t;
  double gt = F;
  double gAM = (gt * QC) / (P * P);
  double gP = -((2.0 * t) / P) * gt;
  double gf = (3.0 * (f * f)) * gF;
  double gs = (2.0 - 2.0 * sv) * gf;
  double gxx = left ? gs : -(gs / (xx * xx));
  gP = gP + div3(gxx);
  double gsd = area * gAM;
  double garea = sd * gAM;
  double gdet = gsd / (2.0 * sd);
  double gk00 = k11 * gdet;
  double gk11 = k00 * gdet;
  double gk01 = -(2.0 * k01) * gdet;
  double go = 0.5 * garea;
  double gdx[3], gdy[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    double gL2 = gP / (2.0 * l[e]);
    gk00 = gk00 + (dx[e] * dx[e]) * gL2;
    gk01 = gk01 + (2.0 * (dx[e] * dy[e])) * gL2;
    gk11 = gk11 + (dy[e] * dy[e]) * gL2;
    gdx[e] = ((2.0 * k00) * dx[e] + (2.0 * k01) * dy[e]) * gL2;
    gdy[e] = ((2.0 * k01) * dx[e] + (2.0 * k11) * dy[e]) * gL2;
  }
  double cg[3][5];
  cg[0][0] = (go * (b.y - c.y) - gdx[0]) + gdx[2];
  cg[1][0] = (go * (c.y - a.y) + gdx[0]) - gdx[1];
  cg[2][0] = (go * (a.y - b.y) + gdx[1]) - gdx[2];
  cg[0][1] = (go * (c.x - b.x) - gdy[0]) + gdy[2];
  cg[1][1] = (go * (a.x - c.x) + gdy[0]) - gdy[1];
  cg[2][1] = (go * (b.x - a.x) + gdy[1]) - gdy[2];
  double m0 = div3(gk00), m1 = div3(gk01), m2 = div3(gk11);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cg[k][2] = m0;
    cg[k][3] = m1;
    cg[k][4] = m2;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int dst = (s + k) % 3;
#pragma unroll
    for (int j = 0; j < 5; ++j) g[dst][j] = cg[k][j];
  }
  return q;
}

// Hash priority for the independent sets (Sec. 3.2): MurmurHash3 fmix32 of
// (local id xor per-round seed).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint32_t prio(uint32_t v, uint32_t seed, uint32_t r) {
  uint32_t sr = seed + 0x9E3779B9u * r;
  return fmix32(v ^ sr);
}

// Id of the vertex in slot s of the mesh whose region starts at vb.
__device__ __forceinline__ uint32_t vid_of(const Store& S, int s, int vb) {
  return S.lid ? (uint32_t)S.lid[s] : (uint32_t)(s - vb);
}

}  // namespace pm
