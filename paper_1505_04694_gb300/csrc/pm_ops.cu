// The adaptation operators (Sec. 2.4) run in rounds of independent sets
// (Sec. 3.2).  One round of coarsening, swapping or smoothing is:
//
//   evaluate  every dirty vertex decides its operation on the current mesh and
//             joins the candidate list (warp-aggregated atomic append, the
//             worklist scheme of Sec. 3.4);
//   select    candidates that beat every candidate neighbour by hash priority
//             form the independent set S; the others stay dirty;
//   apply     each member of S rewrites only its own ball (disjoint between
//             members) and records which vertices' adjacency changes;
//   commit    the deferred update of Sec. 3.3: after the whole set has been
//             applied, every affected vertex rebuilds its own NN/NE rows from
//             the operations of its S neighbours, so exactly one thread writes
//             each list.
//
// Every kernel walks its list with a grid-stride loop over a count that lives
// in device memory, so a round needs no host round trip until the candidate
// count is read to decide termination.
#include <algorithm>
#include <mutex>
#include <string>

#include "pm_internal.cuh"

namespace pm {

namespace {

// ---- shared device helpers ---------------------------------------------------

struct MeshCtx {
  int mi, vb, eb;
};

__device__ __forceinline__ MeshCtx ctx_of(const Store& S, int slot) {
  MeshCtx c;
  c.mi = mesh_of_vslot(S, slot);
  c.vb = S.tab.vbase[c.mi];
  c.eb = S.tab.ebase[c.mi];
  return c;
}

// Which thread takes list entry i.  Contiguous: consecutive entries to
// consecutive threads of a block (coalesced list reads, for long lists).
// Interleaved (`il`): entry i to block i mod gridDim.x, so that a short list
// spreads over every SM instead of the first few blocks; that matters when
// an entry's work is FP64, whose issue cost per warp is the same for one
// active lane as for 32.
__device__ __forceinline__ int grank(bool il) {
  return il ? threadIdx.x * gridDim.x + blockIdx.x : blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ int gsize() { return gridDim.x * blockDim.x; }

__device__ __forceinline__ const int* nn_row(const Store& S, int slot) {
  return S.NN + (size_t)slot * S.W;
}
__device__ __forceinline__ const int* ne_row(const Store& S, int slot) {
  return S.NE + (size_t)slot * S.W;
}

// Per-mesh operation counter, aggregated over the lanes of a warp that share a
// mesh (all lanes must call).
__device__ __forceinline__ void count_op(const Store& S, bool pred, int mi) {
  unsigned act = __ballot_sync(0xffffffffu, pred);
  if (!act) return;
  unsigned grp = __match_any_sync(0xffffffffu, pred ? mi : -1);
  int lane = threadIdx.x & 31;
  if (pred && (__ffs(grp) - 1) == lane) atomicAdd(S.tab.ops + mi, (unsigned long long)__popc(grp));
}

// Advance the per-mesh round counter of every mesh that formed candidates in
// the round whose set was just selected (run by one block before the apply).
__device__ __forceinline__ void advance_rounds(const Store& S) {
  if (blockIdx.x != 0) return;
  for (int i = threadIdx.x; i < S.nmesh; i += blockDim.x) {
    if (S.tab.had[i]) {
      S.tab.r[i] += 1;
      S.tab.had[i] = 0;
    }
  }
}

__device__ __forceinline__ int count_elems_with(const Store& S, const int* ne, int nel, int eb,
                                                int lw) {
  int c = 0;
  for (int k = 0; k < nel; ++k) {
    int4 e = S.EN[eb + ne[k]];
    if (e.x == lw || e.y == lw || e.z == lw) ++c;
  }
  return c;
}


// Inputs of v's evaluation unchanged since tag `et`?  Evaluations read v's
// rows, the elements and vertices of its ball and the rows and positions of
// its neighbours; every change to those stamps v (touch) or, for a change of
// a neighbour x, every vertex adjacent to x after the change (ntouch).  An
// edge (v, x) that exists now existed at x's last change (adding it would
// have changed x again), so ntouch[v] covers every current neighbour.  Only
// evaluations newer than `lo` count.
__device__ __forceinline__ bool unchanged(const Store& S, int v, int vb, int et, int lo) {
  return et > lo && S.touch[v] <= et && S.ntouch[v] <= et;
}

// Measurement only: adds every lane's count of FP64 operations to *work
// (one atomic per warp).  All 32 lanes must call it.  The counts follow the
// arithmetic as written: a metric length 17 operations, an orientation 8, a
// quality 77, a square root or a division 1.
constexpr unsigned kOpsLen2 = 17, kOpsOrient = 8, kOpsQuality = 77;

// Warps per block that own a per-warp shared-memory queue or array in the
// scan phases (blocks hold at most 256 threads).
constexpr int kScanWarps = 8;

__device__ __forceinline__ void add_work(unsigned long long* work, unsigned ops) {
  if (!work) return;
  unsigned tot = __reduce_add_sync(0xffffffffu, ops);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(work, (unsigned long long)tot);
}

// qK of every listed element slot, one element per thread.
__device__ __forceinline__ void elem_quality_phase(const Store& S, const int* list, const int* np,
                                                   unsigned long long* work, bool il = false) {
  const int n = *np;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    unsigned ops = 0;
    if (i < n) {
      int slot = list[i];
      int vb = S.tab.vbase[mesh_of_eslot(S, slot)];
      int4 e = S.EN[slot];
      S.qK[slot] = quality_c(e.x, e.y, e.z, load_vd(S, vb + e.x), load_vd(S, vb + e.y),
                             load_vd(S, vb + e.z));
      ops = kOpsQuality;
    }
    add_work(work, ops);
  }
}

// Stamps the neighbours in `row` (local ids) after a change of their vertex.
__device__ __forceinline__ void stamp_neighbours(const Store& S, const int* row, int len, int vb,
                                                 int stamp) {
#pragma unroll 4
  for (int k = 0; k < len; ++k) S.ntouch[vb + row[k]] = stamp;
}

// ---- worklist initialisation ---------------------------------------------------

// mode 0: every live vertex of an active mesh; mode 1: live interior vertices.
// With `ev`, vertices whose last evaluation (newer than `lo`) found nothing
// and whose inputs are unchanged since are left out: they would find
// nothing again.
__global__ void k_init_list(Store S, int mode, int* list, int* count, const int* ev, int lo) {
  for (int i0 = blockIdx.x * blockDim.x; i0 < S.vused; i0 += gridDim.x * blockDim.x) {
    int s = i0 + threadIdx.x;
    bool take = false;
    if (s < S.vused) {
      int mi = mesh_of_vslot(S, s);
      int vb = S.tab.vbase[mi];
      if (s - vb < S.tab.nv[mi] && S.tab.active[mi]) {
        uint8_t f = S.vflag[s];
        take = (f & VF_ALIVE) && (mode == 0 || !(f & VF_BND));
        if (take && ev) take = !unchanged(S, s, vb, ev[s], lo);
      }
    }
    warp_append(take, s, list, count);
  }
}

// ---- independent set (Sec. 3.2) -------------------------------------------------
// v joins S when prio(v) exceeds the priority of every neighbour that is a
// candidate of the same round.  Losers go to `keep` (still dirty / pending).
__global__ void k_select(Store S, const int* C, const int* nCp, const int* cmark, int* smark,
                         int tag, int* Sl, int* nS, int* keep, int* nkeep, int* kmark) {
  const int n = *nCp;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    int i = i0 + threadIdx.x;
    bool win = false, lose = false;
    int v = 0;
    if (i < n) {
      v = C[i];
      MeshCtx c = ctx_of(S, v);
      uint32_t seed = S.tab.seed[c.mi], r = S.tab.r[c.mi];
      uint32_t pv = prio(vid_of(S, v, c.vb), seed, r);
      const int* nn = nn_row(S, v);
      int nnl = S.NNlen[v];
      win = true;
#pragma unroll 4
      for (int k = 0; k < nnl; ++k) {
        int u = c.vb + nn[k];
        int cu = cmark[u];
        uint32_t iu = vid_of(S, u, c.vb);
        win &= !(cu == tag && prio(iu, seed, r) > pv);
      }
      if (win) smark[v] = tag;
      else if (keep) lose = stamp_first(kmark, v, tag);
    }
    warp_append(win, v, Sl, nS);
    if (keep) warp_append(lose, v, keep, nkeep);
  }
}

// Whether candidate v is a local maximum of the priority among this round's
// candidates (cmark == tag) in its neighbourhood.
__device__ __forceinline__ bool local_max(const Store& S, int v, const int* cmark, int tag) {
  MeshCtx c = ctx_of(S, v);
  uint32_t seed = S.tab.seed[c.mi], r = S.tab.r[c.mi];
  // colour-class sets: only the candidates of colour r mod ncol compete
  const bool by_colour = S.tab.select[c.mi] == PM_SELECT_COLOUR;
  const int cls = by_colour ? (int)(r % (uint32_t)S.tab.ncol[c.mi]) : 0;
  if (by_colour && S.tab.col[v] != cls) return false;
  uint32_t pv = prio(vid_of(S, v, c.vb), seed, r);
  const int* nn = nn_row(S, v);
  int nnl = S.NNlen[v];
  bool win = true;
#pragma unroll 4
  for (int k = 0; k < nnl; ++k) {
    int u = c.vb + nn[k];
    int cu = cmark[u];
    uint32_t iu = vid_of(S, u, c.vb);
    win &= !(cu == tag && (!by_colour || S.tab.col[u] == cls) && prio(iu, seed, r) > pv);
  }
  return win;
}

// ---- colouring of the vertex graph (Sec. 3.2, colour-class sets) --------------
// Speculative rounds on a snapshot, the same as the oracle's: every uncoloured
// live vertex of a mesh in colour mode proposes the smallest colour no
// coloured neighbour holds; of two uncoloured neighbours proposing the same
// colour the one of lower priority (prio with the mesh's round counter at the
// start of the pass) withdraws; the others keep their proposals.  The
// proposals of a round are stamped with the round, so the resolve pass reads
// only stamps and proposals while it writes colours.
__global__ void k_colour_init(Store S, int* U, int* nU) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nmesh; i += gridDim.x * blockDim.x)
    S.tab.ncol[i] = 1;
  for (int i0 = blockIdx.x * blockDim.x; i0 < S.vused; i0 += gridDim.x * blockDim.x) {
    const int s = i0 + threadIdx.x;
    bool take = false;
    if (s < S.vused) {
      S.tab.col[s] = -1;
      const int mi = mesh_of_vslot(S, s);
      take = s - S.tab.vbase[mi] < S.tab.nv[mi] && S.tab.active[mi] &&
             S.tab.select[mi] == PM_SELECT_COLOUR && (S.vflag[s] & VF_ALIVE);
    }
    warp_append(take, s, U, nU);
  }
}

__global__ void k_colour_propose(Store S, const int* U, const int* nUp, int* prop, int* stamp,
                                 int rt) {
  const int n = *nUp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int v = U[i];
    const int vb = S.tab.vbase[mesh_of_vslot(S, v)];
    const int* nn = nn_row(S, v);
    const int nnl = S.NNlen[v];
    RowMask used;  // colours 0..127 held by coloured neighbours
#pragma unroll 4
    for (int k = 0; k < nnl; ++k) {
      const int c = S.tab.col[vb + nn[k]];
      if (c >= 0 && c < MAXW) used.set(c);
    }
    int c = 0;
    if (~used.lo) c = __ffsll((long long)~used.lo) - 1;
    else if (~used.hi) c = 64 + __ffsll((long long)~used.hi) - 1;
    else c = MAXW;  // a vertex of degree MAXW whose neighbours hold 0..MAXW-1
    prop[v] = c;
    stamp[v] = rt;
  }
}

__global__ void k_colour_resolve(Store S, const int* U, const int* nUp, const int* prop,
                                 const int* stamp, int rt, int* Un, int* nUn) {
  const int n = *nUp;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    bool again = false;
    int v = 0;
    if (i < n) {
      v = U[i];
      const int mi = mesh_of_vslot(S, v);
      const int vb = S.tab.vbase[mi];
      const uint32_t seed = S.tab.seed[mi], r = S.tab.r[mi];
      const uint32_t pv = prio(vid_of(S, v, vb), seed, r);
      const int pc = prop[v];
      const int* nn = nn_row(S, v);
      const int nnl = S.NNlen[v];
      bool keep = true;
#pragma unroll 4
      for (int k = 0; k < nnl; ++k) {
        const int u = vb + nn[k];
        keep &= !(stamp[u] == rt && prop[u] == pc && prio(vid_of(S, u, vb), seed, r) > pv);
      }
      if (keep) {
        S.tab.col[v] = pc;
        atomicMax(S.tab.ncol + mi, pc + 1);
      }
      again = !keep;
    }
    warp_append(again, v, Un, nUn);
  }
}


// End of a fused select-and-apply launch: the last block to finish advances
// the round counter of every mesh that formed candidates (every block has
// read the counters by then) and re-arms the block counter.
__device__ __forceinline__ void round_done(const Store& S, unsigned* done) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i < S.nmesh; i += blockDim.x) {
    if (S.tab.had[i]) {
      S.tab.r[i] += 1;
      S.tab.had[i] = 0;
    }
  }
  if (threadIdx.x == 0) *done = 0;
}

// ---- tile-parallel evaluation: 8 lanes per vertex, one ball element each ----
// Sums keep the ascending order of the definition (every lane accumulates the
// lanes' terms in order through shuffles); minima and all-of votes do not
// depend on order.  All lanes of a tile end with the same result.

constexpr int TW = 8;

struct Tile {
  int tl;          // lane within the tile
  unsigned mask;   // the tile's lanes in the warp
  int shift;       // bit offset of the tile in a warp ballot
};

__device__ __forceinline__ Tile tile_of() {
  int lane = threadIdx.x & 31;
  Tile t;
  t.tl = lane & (TW - 1);
  t.shift = lane & ~(TW - 1);
  t.mask = 0xFFu << t.shift;
  return t;
}

__device__ __forceinline__ double tshfl(const Tile& t, double x, int src) {
  return __shfl_sync(t.mask, x, src, TW);
}

__device__ __forceinline__ double tmin(const Tile& t, double x) {
#pragma unroll
  for (int o = TW / 2; o > 0; o >>= 1) {
    double y = __shfl_xor_sync(t.mask, x, o, TW);
    x = dlt(y, x) ? y : x;
  }
  return x;
}

__device__ __forceinline__ bool tall(const Tile& t, bool p) {
  return ((__ballot_sync(t.mask, !p) >> t.shift) & 0xFFu) == 0u;
}

__device__ __forceinline__ int tsum(const Tile& t, int x) {
  return __reduce_add_sync(t.mask, x);
}

// Position of tile `tid` and the number of tiles of the grid.  Interleaved
// (`il`): tile i to block i mod gridDim.x (see grank).
__device__ __forceinline__ int trank(bool il) {
  const int tpb = blockDim.x / TW, tib = threadIdx.x / TW;
  return il ? tib * gridDim.x + blockIdx.x : blockIdx.x * tpb + tib;
}
__device__ __forceinline__ int tcount() { return gridDim.x * (blockDim.x / TW); }

// ---- coarsening (Sec. 2.4.1) ---------------------------------------------------

struct CoarsenCtx;
__device__ __forceinline__ double S_L_up(const CoarsenCtx& x);

struct CoarsenCtx {
  const Store* S;
  MeshCtx c;
  int v, lv;
  const int* nn;
  int nnl;
  const int* ne;
  int nel;
  VD dv;
  bool bnd;
};

__device__ __forceinline__ double S_L_up(const CoarsenCtx& x) { return x.S->tab.L_up[x.c.mi]; }

// The integer part of the validity of collapsing v onto local neighbour u:
// the link condition (|NN(v) & NN(u)| = 2 for an interior edge, 1 for a
// boundary edge; a boundary vertex only along a boundary edge).
__device__ bool collapse_link(const Store& S, const CoarsenCtx& x, int u) {
  const bool bedge = count_elems_with(S, x.ne, x.nel, x.c.eb, u) == 1;
  if (x.bnd && !bedge) return false;
  const int ws = x.c.vb + u;
  const int* nnw = nn_row(S, ws);
  const int nnwl = S.NNlen[ws];
  int common = 0, a = 0, b = 0;
  while (a < x.nnl && b < nnwl) {
    const int p = x.nn[a], q = nnw[b];
    if (p == q) {
      ++common;
      ++a;
      ++b;
    } else if (p < q) {
      ++a;
    } else {
      ++b;
    }
  }
  return common == (bedge ? 1 : 2);
}

// collapse_valid with the lanes of a tile splitting v's ball elements (the
// element count of the edge and the orientations with v on u) and v's
// neighbours (the link condition and the new edge lengths): the same
// conjunction of the same tests.  Every lane returns the tile's answer.
__device__ bool tile_collapse_valid(const Tile& t, const CoarsenCtx& x, int u, double4 band,
                                    unsigned& ops) {
  const double L_up = S_L_up(x);
  const Store& S = *x.S;
  int cnt = 0;
  for (int k = t.tl; k < x.nel; k += TW) {
    int4 e = S.EN[x.c.eb + x.ne[k]];
    cnt += (e.x == u || e.y == u || e.z == u) ? 1 : 0;
  }
  const bool bedge = tsum(t, cnt) == 1;
  if (x.bnd && !bedge) return false;
  const int ws = x.c.vb + u;
  const int* nnw = nn_row(S, ws);
  const int nnwl = S.NNlen[ws];
  int common = 0;
  for (int k = t.tl; k < x.nnl; k += TW) common += row_has(nnw, nnwl, x.nn[k]) ? 1 : 0;
  if (tsum(t, common) != (bedge ? 1 : 2)) return false;
  const VD dw = load_vd(S, ws);
  bool ok = true;
  for (int k = t.tl; k < x.nel; k += TW) {
    int4 e = S.EN[x.c.eb + x.ne[k]];
    if (e.x == u || e.y == u || e.z == u) continue;
    VD d0 = (e.x == x.lv) ? dw : load_vd(S, x.c.vb + e.x);
    VD d1 = (e.y == x.lv) ? dw : load_vd(S, x.c.vb + e.y);
    VD d2 = (e.z == x.lv) ? dw : load_vd(S, x.c.vb + e.z);
    ok &= orient_sign(d0, d1, d2) > 0;
    ops += kOpsOrient;
  }
  if (!tall(t, ok)) return false;
  for (int k = t.tl; k < x.nnl; k += TW) {
    int y = x.nn[k];
    if (y == u || row_has(nnw, nnwl, y)) continue;
    ok &= !len_gt(metric_len2(dw, load_vd(S, x.c.vb + y)), band.z, band.w, L_up);
    ops += kOpsLen2;
  }
  return tall(t, ok);
}

// Collapse candidates of v: neighbours with metric length below L_low (a
// boundary vertex: only along boundary edges), sorted by (length, id) into
// out[0..n); corners and dead vertices have none.  The lanes of a tile split
// v's neighbours: lane tl holds neighbours tl, tl + 8, ...; each candidate's
// place in the order is the number of candidates before it (a neighbour of
// lower index has the lower id: rows are sorted), which is the stable order
// by length the definition asks for.  Returns the candidate count (every
// lane).
__device__ int tile_coarsen_candidates(const Tile& t, const Store& S, int v, MeshCtx c, int* out,
                                       unsigned& ops) {
  uint8_t f = S.vflag[v];
  if (!(f & VF_ALIVE) || (f & VF_CORNER)) return 0;
  const bool bnd = (f & VF_BND) != 0;
  const int* nn = nn_row(S, v);
  const int nnl = S.NNlen[v];
  const int* ne = ne_row(S, v);
  const int nel = S.NElen[v];
  const VD dv = load_vd(S, v);
  const double L_low = S.tab.L_low[c.mi];
  const double4 band = S.tab.band[c.mi];
  constexpr int kPer = MAXW / TW;
  double L[kPer];
  bool is[kPer];
  int mine = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = j * TW + t.tl;
    is[j] = false;
    L[j] = 0.0;
    if (k < nnl) {
      const int u = nn[k];
      const double L2 = metric_len2(dv, load_vd(S, c.vb + u));
      ops += kOpsLen2;
      bool cand = len_lt(L2, band.x, band.y, L_low);
      if (cand && bnd) cand = count_elems_with(S, ne, nel, c.eb, u) == 1;
      if (cand) {
        L[j] = sqrt(L2);
        ++ops;
        is[j] = true;
        ++mine;
      }
    }
  }
  const int steps = (nnl + TW - 1) / TW;
  for (int j = 0; j < steps; ++j) {
    int rank = 0;
    for (int j2 = 0; j2 < steps; ++j2) {
#pragma unroll
      for (int src = 0; src < TW; ++src) {
        const double Lo = tshfl(t, L[j2], src);
        const bool co = __shfl_sync(t.mask, is[j2] ? 1 : 0, src, TW) != 0;
        const int ko = j2 * TW + src, k = j * TW + t.tl;
        if (co && (dlt(Lo, L[j]) || (dbits(Lo) == dbits(L[j]) && ko < k))) ++rank;
      }
    }
    if (is[j]) out[rank] = nn[j * TW + t.tl];
  }
  return tsum(t, mine);
}

__device__ __forceinline__ CoarsenCtx coarsen_ctx(const Store& S, int v, MeshCtx c) {
  CoarsenCtx x;
  x.S = &S;
  x.c = c;
  x.v = v;
  x.lv = v - c.vb;
  x.nn = nn_row(S, v);
  x.nnl = S.NNlen[v];
  x.ne = ne_row(S, v);
  x.nel = S.NElen[v];
  x.dv = load_vd(S, v);
  x.bnd = (S.vflag[v] & VF_BND) != 0;
  return x;
}

// Collapse evaluation.  The target of v is the first candidate, by (metric
// length, id), whose collapse is valid.  Pass 1 (per dirty vertex) reuses an
// unchanged earlier result or lists v's sorted candidates; a dense pass then
// checks every listed vertex's best candidate (one work item each), and a
// last pass goes through the remaining candidates of the vertices whose best
// one failed.  Candidates are listed by an 8-lane tile per vertex (see
// tile_coarsen_candidates), so the FP64 lengths of the neighbours run side
// by side.  The tile takes the stamp decision from lane 0 before lane 0
// overwrites the stamp.
// Pass 1 of the large rounds, one dirty vertex per thread: reuse an unchanged
// earlier result, or list v's collapse candidates.  The metric lengths of all
// the warp's vertices' edges are the FP64 work; they are evaluated 32 at a
// time from a per-warp queue (full warps on the FP64 pipe, where a tile per
// vertex kept about 19 of 32 lanes busy), each candidate's length stored in
// a scratch row and its bit in a per-lane mask; then each thread places its
// own candidates by rank in the (length, id) order, as tile_coarsen_candidates
// does in the persistent rounds.
__device__ __forceinline__ void coarsen_len_chunk(const Store& S, const int2* q, int cnt, int v,
                                                  MeshCtx c, unsigned long long (*cm)[2],
                                                  double* Lbuf) {
  const int lane = threadIdx.x & 31;
  const int2 r = lane < cnt ? q[lane] : make_int2(lane, 0);
  const int ov = __shfl_sync(0xffffffffu, v, r.x);
  const int ovb = __shfl_sync(0xffffffffu, c.vb, r.x);
  const int oeb = __shfl_sync(0xffffffffu, c.eb, r.x);
  const int omi = __shfl_sync(0xffffffffu, c.mi, r.x);
  if (lane < cnt) {
    const int u = nn_row(S, ov)[r.y];
    const double L2 = metric_len2(load_vd(S, ov), load_vd(S, ovb + u));
    const double4 band = S.tab.band[omi];
    bool is = len_lt(L2, band.x, band.y, S.tab.L_low[omi]);
    // a boundary vertex collapses only along a boundary edge
    if (is && (S.vflag[ov] & VF_BND)) is = count_elems_with(S, ne_row(S, ov), S.NElen[ov], oeb, u) == 1;
    if (is) {
      Lbuf[(size_t)ov * S.W + r.y] = sqrt(L2);
      atomicOr(&cm[r.x][r.y >> 6], 1ull << (r.y & 63));
    }
  }
}

__device__ __forceinline__ void coarsen_scan_phase(Store S, const int* D, const int* nDp,
                                                   int* target, int* cand, int* ncand, int* C,
                                                   int* nC, int* cmark, int tag, int pass0,
                                                   int2* W0, int* nW0, double* Lbuf) {
  __shared__ int2 sq[kScanWarps][64];
  __shared__ unsigned long long scm[kScanWarps][32][2];
  const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) % kScanWarps;
  const unsigned lt = (1u << lane) - 1u;
  const int n = *nDp;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    int v = 0, nnl = 0;
    bool reuse_cand = false, eval = false;
    MeshCtx c{0, 0, 0};
    if (i < n) {
      v = D[i];
      c = ctx_of(S, v);
      if (unchanged(S, v, c.vb, S.evc[v], pass0)) {
        reuse_cand = target[v] >= 0;
        if (reuse_cand) {
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        }
      } else {
        S.evc[v] = tag;
        eval = true;
        const uint8_t f = S.vflag[v];
        // corners and dead vertices have no candidates
        if ((f & VF_ALIVE) && !(f & VF_CORNER)) nnl = S.NNlen[v];
      }
    }
    scm[wq][lane][0] = scm[wq][lane][1] = 0ull;
    __syncwarp();
    const int tmax = __reduce_max_sync(0xffffffffu, nnl);
    int qn = 0;  // the same in every lane
    for (int t = 0; t < tmax; ++t) {
      const bool p = t < nnl;
      const unsigned m = __ballot_sync(0xffffffffu, p);
      if (p) sq[wq][qn + __popc(m & lt)] = make_int2(lane, t);
      qn += __popc(m);
      __syncwarp();
      if (qn >= 32) {
        coarsen_len_chunk(S, sq[wq], 32, v, c, scm[wq], Lbuf);
        __syncwarp();
        if (lane < qn - 32) sq[wq][lane] = sq[wq][32 + lane];
        qn -= 32;
        __syncwarp();
      }
    }
    if (qn > 0) coarsen_len_chunk(S, sq[wq], qn, v, c, scm[wq], Lbuf);
    __syncwarp();
    int nc = 0;
    if (eval) {
      RowMask cm;
      cm.lo = scm[wq][lane][0];
      cm.hi = scm[wq][lane][1];
      nc = cm.count();
      const int* nn = nn_row(S, v);
      const double* L = Lbuf + (size_t)v * S.W;
      int* out = cand + (size_t)v * S.W;
      RowMask a = cm;
      while (a.any()) {
        const int k = a.pop();
        const double Lk = L[k];
        int rank = 0;
        RowMask b = cm;
        while (b.any()) {
          const int k2 = b.pop();
          const double Lo = L[k2];
          if (dlt(Lo, Lk) || (dbits(Lo) == dbits(Lk) && k2 < k)) ++rank;
        }
        out[rank] = nn[k];
      }
      ncand[v] = nc;
      if (nc == 0) target[v] = -1;
    }
    warp_append(reuse_cand, v, C, nC);
    warp_append_t(eval && nc > 0, make_int2(v, 0), W0, nW0);
  }
}

__global__ void k_coarsen_scan(Store S, const int* D, const int* nDp, int* target, int* cand,
                               int* ncand, int* C, int* nC, int* cmark, int tag, int pass0,
                               int2* W0, int* nW0, double* Lbuf) {
  coarsen_scan_phase(S, D, nDp, target, cand, ncand, C, nC, cmark, tag, pass0, W0, nW0, Lbuf);
}

// The check passes, one work item (v, k) per thread: is collapsing v onto
// its k-th candidate valid (in the last pass: the first valid one from k on)?
// Validity is the conjunction of the link condition and, for the collapse
// with v on u, every remaining ball element counter-clockwise and no new edge
// longer than L_up (collapse_valid below, tile form).  Balls differ in size
// and most tests need no arithmetic (elements containing u, neighbours
// shared with u), so the FP64 tests of a warp's items are queued in shared
// memory per warp, orientations and lengths apart, and evaluated 32 at a
// time: full warps on the FP64 pipe instead of the lanes whose own loop is
// still running.  Any failed test clears the owner's flag; the conjunction
// does not depend on the order of its tests.
constexpr int kCheckWarps = 8;

struct CheckQueues {
  int4* qo;  // orientations: (owner lane, element's local vertex ids)
  int2* ql;  // lengths: (owner lane, neighbour's local id)
  int* ok;   // per lane of the warp: its item's conjunction so far
};

// Evaluate the first `cnt` (<= 32) queued orientations; all lanes call.
__device__ __forceinline__ void check_orient_chunk(const Store& S, const CheckQueues& Q, int cnt,
                                                   int vb, int lv, int ws, unsigned& ops) {
  const int lane = threadIdx.x & 31;
  const int4 r = lane < cnt ? Q.qo[lane] : make_int4(lane, 0, 0, 0);
  const int o_vb = __shfl_sync(0xffffffffu, vb, r.x);
  const int o_lv = __shfl_sync(0xffffffffu, lv, r.x);
  const int o_ws = __shfl_sync(0xffffffffu, ws, r.x);
  if (lane < cnt) {
    const VD dw = load_vd(S, o_ws);
    const VD d0 = (r.y == o_lv) ? dw : load_vd(S, o_vb + r.y);
    const VD d1 = (r.z == o_lv) ? dw : load_vd(S, o_vb + r.z);
    const VD d2 = (r.w == o_lv) ? dw : load_vd(S, o_vb + r.w);
    if (orient_sign(d0, d1, d2) <= 0) Q.ok[r.x] = 0;
    ops += kOpsOrient;
  }
}

// Evaluate the first `cnt` (<= 32) queued new-edge lengths; all lanes call.
__device__ __forceinline__ void check_len_chunk(const Store& S, const CheckQueues& Q, int cnt,
                                                int vb, int ws, int mi, unsigned& ops) {
  const int lane = threadIdx.x & 31;
  const int2 r = lane < cnt ? Q.ql[lane] : make_int2(lane, 0);
  const int o_vb = __shfl_sync(0xffffffffu, vb, r.x);
  const int o_ws = __shfl_sync(0xffffffffu, ws, r.x);
  const int o_mi = __shfl_sync(0xffffffffu, mi, r.x);
  if (lane < cnt) {
    const double4 band = S.tab.band[o_mi];
    const double L_up = S.tab.L_up[o_mi];
    if (len_gt(metric_len2(load_vd(S, o_ws), load_vd(S, o_vb + r.y)), band.z, band.w, L_up))
      Q.ok[r.x] = 0;
    ops += kOpsLen2;
  }
}

__device__ __forceinline__ void coarsen_check_phase(Store S, const int2* Win, const int* nWin,
                                                    int2* Wout, int* nWout, int* target,
                                                    const int* cand, const int* ncand, int* C,
                                                    int* nC, int* cmark, int tag, int last,
                                                    unsigned long long* work) {
  __shared__ int4 sqo[kCheckWarps][64];
  __shared__ int2 sql[kCheckWarps][64];
  __shared__ int sok[kCheckWarps][32];
  const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) % kCheckWarps;
  CheckQueues Q{sqo[wq], sql[wq], sok[wq]};
  const unsigned lt = (1u << lane) - 1u;
  unsigned ops = 0;
  const int n = *nWin;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    int v = 0, k = 0, nc = 0;
    bool found = false, done = i >= n;
    CoarsenCtx x{};
    const int* cv = nullptr;
    if (!done) {
      const int2 it = Win[i];
      v = it.x;
      k = it.y;
      x = coarsen_ctx(S, v, ctx_of(S, v));
      cv = cand + (size_t)v * S.W;
      nc = ncand[v];
    }
    // one candidate per lane and turn; the last pass moves on to the next
    // candidate of each lane whose candidate failed
    while (__ballot_sync(0xffffffffu, !done)) {
      const int u = done ? 0 : cv[k];
      const bool link = !done && collapse_link(S, x, u);
      const int ws = x.c.vb + u;
      const int* nnw = link ? nn_row(S, ws) : nullptr;
      const int nnwl = link ? S.NNlen[ws] : 0;
      Q.ok[lane] = link ? 1 : 0;
      const int T = link ? x.nel + x.nnl : 0;
      const int Tmax = __reduce_max_sync(0xffffffffu, T);
      int no = 0, nl = 0;  // queue lengths, the same in every lane
      __syncwarp();
      for (int t = 0; t < Tmax; ++t) {
        bool po = false, pl = false;
        int4 ro = make_int4(lane, 0, 0, 0);
        int2 rl = make_int2(lane, 0);
        if (t < T) {
          if (t < x.nel) {
            const int4 e = S.EN[x.c.eb + x.ne[t]];
            po = e.x != u && e.y != u && e.z != u;
            ro = make_int4(lane, e.x, e.y, e.z);
          } else {
            const int y = x.nn[t - x.nel];
            pl = y != u && !row_has(nnw, nnwl, y);
            rl = make_int2(lane, y);
          }
        }
        const unsigned mo = __ballot_sync(0xffffffffu, po);
        const unsigned ml = __ballot_sync(0xffffffffu, pl);
        if (po) Q.qo[no + __popc(mo & lt)] = ro;
        if (pl) Q.ql[nl + __popc(ml & lt)] = rl;
        no += __popc(mo);
        nl += __popc(ml);
        __syncwarp();
        if (no >= 32) {
          check_orient_chunk(S, Q, 32, x.c.vb, x.lv, ws, ops);
          __syncwarp();
          if (lane < no - 32) Q.qo[lane] = Q.qo[32 + lane];
          no -= 32;
          __syncwarp();
        }
        if (nl >= 32) {
          check_len_chunk(S, Q, 32, x.c.vb, ws, x.c.mi, ops);
          __syncwarp();
          if (lane < nl - 32) Q.ql[lane] = Q.ql[32 + lane];
          nl -= 32;
          __syncwarp();
        }
      }
      if (no > 0) check_orient_chunk(S, Q, no, x.c.vb, x.lv, ws, ops);
      if (nl > 0) check_len_chunk(S, Q, nl, x.c.vb, ws, x.c.mi, ops);
      __syncwarp();
      if (!done) {
        found = Q.ok[lane] != 0;
        if (found || !last || k + 1 >= nc) done = true;
        else ++k;
      }
      __syncwarp();
    }
    bool next = false;
    if (i < n) {
      if (found) {
        target[v] = cv[k];
        cmark[v] = tag;
        S.tab.had[x.c.mi] = 1;
      } else if (!last && k + 1 < nc) {
        next = true;
      } else {
        target[v] = -1;
      }
    }
    warp_append(found, v, C, nC);
    if (!last) warp_append_t(next, make_int2(v, k + 1), Wout, nWout);
  }
  add_work(work, ops);
}

__global__ void k_coarsen_check(Store S, const int2* Win, const int* nWin, int2* Wout, int* nWout,
                                int* target, const int* cand, const int* ncand, int* C, int* nC,
                                int* cmark, int tag, int last, unsigned long long* work) {
  coarsen_check_phase(S, Win, nWin, Wout, nWout, target, cand, ncand, C, nC, cmark, tag, last,
                      work);
}

// One tile per listed vertex, listing and checking at once (persistent
// rounds): reuse or re-evaluate, then the candidates in order until one is a
// valid collapse.  Same results as coarsen_scan_phase and the two check passes.
__device__ __forceinline__ void coarsen_eval_phase(Store S, const int* D, const int* nDp,
                                                   int* target, int* cand, int* ncand, int* C,
                                                   int* nC, int* cmark, int tag, int pass0,
                                                   unsigned long long* work, bool il = false) {
  const Tile t = tile_of();
  const int n = *nDp;
  unsigned ops = 0;
  for (int i0 = 0; i0 < n; i0 += tcount()) {
    const int i = i0 + trank(il);
    int v = 0;
    bool found = false;
    if (i < n) {
      v = D[i];
      MeshCtx c = ctx_of(S, v);
      const int et = __shfl_sync(t.mask, S.evc[v], 0, TW);
      if (unchanged(S, v, c.vb, et, pass0)) {
        found = target[v] >= 0;
      } else {
        if (t.tl == 0) S.evc[v] = tag;
        int* cv = cand + (size_t)v * S.W;
        int nc = tile_coarsen_candidates(t, S, v, c, cv, ops);
        if (t.tl == 0) ncand[v] = nc;
        __syncwarp(t.mask);  // the candidates written by every lane
        if (nc > 0) {
          CoarsenCtx x = coarsen_ctx(S, v, c);
          const double4 band = S.tab.band[c.mi];
          for (int k = 0; k < nc && !found; ++k)
            if (tile_collapse_valid(t, x, cv[k], band, ops)) {
              found = true;
              if (t.tl == 0) target[v] = cv[k];
            }
        }
        if (!found && t.tl == 0) target[v] = -1;
      }
      if (found && t.tl == 0) {
        cmark[v] = tag;
        S.tab.had[c.mi] = 1;
      }
    }
    warp_append(found && t.tl == 0, v, C, nC);
  }
  add_work(work, ops);
}

// Apply the collapses of S: elements containing edge (v, w) die, the other
// ball elements take w in v's place (slot and orientation kept), v dies.
// Neighbours of v are affected (rows change) and dirty for the next round.
// The qualities of the elements that change are not computed here: their
// slots join list Q and a dense pass computes them (one element per thread
// instead of a serial chain of qualities per collapse).
__device__ __forceinline__ void coarsen_apply_one(const Store& S, bool ok, int v,
                                                  const int* target, int* A, int* nA,
                                                  int* amark, int* Dn, int* nDn, int* dmark,
                                                  int tag, int* Q, int* nQ) {
  {
    int nnl = 0, mi = 0, vb = 0, eb = 0;
    const int* nn = nullptr;
    const int* ne_v = nullptr;
    RowMask qbits;
    if (ok) {
      MeshCtx c = ctx_of(S, v);
      mi = c.mi;
      vb = c.vb;
      int lv = v - c.vb;
      int w = target[v];
      const int* ne = ne_row(S, v);
      int nel = S.NElen[v];
      for (int k = 0; k < nel; ++k) {
        int4* pe = S.EN + c.eb + ne[k];
        int4 e = *pe;
        if (e.x == w || e.y == w || e.z == w) {
          e.w = 0;
        } else {
          if (e.x == lv) e.x = w;
          if (e.y == lv) e.y = w;
          if (e.z == lv) e.z = w;
          qbits.set(k);
        }
        *pe = e;
      }
      S.vflag[v] = (uint8_t)(S.vflag[v] & ~VF_ALIVE);
      nn = nn_row(S, v);
      nnl = S.NNlen[v];
      ne_v = ne;
      eb = c.eb;
    }
    count_op(S, ok, mi);
    int pq = warp_reserve(qbits.count(), nQ);
    while (qbits.any()) Q[pq++] = eb + ne_v[qbits.pop()];
    RowMask fa, fd;
#pragma unroll 4
    for (int k = 0; k < nnl; ++k) {
      int s = vb + nn[k];
      if (stamp_first(amark, s, tag)) fa.set(k);
      if (stamp_first(dmark, s, tag)) fd.set(k);
    }
    int pa = warp_reserve(fa.count(), nA);
    int pd = warp_reserve(fd.count(), nDn);
    write_row_bits(fa, nn, vb, A, pa);
    write_row_bits(fd, nn, vb, Dn, pd);
  }
}

// One round's independent set and its collapses: a winner applies its
// collapse at once (no other vertex of the round reads what a collapse
// writes); losers stay dirty for the next round.
__device__ __forceinline__ void coarsen_select_apply_phase(Store S, const int* C, const int* nCp,
                                                           const int* cmark, int* smark, int tag,
                                                           const int* target, int* A, int* nA,
                                                           int* amark, int* Dn, int* nDn,
                                                           int* dmark,
                                                           int* Q, int* nQ,
                                                           bool il = false) {
  const int n = *nCp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    bool win = false, lose = false;
    int v = 0;
    if (i < n) {
      v = C[i];
      win = local_max(S, v, cmark, tag);
      if (win) smark[v] = tag;
      else lose = stamp_first(dmark, v, tag);
    }
    warp_append(lose, v, Dn, nDn);
    coarsen_apply_one(S, win, v, target, A, nA, amark, Dn, nDn, dmark, tag, Q, nQ);
  }
}

__global__ void k_coarsen_select_apply(Store S, const int* C, const int* nCp, const int* cmark,
                                       int* smark, int tag, const int* target, int* A, int* nA,
                                       int* amark, int* Dn, int* nDn, int* dmark, int* Q, int* nQ,
                                       unsigned* done) {
  coarsen_select_apply_phase(S, C, nCp, cmark, smark, tag, target, A, nA, amark, Dn, nDn, dmark,
                             Q, nQ);
  round_done(S, done);
}

// Deferred-update commit of a coarsening round for affected vertex u:
//   NN(u) <- (NN(u) minus collapsed neighbours) + their targets, and when u is
//            the target of x: + NN(x) minus u;
//   NE(u) <- live elements of NE(u) + (when u is the target of x) NE(x).
__device__ __forceinline__ void coarsen_commit_phase(Store S, const int* A, const int* nAp,
                                                     const int* target, const int* smark, int tag,
                                                     DevStatus* st, bool il = false) {
  const int n = *nAp;
  for (int i = grank(il); i < n; i += gsize()) {
    int u = A[i];
    S.touch[u] = tag + 1;
    MeshCtx c = ctx_of(S, u);
    int lu = u - c.vb;
    const int* nn = nn_row(S, u);
    const int* ne = ne_row(S, u);
    int nnl = S.NNlen[u], nel = S.NElen[u];
    int nb[MAXW], eb[MAXW];
    int nn2 = 0, ne2 = 0;
    bool ok = true;
    // gather the per-entry facts first so that their loads overlap
    RowMask alive, sel;
#pragma unroll 4
    for (int k = 0; k < nel; ++k)
      if (S.EN[c.eb + ne[k]].w) alive.set(k);
#pragma unroll 4
    for (int k = 0; k < nnl; ++k)
      if (smark[c.vb + nn[k]] == tag) sel.set(k);
    for (int k = 0; k < nel; ++k)
      if (alive.test(k)) ok &= sorted_insert(eb, ne2, MAXW, ne[k]);
    for (int k = 0; k < nnl; ++k) {
      int x = nn[k];
      int xs = c.vb + x;
      if (!sel.test(k)) {
        ok &= sorted_insert(nb, nn2, MAXW, x);
        continue;
      }
      int t = target[xs];
      if (t != lu) {
        ok &= sorted_insert(nb, nn2, MAXW, t);
        continue;
      }
      // the collapsed neighbour's rows, read in chunks; its elements'
      // liveness gathered before the merge so that those loads overlap
      int rb[MAXW];
      const int nnxl = S.NNlen[xs];
      load_row(nn_row(S, xs), nnxl, rb);
      for (int j = 0; j < nnxl; ++j)
        if (rb[j] != lu) ok &= sorted_insert(nb, nn2, MAXW, rb[j]);
      const int nexl = S.NElen[xs];
      load_row(ne_row(S, xs), nexl, rb);
      RowMask live;
#pragma unroll 4
      for (int j = 0; j < nexl; ++j)
        if (S.EN[c.eb + rb[j]].w) live.set(j);
      for (int j = 0; j < nexl; ++j)
        if (live.test(j)) ok &= sorted_insert(eb, ne2, MAXW, rb[j]);
    }
    if (!ok || nn2 > S.W || ne2 > S.W) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->maxdeg, max(nn2, ne2));
      continue;
    }
    int* wn = S.NN + (size_t)u * S.W;
    int* we = S.NE + (size_t)u * S.W;
    for (int k = 0; k < nn2; ++k) wn[k] = nb[k];
    for (int k = 0; k < ne2; ++k) we[k] = eb[k];
    S.NNlen[u] = nn2;
    S.NElen[u] = ne2;
    stamp_neighbours(S, nb, nn2, c.vb, tag + 1);
  }
}

__global__ void k_coarsen_commit(Store S, const int* A, const int* nAp, const int* target,
                                 const int* smark, int tag, DevStatus* st) {
  coarsen_commit_phase(S, A, nAp, target, smark, tag, st);
}

// ---- swapping (Sec. 2.4.3) ------------------------------------------------------

// Balls of at most this many elements take the register path of the flip
// scan (the ball's vertices gathered once); larger ones search the elements.
constexpr int kBallFast = 16;

// Warp-aggregated append of a work item into a list of capacity `cap`.
__device__ __forceinline__ void append_item(bool pred, int2 val, int2* list, int* count, int cap,
                                            DevStatus* st) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0) return;
  int lane = threadIdx.x & 31, leader = __ffs(m) - 1, base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    int pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < cap) list[pos] = val;
    else set_err(st, PM_ERR_CAPACITY);
  }
}

// A vertex whose ball holds more than kBallFast elements, listed by the whole
// warp (all lanes call): lane l gathers elements l, l + 32, ... into the
// warp's shared arrays and then finds the partner elements of its own poor
// elements there; the same pairs, in the same order per poor element, as the
// register path below.  One such vertex used to hold up its round: one thread
// walked its whole ball for every poor element.

__device__ __forceinline__ void swap_scan_heavy(const Store& S, int v, int* sx, int* sp,
                                                int2* items, int* nI, int icap, double* gains,
                                                DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const MeshCtx c = ctx_of(S, v);
  const int lv = v - c.vb;
  const int* ne = ne_row(S, v);
  const int nel = S.NElen[v];
  const double qt = S.tab.q_thresh[c.mi];
  unsigned pw[MAXW / 32];
#pragma unroll
  for (int j = 0; j < MAXW / 32; ++j) {
    const int k = 32 * j + lane;
    bool poor = false;
    if (k < nel) {
      const int K = ne[k];
      const int4 f = S.EN[c.eb + K];
      sx[k] = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;  // after v
      sp[k] = (f.x == lv) ? f.z : (f.y == lv) ? f.x : f.y;  // before v
      poor = dlt(S.qK[c.eb + K], qt);
      gains[(size_t)v * S.W + k] = -1.0;
    }
    pw[j] = __ballot_sync(0xffffffffu, poor);
  }
  __syncwarp();
  int at = 0;
  for (int pass = 0; pass < 2; ++pass) {  // count, reserve, write
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < MAXW / 32; ++j) {
      const int kb = 32 * j + lane;
      if (kb >= nel || !((pw[j] >> lane) & 1u)) continue;
      const int w = sx[kb], cc = sp[kb];
      int k2 = -1, k1 = -1;
      for (int k = 0; k < nel && (k2 < 0 || k1 < 0); ++k) {  // the first match wins
        if (k == kb) continue;
        if (k2 < 0 && sp[k] == w) k2 = k;
        if (k1 < 0 && sx[k] == cc) k1 = k;
      }
      if (k2 >= 0) {
        if (pass == 1) {
          if (at < icap) items[at] = make_int2(v, kb | (k2 << 8));
          else set_err(st, PM_ERR_CAPACITY);
          ++at;
        }
        ++cnt;
      }
      bool k1poor = false;
#pragma unroll
      for (int jj = 0; jj < MAXW / 32; ++jj)
        if (k1 >= 0 && (k1 >> 5) == jj) k1poor = (pw[jj] >> (k1 & 31)) & 1u;
      if (k1 >= 0 && !k1poor) {
        if (pass == 1) {
          if (at < icap) items[at] = make_int2(v, k1 | (kb << 8));
          else set_err(st, PM_ERR_CAPACITY);
          ++at;
        }
        ++cnt;
      }
    }
    if (pass == 0) at = warp_reserve(cnt, nI);
  }
  __syncwarp();  // the shared arrays serve the next heavy vertex
}

// Flip evaluation in three passes so that the FP64 work runs on full warps.
// Pass 1 (per dirty vertex): reuse an unchanged earlier result, or list the
// vertex's interior edges whose two elements' cached minimum quality is below
// q_thresh and whose flip would not duplicate an edge.
__device__ __forceinline__ void swap_scan_phase(Store S, const int* D, const int* nDp,
                                                const int4* opA, int* C, int* nC, int* cmark,
                                                int tag, int pass0, int* E, int* nE, int2* items,
                                                int* nI, int icap, double* gains, DevStatus* st,
                                                bool il = false) {
  __shared__ int s_hx[kScanWarps][MAXW], s_hp[kScanWarps][MAXW];
  const int wq = (threadIdx.x >> 5) % kScanWarps;
  const int n = *nDp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    int v = 0, nel = 0;
    bool reuse_cand = false, eval = false;
    MeshCtx c{0, 0, 0};
    const int* ne = nullptr;
    if (i < n) {
      v = D[i];
      c = ctx_of(S, v);
      if (unchanged(S, v, c.vb, S.evs[v], pass0)) {
        reuse_cand = opA[v].x >= 0;
        if (reuse_cand) {
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        }
      } else if (S.vflag[v] & VF_ALIVE) {
        eval = true;
        S.evs[v] = tag;
        ne = ne_row(S, v);
        nel = S.NElen[v];
      }
    }
    warp_append(reuse_cand, v, C, nC);
    warp_append(eval, v, E, nE);
    const int lv = v - c.vb;
    const double qt = eval ? S.tab.q_thresh[c.mi] : 0.0;
    // An edge (v, w) qualifies only when one of its two elements has quality
    // below q_thresh, so the pairs are found from v's poor elements alone.
    // Each poor element kb = (v, w, c) gives the pair (kb, k2), k2 the
    // element (v, d, w) after it around v, and the pair (k1, kb), k1 the
    // element before it, when k1 is not poor itself (else that pair is found
    // from k1).  Whether the flipped edge (c, d) already exists is left to
    // the gain evaluation (gain -1): the scan reads no adjacency row, so its
    // loop over the poor elements is register arithmetic.  Items are counted
    // first, reserved with one atomic per warp, then written.
    // balls above kBallFast elements are listed by the whole warp after the
    // register path, which the other lanes take
    const bool heavy = nel > kBallFast;
    const int nfast = heavy ? 0 : nel;
    {
      // the ball's vertices after and before v and its poor elements,
      // gathered once into registers (unrolled: the loads of all elements
      // are in flight together)
      int nx[kBallFast], pv[kBallFast];
      RowMask poor0;
#pragma unroll
      for (int k = 0; k < kBallFast; ++k) {
        nx[k] = pv[k] = -1;
        if (k < nfast) {
          const int K = ne[k];
          const int4 f = S.EN[c.eb + K];
          nx[k] = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;
          pv[k] = (f.x == lv) ? f.z : (f.y == lv) ? f.x : f.y;
          if (dlt(S.qK[c.eb + K], qt)) poor0.set(k);
          gains[(size_t)v * S.W + k] = -1.0;
        }
      }
      // pass 0 counts the items, pass 1 writes them
      int at = 0;
      for (int pass = 0; pass < 2; ++pass) {
        RowMask pm = poor0;
        int cnt = 0;
        while (pm.any()) {
          const int kb = pm.pop();
          int w = -1, cc = -1;
#pragma unroll
          for (int k = 0; k < kBallFast; ++k)
            if (k == kb) {
              w = nx[k];
              cc = pv[k];
            }
          int k2 = -1, k1 = -1;
#pragma unroll
          for (int k = kBallFast - 1; k >= 0; --k) {  // the first match wins
            if (k == kb || k >= nfast) continue;
            if (pv[k] == w) k2 = k;
            if (nx[k] == cc) k1 = k;
          }
          if (k2 >= 0) {
            if (pass == 1) {
              if (at < icap) items[at] = make_int2(v, kb | (k2 << 8));
              else set_err(st, PM_ERR_CAPACITY);
              ++at;
            }
            ++cnt;
          }
          if (k1 >= 0 && !poor0.test(k1)) {
            if (pass == 1) {
              if (at < icap) items[at] = make_int2(v, k1 | (kb << 8));
              else set_err(st, PM_ERR_CAPACITY);
              ++at;
            }
            ++cnt;
          }
        }
        if (pass == 0) at = warp_reserve(cnt, nI);
      }
    }
    for (unsigned hb = __ballot_sync(0xffffffffu, heavy); hb; hb &= hb - 1u) {
      const int hv = __shfl_sync(0xffffffffu, v, __ffs(hb) - 1);
      swap_scan_heavy(S, hv, s_hx[wq], s_hp[wq], items, nI, icap, gains, st);
    }
  }
}

__global__ void k_swap_scan(Store S, const int* D, const int* nDp, const int4* opA, int* C, int* nC,
                            int* cmark, int tag, int pass0, int* E, int* nE, int2* items, int* nI,
                            int icap, double* gains, DevStatus* st) {
  swap_scan_phase(S, D, nDp, opA, C, nC, cmark, tag, pass0, E, nE, items, nI, icap, gains, st);
}

// Pass 2 (per listed edge, dense FP64): both flipped elements counter-
// clockwise and their minimum quality above the old minimum -> the gain.
// Gain of flipping edge (v, w) shared by K1 = (v, w, c) and K2 = (v, d, w)
// (ball slots k1, k2 of v): both new elements counter-clockwise and their
// minimum quality above the old minimum, else -1.  The flip's c and d go to
// *cc and *d.
__device__ __forceinline__ double flip_gain(const Store& S, MeshCtx c, int lv, const int* ne,
                                            int k1, int k2, int* cc_out, int* d_out,
                                            unsigned& ops) {
  int K1 = ne[k1], K2 = ne[k2];
  int4 e = S.EN[c.eb + K1];
  int4 f = S.EN[c.eb + K2];
  int w = (e.x == lv) ? e.y : (e.y == lv) ? e.z : e.x;
  int cc = (e.x == lv) ? e.z : (e.y == lv) ? e.x : e.y;
  int d = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;
  *cc_out = cc;
  *d_out = d;
  double q1 = S.qK[c.eb + K1], q2 = S.qK[c.eb + K2];
  double qold = dlt(q1, q2) ? q1 : q2;
  VD dv = load_vd(S, c.vb + lv), dw = load_vd(S, c.vb + w), dc = load_vd(S, c.vb + cc),
     dd = load_vd(S, c.vb + d);
  // The gain is -1 unless all four hold: (v, d, c) and (d, w, c)
  // counter-clockwise, n1 > qold, n2 > qold.  A conjunction may be decided in
  // any order: the orientation filters first (a decided negative sign ends
  // it), then the qualities, and only then the exact sign of an orientation
  // the filter left open (nearly or exactly collinear points, whose element
  // has quality near zero and so has almost always failed by then).  Every
  // test is still made before a gain is returned, so the result is the one
  // of the order orientations-then-qualities whatever the values.
  const int s1 = orient_filter(dv, dd, dc);
  ops += kOpsOrient;
  if (s1 < 0) return -1.0;
  const int s2 = orient_filter(dd, dw, dc);
  ops += kOpsOrient;
  if (s2 < 0) return -1.0;
  ops += kOpsQuality;
  const double n1 = quality_c(lv, d, cc, dv, dd, dc);
  if (!dgt(n1, qold)) return -1.0;
  ops += kOpsQuality;
  const double n2 = quality_c(d, w, cc, dd, dw, dc);
  if (!dgt(n2, qold)) return -1.0;
  if (s1 == 0 || s2 == 0) {
    const VD pv = load_xy_again(S, c.vb + lv), pw = load_xy_again(S, c.vb + w),
             pc = load_xy_again(S, c.vb + cc), pd = load_xy_again(S, c.vb + d);
    if (s1 == 0 && orient_resolve(pv, pd, pc) <= 0) return -1.0;
    if (s2 == 0 && orient_resolve(pd, pw, pc) <= 0) return -1.0;
  }
  ops += 1;
  return (dlt(n1, n2) ? n1 : n2) - qold;
}

// An edge both of whose end points are evaluated this round is listed from
// both ends with the same two new elements: in canonical rotation their
// qualities and orientations, hence the gain, are bitwise equal from either
// side.  The end point with the smaller id evaluates it and writes the gain
// into both vertices' slots (the other's slot of the same element pair is
// found in its sorted element row); the other item does no arithmetic.
//
// A warp pays the FP64 issue cost of an instruction once whatever its active
// lanes, so the items that need arithmetic are collected in per-warp queues
// in shared memory and evaluated 32 at a time (full warps).  The tests of a
// gain end early (a decided negative orientation, a quality not above the
// old minimum), so each stage has its own queue: orientations, first
// quality, second quality and gain; an item that passes a stage joins the
// next stage's queue.  Only the last batch of each queue may be partial.
// At most 8 warps per block.
constexpr int kEdgeQueueWarps = 8;

// Queued item q = (v, k1 | k2 << 8 | both << 16 | open << 17, mesh, slot of
// w): the flip of edge (v, w) between v's ball elements k1 and k2.
struct FlipGeom {
  MeshCtx c;
  int lv, w, cc, d, K1, K2;
};

__device__ __forceinline__ FlipGeom flip_geom(const Store& S, int4 q) {
  FlipGeom g;
  g.c.mi = q.z;
  g.c.vb = S.tab.vbase[q.z];
  g.c.eb = S.tab.ebase[q.z];
  g.lv = q.x - g.c.vb;
  const int* ne = ne_row(S, q.x);
  g.K1 = ne[q.y & 0xFF];
  g.K2 = ne[(q.y >> 8) & 0xFF];
  const int4 e = S.EN[g.c.eb + g.K1];
  const int4 f = S.EN[g.c.eb + g.K2];
  g.w = (e.x == g.lv) ? e.y : (e.y == g.lv) ? e.z : e.x;
  g.cc = (e.x == g.lv) ? e.z : (e.y == g.lv) ? e.x : e.y;
  g.d = (f.x == g.lv) ? f.y : (f.y == g.lv) ? f.z : f.x;
  return g;
}

__device__ __forceinline__ double flip_qold(const Store& S, const FlipGeom& g) {
  const double q1 = S.qK[g.c.eb + g.K1], q2 = S.qK[g.c.eb + g.K2];
  return dlt(q1, q2) ? q1 : q2;
}

// The tests of flip_gain in the same order, one stage per queue: A the two
// orientation filters (0: failed, else 1 | the open signs << 1), B the first
// new quality, C the second, the open signs exactly, the gain.
__device__ __forceinline__ int flip_stage_a(const Store& S, int4 q, unsigned& ops) {
  const FlipGeom g = flip_geom(S, q);
  // the flipped edge (c, d) must not exist already
  if (row_has(nn_row(S, g.c.vb + g.d), S.NNlen[g.c.vb + g.d], g.cc)) return 0;
  const VD dv = load_vd(S, g.c.vb + g.lv), dw = load_vd(S, g.c.vb + g.w),
           dc = load_vd(S, g.c.vb + g.cc), dd = load_vd(S, g.c.vb + g.d);
  const int s1 = orient_filter(dv, dd, dc);
  ops += kOpsOrient;
  if (s1 < 0) return 0;
  const int s2 = orient_filter(dd, dw, dc);
  ops += kOpsOrient;
  if (s2 < 0) return 0;
  return 1 | (s1 == 0 ? 2 : 0) | (s2 == 0 ? 4 : 0);
}

__device__ __forceinline__ bool flip_stage_b(const Store& S, int4 q, double& n1, unsigned& ops) {
  const FlipGeom g = flip_geom(S, q);
  const VD dv = load_vd(S, g.c.vb + g.lv), dc = load_vd(S, g.c.vb + g.cc),
           dd = load_vd(S, g.c.vb + g.d);
  n1 = quality_c(g.lv, g.d, g.cc, dv, dd, dc);
  ops += kOpsQuality;
  return dgt(n1, flip_qold(S, g));
}

__device__ __forceinline__ double flip_stage_c(const Store& S, int4 q, double n1, unsigned& ops) {
  const FlipGeom g = flip_geom(S, q);
  const double qold = flip_qold(S, g);
  const VD dw = load_vd(S, g.c.vb + g.w), dc = load_vd(S, g.c.vb + g.cc),
           dd = load_vd(S, g.c.vb + g.d);
  const double n2 = quality_c(g.d, g.w, g.cc, dd, dw, dc);
  ops += kOpsQuality;
  if (!dgt(n2, qold)) return -1.0;
  const int open = (q.y >> 18) & 3;
  if (open) {
    const VD pv = load_xy_again(S, g.c.vb + g.lv), pw = load_xy_again(S, g.c.vb + g.w),
             pc = load_xy_again(S, g.c.vb + g.cc), pd = load_xy_again(S, g.c.vb + g.d);
    if ((open & 1) && orient_resolve(pv, pd, pc) <= 0) return -1.0;
    if ((open & 2) && orient_resolve(pd, pw, pc) <= 0) return -1.0;
  }
  ops += 1;
  return (dlt(n1, n2) ? n1 : n2) - qold;
}

// The gain of item q into v's slot and, when w evaluates the same edge this
// round, into w's slot of the same element pair.
__device__ __forceinline__ void flip_store_gain(const Store& S, int4 q, double g, double* gains) {
  const int v = q.x;
  gains[(size_t)v * S.W + (q.y & 0xFF)] = g;
  if ((q.y >> 16) & 1) {
    // from w's side the pair is (K2, K1): w's slot of K2
    const int K2 = ne_row(S, v)[(q.y >> 8) & 0xFF];
    const int* nw = ne_row(S, q.w);
    const int nwl = S.NElen[q.w];
    int kk = 0;
    while (kk < nwl && nw[kk] < K2) ++kk;
    if (kk < nwl) gains[(size_t)q.w * S.W + kk] = g;
  }
}

// Per-warp stage queues (shared memory), each holding fewer than 32 entries
// between calls; the counts are the same in every lane.  All lanes call.
struct FlipQueues {
  int4 *a, *b, *c;
  double* n1;
  int na, nb, nc;
};

__device__ __forceinline__ void flip_run_c(const Store& S, FlipQueues& Q, int cnt, double* gains,
                                           unsigned& ops) {
  const int lane = threadIdx.x & 31;
  if (lane < cnt) {
    const int4 q = Q.c[lane];
    flip_store_gain(S, q, flip_stage_c(S, q, Q.n1[lane], ops), gains);
  }
  __syncwarp();
  if (lane < Q.nc - cnt) {
    Q.c[lane] = Q.c[cnt + lane];
    Q.n1[lane] = Q.n1[cnt + lane];
  }
  Q.nc -= cnt;
  __syncwarp();
}

__device__ __forceinline__ void flip_run_b(const Store& S, FlipQueues& Q, int cnt, double* gains,
                                           unsigned& ops) {
  const int lane = threadIdx.x & 31;
  bool pass = false;
  int4 q = make_int4(0, 0, 0, 0);
  double n1 = 0.0;
  if (lane < cnt) {
    q = Q.b[lane];
    pass = flip_stage_b(S, q, n1, ops);
    if (!pass) flip_store_gain(S, q, -1.0, gains);
  }
  __syncwarp();
  if (lane < Q.nb - cnt) Q.b[lane] = Q.b[cnt + lane];
  Q.nb -= cnt;
  const unsigned m = __ballot_sync(0xffffffffu, pass);
  if (pass) {
    const int at = Q.nc + __popc(m & ((1u << lane) - 1u));
    Q.c[at] = q;
    Q.n1[at] = n1;
  }
  Q.nc += __popc(m);
  __syncwarp();
  if (Q.nc >= 32) flip_run_c(S, Q, 32, gains, ops);
}

__device__ __forceinline__ void flip_run_a(const Store& S, FlipQueues& Q, int cnt, double* gains,
                                           unsigned& ops) {
  const int lane = threadIdx.x & 31;
  bool pass = false;
  int4 q = make_int4(0, 0, 0, 0);
  if (lane < cnt) {
    q = Q.a[lane];
    const int r = flip_stage_a(S, q, ops);
    pass = r != 0;
    if (pass) q.y |= (r >> 1) << 18;
    else flip_store_gain(S, q, -1.0, gains);
  }
  __syncwarp();
  if (lane < Q.na - cnt) Q.a[lane] = Q.a[cnt + lane];
  Q.na -= cnt;
  const unsigned m = __ballot_sync(0xffffffffu, pass);
  if (pass) Q.b[Q.nb + __popc(m & ((1u << lane) - 1u))] = q;
  Q.nb += __popc(m);
  __syncwarp();
  if (Q.nb >= 32) flip_run_b(S, Q, 32, gains, ops);
}

__device__ __forceinline__ void swap_edge_phase(Store S, const int2* items, const int* nIp,
                                                double* gains, int tag, unsigned long long* work,
                                                bool il = false) {
  __shared__ int4 sqa[kEdgeQueueWarps][64];
  __shared__ int4 sqb[kEdgeQueueWarps][64];
  __shared__ int4 sqc[kEdgeQueueWarps][64];
  __shared__ double sn1[kEdgeQueueWarps][64];
  const int n = *nIp;
  const int lane = threadIdx.x & 31;
  const int wq = (threadIdx.x >> 5) % kEdgeQueueWarps;
  FlipQueues Q{sqa[wq], sqb[wq], sqc[wq], sn1[wq], 0, 0, 0};
  unsigned ops = 0;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    const int i = i0 + grank(il);
    bool need = false;
    int4 rec = make_int4(0, 0, 0, 0);
    if (i < n) {
      int2 it = items[i];
      int v = it.x, k1 = it.y & 0xFF, k2 = it.y >> 8;
      MeshCtx c = ctx_of(S, v);
      const int lv = v - c.vb;
      const int4 e = S.EN[c.eb + ne_row(S, v)[k1]];
      const int w = (e.x == lv) ? e.y : (e.y == lv) ? e.z : e.x;
      const int sw = c.vb + w;
      const bool both = S.evs[sw] == tag;
      need = !both || lv < w;
      rec = make_int4(v, k1 | (k2 << 8) | ((both ? 1 : 0) << 16), c.mi, sw);
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) Q.a[Q.na + __popc(m & ((1u << lane) - 1u))] = rec;
    Q.na += __popc(m);
    __syncwarp();
    if (Q.na >= 32) flip_run_a(S, Q, 32, gains, ops);
  }
  if (Q.na > 0) flip_run_a(S, Q, Q.na, gains, ops);
  if (Q.nb > 0) flip_run_b(S, Q, Q.nb, gains, ops);
  if (Q.nc > 0) flip_run_c(S, Q, Q.nc, gains, ops);
  add_work(work, ops);
}

__global__ void k_swap_edge(Store S, const int2* items, const int* nIp, double* gains, int tag,
                            unsigned long long* work) {
  swap_edge_phase(S, items, nIp, gains, tag, work);
}

// Pass 3 (per evaluated vertex): largest strictly positive gain, ties to the
// smallest w; the flip record (w, c, d, K1, K2) of the winner.
__device__ __forceinline__ void swap_pick_phase(Store S, const int* E, const int* nEp,
                                                const double* gains, int4* opA, int* opK2, int* C,
                                                int* nC, int* cmark, int tag, bool il = false) {
  const int n = *nEp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    int v = 0;
    bool found = false;
    if (i < n) {
      v = E[i];
      MeshCtx c = ctx_of(S, v);
      int lv = v - c.vb;
      const int* ne = ne_row(S, v);
      int nel = S.NElen[v];
      double best = 0.0;
      int bw = 0, bk = -1;
      if (nel <= kBallFast) {
        // gains, elements and the vertices after and before v gathered in
        // one unrolled pass (all loads in flight together), then decided in
        // registers
        int nx[kBallFast], pv[kBallFast], K[kBallFast];
        double g[kBallFast];
#pragma unroll
        for (int k = 0; k < kBallFast; ++k) {
          nx[k] = pv[k] = K[k] = -1;
          g[k] = -1.0;
          if (k < nel) {
            K[k] = ne[k];
            g[k] = gains[(size_t)v * S.W + k];
            const int4 f = S.EN[c.eb + K[k]];
            nx[k] = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;
            pv[k] = (f.x == lv) ? f.z : (f.y == lv) ? f.x : f.y;
          }
        }
        int bc = 0;
#pragma unroll
        for (int k = 0; k < kBallFast; ++k) {
          if (k < nel && dgt(g[k], 0.0) &&
              (!found || dgt(g[k], best) || (dbits(g[k]) == dbits(best) && nx[k] < bw))) {
            found = true;
            best = g[k];
            bw = nx[k];
            bk = k;
            bc = pv[k];
          }
        }
        if (found) {
          int k2 = -1;
#pragma unroll
          for (int k = kBallFast - 1; k >= 0; --k)  // the first match wins
            if (k < nel && pv[k] == bw) k2 = k;
          int K1 = -1, K2 = -1, d = -1;
#pragma unroll
          for (int k = 0; k < kBallFast; ++k) {
            if (k == bk) K1 = K[k];
            if (k == k2) {
              K2 = K[k];
              d = nx[k];
            }
          }
          opA[v] = make_int4(bw, bc, d, K1);
          opK2[v] = K2;
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        } else {
          opA[v].x = -1;
        }
      } else {
#pragma unroll 8
        for (int k = 0; k < nel; ++k) {
          double g = gains[(size_t)v * S.W + k];
          if (!dgt(g, 0.0)) continue;
          int4 e = S.EN[c.eb + ne[k]];
          int w = (e.x == lv) ? e.y : (e.y == lv) ? e.z : e.x;
          if (!found || dgt(g, best) || (dbits(g) == dbits(best) && w < bw)) {
            found = true;
            best = g;
            bw = w;
            bk = k;
          }
        }
        if (found) {
          int4 e = S.EN[c.eb + ne[bk]];
          int cc = (e.x == lv) ? e.z : (e.y == lv) ? e.x : e.y;
          int k2 = -1;
#pragma unroll 8
          for (int k = nel - 1; k >= 0; --k) {  // the first match wins
            int4 f = S.EN[c.eb + ne[k]];
            int pv = (f.x == lv) ? f.z : (f.y == lv) ? f.x : f.y;
            if (pv == bw) k2 = k;
          }
          int4 f = S.EN[c.eb + ne[k2]];
          int d = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;
          opA[v] = make_int4(bw, cc, d, ne[bk]);
          opK2[v] = ne[k2];
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        } else {
          opA[v].x = -1;
        }
      }
    }
    warp_append(found, v, C, nC);
  }
}

__global__ void k_swap_pick(Store S, const int* E, const int* nEp, const double* gains, int4* opA,
                            int* opK2, int* C, int* nC, int* cmark, int tag) {
  swap_pick_phase(S, E, nEp, gains, opA, opK2, C, nC, cmark, tag);
}

// Passes 1-3 in one, for persistent rounds whose list fits one pass of the
// grid's tiles: lane j of v's tile takes v's ball elements j, j + 8, ... as
// K1 of the edge (v, w) that follows v in it, lists the edge by pass 1's rule
// (interior, one of the pair below q_thresh, the flip duplicates no edge),
// evaluates its gain (pass 2), and the tile keeps the largest positive gain,
// ties to the smallest w (pass 3's order: a total order, w differs between
// v's edges).  Each edge of v is the K1 edge of exactly one ball element, so
// the candidate edges are those pass 1 lists.  Two barriers fewer per round.
__device__ __forceinline__ bool flip_better(bool f2, double g2, int w2, bool f, double g, int w) {
  return f2 && (!f || dgt(g2, g) || (dbits(g2) == dbits(g) && w2 < w));
}

__device__ __forceinline__ void swap_scan_eval_phase(Store S, const int* D, const int* nDp,
                                                     int4* opA, int* opK2, int* C, int* nC,
                                                     int* cmark, int tag, int pass0,
                                                     unsigned long long* work) {
  const Tile t = tile_of();
  const int n = *nDp;
  unsigned ops = 0;
  for (int i0 = 0; i0 < n; i0 += tcount()) {
    const int i = i0 + trank(true);
    int v = 0;
    bool cand = false;
    if (i < n) {
      v = D[i];
      MeshCtx c = ctx_of(S, v);
      const int et = __shfl_sync(t.mask, S.evs[v], 0, TW);
      if (unchanged(S, v, c.vb, et, pass0)) {
        cand = opA[v].x >= 0;
        if (cand && t.tl == 0) {
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        }
      } else if (S.vflag[v] & VF_ALIVE) {
        if (t.tl == 0) S.evs[v] = tag;
        const int lv = v - c.vb;
        const int* ne = ne_row(S, v);
        const int nel = S.NElen[v];
        const double qt = S.tab.q_thresh[c.mi];
        bool found = false;
        double best = 0.0;
        int bw = 0, bk1 = -1, bk2 = -1, bc = 0, bd = 0;
        for (int k = t.tl; k < nel; k += TW) {
          const int K1 = ne[k];
          const int4 e = S.EN[c.eb + K1];
          const int w = (e.x == lv) ? e.y : (e.y == lv) ? e.z : e.x;   // after v
          const int cc = (e.x == lv) ? e.z : (e.y == lv) ? e.x : e.y;  // before v
          int k2 = -1, d = 0;
          for (int j = 0; j < nel; ++j) {
            if (j == k) continue;
            const int4 f = S.EN[c.eb + ne[j]];
            if (((f.x == lv) ? f.z : (f.y == lv) ? f.x : f.y) == w) {
              k2 = j;
              d = (f.x == lv) ? f.y : (f.y == lv) ? f.z : f.x;
              break;
            }
          }
          if (k2 < 0) continue;  // boundary edge
          if (!dlt(S.qK[c.eb + K1], qt) && !dlt(S.qK[c.eb + ne[k2]], qt)) continue;
          if (row_has(nn_row(S, c.vb + d), S.NNlen[c.vb + d], cc)) continue;
          int c2, d2;
          const double g = flip_gain(S, c, lv, ne, k, k2, &c2, &d2, ops);
          if (!dgt(g, 0.0)) continue;
          if (flip_better(true, g, w, found, best, bw)) {
            found = true;
            best = g;
            bw = w;
            bk1 = k;
            bk2 = k2;
            bc = cc;
            bd = d;
          }
        }
#pragma unroll
        for (int o = TW / 2; o > 0; o >>= 1) {
          const bool f2 = __shfl_xor_sync(t.mask, found ? 1 : 0, o, TW) != 0;
          const double g2 = __shfl_xor_sync(t.mask, best, o, TW);
          const int w2 = __shfl_xor_sync(t.mask, bw, o, TW);
          const int k1b = __shfl_xor_sync(t.mask, bk1, o, TW);
          const int k2b = __shfl_xor_sync(t.mask, bk2, o, TW);
          const int cb = __shfl_xor_sync(t.mask, bc, o, TW);
          const int db = __shfl_xor_sync(t.mask, bd, o, TW);
          if (flip_better(f2, g2, w2, found, best, bw)) {
            found = true;
            best = g2;
            bw = w2;
            bk1 = k1b;
            bk2 = k2b;
            bc = cb;
            bd = db;
          }
        }
        if (t.tl == 0) {
          if (found) {
            opA[v] = make_int4(bw, bc, bd, ne[bk1]);
            opK2[v] = ne[bk2];
            cmark[v] = tag;
            S.tab.had[c.mi] = 1;
          } else {
            opA[v].x = -1;
          }
        }
        cand = found;
      }
    }
    warp_append(cand && t.tl == 0, v, C, nC);
  }
  add_work(work, ops);
}

// The two new elements' qualities are left to a dense pass (their slots join
// list Q), as for collapses.
__device__ __forceinline__ void swap_apply_one(const Store& S, bool ok, int v, const int4* opA,
                                               const int* opK2, int* A, int* nA, int* amark,
                                               int* Dn, int* nDn, int* dmark, int tag, int* Q,
                                               int* nQ) {
  {
    int mi = 0, q1 = 0, q2 = 0;
    int t[4] = {0, 0, 0, 0};
    if (ok) {
      MeshCtx c = ctx_of(S, v);
      mi = c.mi;
      int lv = v - c.vb;
      int4 op = opA[v];
      int K2 = opK2[v];
      int4 t1 = make_int4(lv, op.z, op.y, 1);  // K1 = (v, d, c)
      int4 t2 = make_int4(op.z, op.x, op.y, 1);  // K2 = (d, w, c)
      S.EN[c.eb + op.w] = t1;
      S.EN[c.eb + K2] = t2;
      q1 = c.eb + op.w;
      q2 = c.eb + K2;
      t[0] = v;
      t[1] = c.vb + op.x;
      t[2] = c.vb + op.y;
      t[3] = c.vb + op.z;
    }
    count_op(S, ok, mi);
    bool fa[4], fd[4];
    int na = 0, nd = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      fa[k] = ok && stamp_first(amark, t[k], tag);
      fd[k] = ok && stamp_first(dmark, t[k], tag);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      na += fa[k];
      nd += fd[k];
    }
    int pa = warp_reserve(na, nA);
    int pd = warp_reserve(nd, nDn);
    int pq = warp_reserve(ok ? 2 : 0, nQ);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (fa[k]) A[pa++] = t[k];
      if (fd[k]) Dn[pd++] = t[k];
    }
    if (ok) {
      Q[pq] = q1;
      Q[pq + 1] = q2;
    }
  }
}

// One round's independent set and its flips (see k_coarsen_select_apply).
__device__ __forceinline__ void swap_select_apply_phase(Store S, const int* C, const int* nCp,
                                                        const int* cmark, int* smark, int tag,
                                                        const int4* opA, const int* opK2, int* A,
                                                        int* nA, int* amark, int* Dn, int* nDn,
                                                        int* dmark, int* Q, int* nQ,
                                                        bool il = false) {
  const int n = *nCp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    bool win = false, lose = false;
    int v = 0;
    if (i < n) {
      v = C[i];
      win = local_max(S, v, cmark, tag);
      if (win) smark[v] = tag;
      else lose = stamp_first(dmark, v, tag);
    }
    warp_append(lose, v, Dn, nDn);
    swap_apply_one(S, win, v, opA, opK2, A, nA, amark, Dn, nDn, dmark, tag, Q, nQ);
  }
}

__global__ void k_swap_select_apply(Store S, const int* C, const int* nCp, const int* cmark,
                                    int* smark, int tag, const int4* opA, const int* opK2, int* A,
                                    int* nA, int* amark, int* Dn, int* nDn, int* dmark, int* Q,
                                    int* nQ, unsigned* done) {
  swap_select_apply_phase(S, C, nCp, cmark, smark, tag, opA, opK2, A, nA, amark, Dn, nDn, dmark,
                          Q, nQ);
  round_done(S, done);
}

// Deferred-update commit of a swap round for affected vertex u, from the
// flips of u itself and of its S neighbours (records w, c, d, K1, K2):
//   u == v: NN -w, NE -K2;  u == w: NN -v, NE -K1;
//   u == c: NN +d, NE +K2;  u == d: NN +c, NE +K1.
__device__ __forceinline__ void swap_commit_phase(Store S, const int* A, const int* nAp,
                                                  const int4* opA, const int* opK2,
                                                  const int* smark, int tag, DevStatus* st,
                                                  bool il = false) {
  const int n = *nAp;
  for (int i = grank(il); i < n; i += gsize()) {
    int u = A[i];
    S.touch[u] = tag + 1;
    MeshCtx c = ctx_of(S, u);
    int lu = u - c.vb;
    int* nn = S.NN + (size_t)u * S.W;
    int* ne = S.NE + (size_t)u * S.W;
    int nnl = S.NNlen[u], nel = S.NElen[u];
    int nb[MAXW], eb[MAXW];
    load_row(nn, nnl, nb);
    load_row(ne, nel, eb);
    int nn2 = nnl, ne2 = nel;
    bool ok = true;
    RowMask sel;
#pragma unroll 4
    for (int k = 0; k < nnl; ++k)
      if (smark[c.vb + nn[k]] == tag) sel.set(k);
    const bool self = smark[u] == tag;
    for (int k = -1; k < nnl; ++k) {
      if (k < 0 ? !self : !sel.test(k)) continue;
      int x = (k < 0) ? lu : nn[k];
      int xs = c.vb + x;
      int4 op = opA[xs];
      int K2 = opK2[xs];
      if (x == lu) {
        sorted_erase(nb, nn2, op.x);
        sorted_erase(eb, ne2, K2);
      }
      if (op.x == lu) {
        sorted_erase(nb, nn2, x);
        sorted_erase(eb, ne2, op.w);
      }
      if (op.y == lu) {
        ok &= sorted_insert(nb, nn2, MAXW, op.z);
        ok &= sorted_insert(eb, ne2, MAXW, K2);
      }
      if (op.z == lu) {
        ok &= sorted_insert(nb, nn2, MAXW, op.y);
        ok &= sorted_insert(eb, ne2, MAXW, op.w);
      }
    }
    if (!ok || nn2 > S.W || ne2 > S.W) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->maxdeg, max(nn2, ne2));
      continue;
    }
    for (int k = 0; k < nn2; ++k) nn[k] = nb[k];
    for (int k = 0; k < ne2; ++k) ne[k] = eb[k];
    S.NNlen[u] = nn2;
    S.NElen[u] = ne2;
    stamp_neighbours(S, nb, nn2, c.vb, tag + 1);
  }
}

__global__ void k_swap_commit(Store S, const int* A, const int* nAp, const int4* opA,
                              const int* opK2, const int* smark, int tag, DevStatus* st) {
  swap_commit_phase(S, A, nAp, opA, opK2, smark, tag, st);
}

// ---- smoothing (Sec. 2.4.4) -------------------------------------------------------

__device__ __forceinline__ double ball_min_quality(const Store& S, MeshCtx c, const int* ne,
                                                   int nel, double* qsum) {
  double qmin = 0.0, sum = 0.0;
#pragma unroll 4
  for (int k = 0; k < nel; ++k) {
    double q = S.qK[c.eb + ne[k]];
    if (k == 0 || dlt(q, qmin)) qmin = q;
    sum = sum + q;
  }
  if (qsum) *qsum = sum;
  return qmin;
}

// Smoothing evaluation in two passes.  Pass 1 (per pending vertex): reuse an
// unchanged earlier result, drop vertices whose ball is already good enough
// (cached qualities), list the rest for the full move evaluation.
__device__ __forceinline__ void smooth_scan_phase(Store S, const int* D, const int* nDp,
                                                  double4* mvM, int* C, int* nC, int* cmark,
                                                  int tag, int pass0, int* E, int* nE,
                                                  bool il = false) {
  const int n = *nDp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    int v = 0;
    bool reuse_cand = false, eval = false;
    if (i < n) {
      v = D[i];
      MeshCtx c = ctx_of(S, v);
      if (unchanged(S, v, c.vb, S.evm[v], pass0)) {
        reuse_cand = mvM[v].w != 0.0;
        if (reuse_cand) {
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        }
      } else {
        S.evm[v] = tag;
        uint8_t f = S.vflag[v];
        if ((f & VF_ALIVE) && !(f & VF_BND)) {
          double qold = ball_min_quality(S, c, ne_row(S, v), S.NElen[v], nullptr);
          eval = dlt(qold, S.tab.q_thresh[c.mi]);
        }
        if (!eval) mvM[v].w = 0.0;
      }
    }
    warp_append(reuse_cand, v, C, nC);
    warp_append(eval, v, E, nE);
  }
}

__global__ void k_smooth_scan(Store S, const int* D, const int* nDp, double4* mvM, int* C, int* nC,
                              int* cmark, int tag, int pass0, int* E, int* nE) {
  smooth_scan_phase(S, D, nDp, mvM, C, nC, cmark, tag, pass0, E, nE);
}

// Minimum cached quality of v's ball (and, if asked, its sum in ascending
// element order).
__device__ double tile_ball_quality(const Tile& t, const Store& S, MeshCtx c, const int* ne,
                                    int nel, double* qsum) {
  double qmin = 1e300, sum = 0.0;
  for (int base = 0; base < nel; base += TW) {
    int k = base + t.tl;
    double q = (k < nel) ? S.qK[c.eb + ne[k]] : 1e300;
    qmin = dlt(q, qmin) ? q : qmin;
    if (qsum) {
      int cnt = min(TW, nel - base);
      for (int j = 0; j < cnt; ++j) sum = sum + tshfl(t, q, j);
    }
  }
  if (qsum) *qsum = sum;
  return tmin(t, qmin);
}

// First ball element (ascending id) that contains X, with v at its current
// place: its barycentric metric interpolation.
__device__ bool tile_interpolate(const Tile& t, const Store& S, MeshCtx c, const int* ne, int nel,
                                 double X, double Y, double4& Mout, int* tested = nullptr) {
  VD px{X, Y, 0.0, 0.0, 0.0};
  for (int base = 0; base < nel; base += TW) {
    if (tested) *tested += min(TW, nel - base);
    int k = base + t.tl;
    bool inside = false;
    VD a{}, b{}, d{};
    double o = 1.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (k < nel) {
      int4 e = S.EN[c.eb + ne[k]];
      int i0 = e.x, i1 = e.y, i2 = e.z;
      a = load_vd(S, c.vb + i0);
      b = load_vd(S, c.vb + i1);
      d = load_vd(S, c.vb + i2);
      canon(i0, i1, i2, a, b, d);
      // filters first; a lane with a sign left open (X on or near an edge
      // line) resolves it exactly below, all such lanes in one pass per sign
      int f0 = orient_filter(px, b, d), f1 = orient_filter(a, px, d), f2 = orient_filter(a, b, px);
      while ((f0 | f1 | f2) >= 0 && (f0 == 0 || f1 == 0 || f2 == 0)) {
        const int j = f0 == 0 ? 0 : (f1 == 0 ? 1 : 2);
        const int r = orient_resolve(j == 0 ? px : a, j == 1 ? px : b, j == 2 ? px : d);
        const int fr = r == 0 ? 2 : r;  // decided: an exact zero counts as inside
        if (j == 0) f0 = fr; else if (j == 1) f1 = fr; else f2 = fr;
      }
      inside = f0 > 0 && f1 > 0 && f2 > 0;
      if (inside) {
        o = orient3(a, b, d);
        s0 = orient3(px, b, d);
        s1 = orient3(a, px, d);
        s2 = orient3(a, b, px);
      }
    }
    unsigned bal = (__ballot_sync(t.mask, inside) >> t.shift) & 0xFFu;
    if (bal) {
      int src = __ffs(bal) - 1;
      double m0 = 0.0, m1 = 0.0, m2 = 0.0;
      if (t.tl == src) {
        double l0 = s0 / o, l1 = s1 / o, l2 = s2 / o;
        m0 = (l0 * a.m00 + l1 * b.m00) + l2 * d.m00;
        m1 = (l0 * a.m01 + l1 * b.m01) + l2 * d.m01;
        m2 = (l0 * a.m11 + l1 * b.m11) + l2 * d.m11;
      }
      Mout = make_double4(tshfl(t, m0, src), tshfl(t, m1, src), tshfl(t, m2, src), 0.0);
      return true;
    }
  }
  return false;
}

// Ball with v moved to (X, Y, Mv): every element counter-clockwise, and every
// quality above *floor (strict) or at least *floor (non-strict).  Writes each
// element's new quality to qout[k] and returns the ascending-order sum.
__device__ bool tile_ball_after_move(const Tile& t, const Store& S, MeshCtx c, int lv,
                                     const int* ne, int nel, double X, double Y, double4 Mv,
                                     double floor, bool strict, double* qout, double* qsum) {
  VD nvd{X, Y, Mv.x, Mv.y, Mv.z};
  bool ok = true;
  double sum = 0.0;
  for (int base = 0; base < nel; base += TW) {
    int k = base + t.tl;
    double q = 0.0;
    if (k < nel) {
      int4 e = S.EN[c.eb + ne[k]];
      VD a = (e.x == lv) ? nvd : load_vd(S, c.vb + e.x);
      VD b = (e.y == lv) ? nvd : load_vd(S, c.vb + e.y);
      VD d = (e.z == lv) ? nvd : load_vd(S, c.vb + e.z);
      if (orient_sign(a, b, d) > 0) {
        q = quality_c(e.x, e.y, e.z, a, b, d);
        if (strict ? !dgt(q, floor) : dlt(q, floor)) ok = false;
        if (qout) qout[k] = q;
      } else {
        ok = false;
      }
    }
    if (qsum) {
      int cnt = min(TW, nel - base);
      for (int j = 0; j < cnt; ++j) sum = sum + tshfl(t, q, j);
    }
  }
  if (qsum) *qsum = sum;
  return tall(t, ok);
}

// Quality-constrained Laplacian move of v: metric-weighted neighbour mean,
// metric interpolated at the target, kept when the ball stays valid and its
// minimum quality strictly increases.
// `ops` receives the FP64 operations (+ - * / sqrt) of the path taken: 17 per
// neighbour (Laplacian), 11 (solve), 28 per element tested in the location
// (four orientations), 18 (barycentrics and metric) and 77 per element of the
// ball check (orientation 7 + quality 70).
__device__ bool tile_smooth_eval(const Tile& t, const Store& S, int v, MeshCtx c, double2& Xo,
                                 double4& Mo, double* qout, int& ops) {
  ops = 0;
  uint8_t f = S.vflag[v];
  if (!(f & VF_ALIVE) || (f & VF_BND)) return false;
  const int* ne = ne_row(S, v);
  int nel = S.NElen[v];
  double qold = tile_ball_quality(t, S, c, ne, nel, nullptr);
  if (!dlt(qold, S.tab.q_thresh[c.mi])) return false;
  const int* nn = nn_row(S, v);
  int nnl = S.NNlen[v];
  double4 mv = S.M[v];
  double a00 = 0.0, a01 = 0.0, a11 = 0.0, b0 = 0.0, b1 = 0.0;
  for (int base = 0; base < nnl; base += TW) {
    int k = base + t.tl;
    double w00 = 0.0, w01 = 0.0, w11 = 0.0, t0 = 0.0, t1 = 0.0;
    if (k < nnl) {
      int js = c.vb + nn[k];
      double2 pj = S.xy[js];
      double4 mj = S.M[js];
      w00 = 0.5 * (mv.x + mj.x);
      w01 = 0.5 * (mv.y + mj.y);
      w11 = 0.5 * (mv.z + mj.z);
      t0 = w00 * pj.x + w01 * pj.y;
      t1 = w01 * pj.x + w11 * pj.y;
    }
    int cnt = min(TW, nnl - base);
    for (int j = 0; j < cnt; ++j) {
      a00 = a00 + tshfl(t, w00, j);
      a01 = a01 + tshfl(t, w01, j);
      a11 = a11 + tshfl(t, w11, j);
      b0 = b0 + tshfl(t, t0, j);
      b1 = b1 + tshfl(t, t1, j);
    }
  }
  ops = 17 * nnl + 3;
  double det = a00 * a11 - a01 * a01;
  if (!dgt(det, 0.0)) return false;
  double x = (a11 * b0 - a01 * b1) / det;
  double y = (a00 * b1 - a01 * b0) / det;
  ops += 8;
  double4 Mn;
  int tested = 0;
  bool found = tile_interpolate(t, S, c, ne, nel, x, y, Mn, &tested);
  ops += 28 * tested;
  if (!found) return false;
  ops += 18 + 77 * nel;
  if (!tile_ball_after_move(t, S, c, v - c.vb, ne, nel, x, y, Mn, qold, true, qout, nullptr))
    return false;
  Xo = make_double2(x, y);
  Mo = Mn;
  return true;
}

// Pass 2 (one 8-lane tile per listed vertex): the full quality-constrained move.
__device__ __forceinline__ void smooth_eval_phase(Store S, const int* E, const int* nEp,
                                                  double2* mvxy, double4* mvM, double* qball,
                                                  int* C, int* nC, int* cmark, int tag,
                                                  unsigned long long* work, bool il = false) {
  const int n = *nEp;
  const Tile t = tile_of();
  const int tiles_per_block = blockDim.x / TW;
  const int tile_rank = il ? (threadIdx.x / TW) * gridDim.x + blockIdx.x
                          : blockIdx.x * tiles_per_block + threadIdx.x / TW;
  for (int j0 = 0; j0 < n; j0 += gridDim.x * tiles_per_block) {
    int j = j0 + tile_rank;
    int v = 0, ops = 0;
    bool cand = false;
    if (j < n) {
      v = E[j];
      MeshCtx c = ctx_of(S, v);
      double2 X;
      double4 Mv;
      // the new ball qualities of an accepted move are kept for the apply
      cand = tile_smooth_eval(t, S, v, c, X, Mv, qball + (size_t)v * S.W, ops);
      if (t.tl == 0) {
        if (cand) {
          Mv.w = 1.0;  // marks a stored move
          mvxy[v] = X;
          mvM[v] = Mv;
          cmark[v] = tag;
          S.tab.had[c.mi] = 1;
        } else {
          mvM[v].w = 0.0;
        }
      }
    }
    warp_append(cand && t.tl == 0, v, C, nC);
    if (work) {  // measurement only: one atomic per warp
      unsigned tot = __reduce_add_sync(0xffffffffu, t.tl == 0 ? (unsigned)ops : 0u);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(work, (unsigned long long)tot);
    }
  }
}

// Passes 1 and 2 in one (persistent rounds whose list fits one tile per
// listed vertex): an evaluation whose inputs carry no newer stamp stands, the
// others are made again.  The tile takes the stamp decision from lane 0, after every
// lane has read the stamp (the shuffle) and before lane 0 overwrites it.
__device__ __forceinline__ void smooth_scan_eval_phase(Store S, const int* D, const int* nDp,
                                                       double2* mvxy, double4* mvM, double* qball,
                                                       int* C, int* nC, int* cmark, int tag,
                                                       int pass0, unsigned long long* work) {
  const int n = *nDp;
  const Tile t = tile_of();
  const int tile_rank = (threadIdx.x / TW) * gridDim.x + blockIdx.x;
  const int tiles = gridDim.x * (blockDim.x / TW);
  for (int j0 = 0; j0 < n; j0 += tiles) {
    int j = j0 + tile_rank;
    int v = 0, ops = 0;
    bool cand = false;
    if (j < n) {
      v = D[j];
      MeshCtx c = ctx_of(S, v);
      bool keep = unchanged(S, v, c.vb, S.evm[v], pass0);
      keep = __shfl_sync(t.mask, keep, 0, TW);
      if (keep) {
        if (t.tl == 0) {
          cand = mvM[v].w != 0.0;
          if (cand) {
            cmark[v] = tag;
            S.tab.had[c.mi] = 1;
          }
        }
      } else {
        double2 X;
        double4 Mv;
        cand = tile_smooth_eval(t, S, v, c, X, Mv, qball + (size_t)v * S.W, ops);
        if (t.tl == 0) {
          S.evm[v] = tag;
          if (cand) {
            Mv.w = 1.0;  // marks a stored move
            mvxy[v] = X;
            mvM[v] = Mv;
            cmark[v] = tag;
            S.tab.had[c.mi] = 1;
          } else {
            mvM[v].w = 0.0;
          }
        }
      }
    }
    warp_append(cand && t.tl == 0, v, C, nC);
    if (work) {  // measurement only: one atomic per warp
      unsigned tot = __reduce_add_sync(0xffffffffu, t.tl == 0 ? (unsigned)ops : 0u);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(work, (unsigned long long)tot);
    }
  }
}

__global__ void k_smooth_eval(Store S, const int* E, const int* nEp, double2* mvxy, double4* mvM,
                              double* qball, int* C, int* nC, int* cmark, int tag,
                              unsigned long long* work) {
  smooth_eval_phase(S, E, nEp, mvxy, mvM, qball, C, nC, cmark, tag, work);
}

// Move the members of S; live interior neighbours become pending for the next
// sweep (stamp pmark with the sweep tag).
__device__ __forceinline__ void smooth_apply_one(const Store& S, bool ok, int v,
                                                 const double2* mvxy, const double4* mvM,
                                                 const double* qball, int* P, int* nP,
                                                 int* pmark, int ptag, int stamp) {
  {
    int mi = 0, vb = 0, nnl = 0;
    const int* nn = nullptr;
    if (ok) {
      MeshCtx c = ctx_of(S, v);
      mi = c.mi;
      vb = c.vb;
      S.xy[v] = mvxy[v];
      double4 mv = mvM[v];
      mv.w = 0.0;
      S.M[v] = mv;
      S.touch[v] = stamp;
      const int* ne = ne_row(S, v);
      int nel = S.NElen[v];
      for (int k = 0; k < nel; ++k) S.qK[c.eb + ne[k]] = qball[(size_t)v * S.W + k];
      nn = nn_row(S, v);
      nnl = S.NNlen[v];
      stamp_neighbours(S, nn, nnl, vb, stamp);
    }
    count_op(S, ok, mi);
    RowMask take;
#pragma unroll 4
    for (int k = 0; k < nnl; ++k) {
      int s = vb + nn[k];
      uint8_t f = S.vflag[s];
      if ((f & VF_ALIVE) && !(f & VF_BND) && stamp_first(pmark, s, ptag)) take.set(k);
    }
    int pp = warp_reserve(take.count(), nP);
    write_row_bits(take, nn, vb, P, pp);
  }
}

// One round's independent set and its moves (see k_coarsen_select_apply).
__device__ __forceinline__ void smooth_select_apply_phase(Store S, const int* C, const int* nCp,
                                                          const int* cmark, int* smark, int tag,
                                                          int* Dn, int* nDn, int* dmark,
                                                          const double2* mvxy, const double4* mvM,
                                                          const double* qball, int* P, int* nP,
                                                          int* pmark, int ptag, int stamp,
                                                          bool il = false) {
  const int n = *nCp;
  for (int i0 = 0; i0 < n; i0 += gsize()) {
    int i = i0 + grank(il);
    bool win = false, lose = false;
    int v = 0;
    if (i < n) {
      v = C[i];
      win = local_max(S, v, cmark, tag);
      if (win) smark[v] = tag;
      else lose = stamp_first(dmark, v, tag);
    }
    warp_append(lose, v, Dn, nDn);
    smooth_apply_one(S, win, v, mvxy, mvM, qball, P, nP, pmark, ptag, stamp);
  }
}

__global__ void k_smooth_select_apply(Store S, const int* C, const int* nCp, const int* cmark,
                                      int* smark, int tag, int* Dn, int* nDn, int* dmark,
                                      const double2* mvxy, const double4* mvM, const double* qball,
                                      int* P, int* nP, int* pmark, int ptag, int stamp,
                                      unsigned* done) {
  smooth_select_apply_phase(S, C, nCp, cmark, smark, tag, Dn, nDn, dmark, mvxy, mvM, qball, P, nP,
                            pmark, ptag, stamp);
  round_done(S, done);
}

// Optimisation-based smoothing of one member of S (gradient ascent of the
// ball's quality sum in v's coordinates, metric fixed; step 0.1 * shortest
// incident edge / |g|, halved up to five times; kept when every element stays
// counter-clockwise, the minimum quality does not drop and the sum rises),
// evaluated by an 8-lane tile.
__device__ bool tile_opt_eval(const Tile& t, const Store& S, int v, MeshCtx c, double2& Xo,
                              double4& Mo, double* qout) {
  uint8_t f = S.vflag[v];
  if (!(f & VF_ALIVE) || (f & VF_BND)) return false;
  int lv = v - c.vb;
  const int* ne = ne_row(S, v);
  int nel = S.NElen[v];
  double gx = 0.0, gy = 0.0;
  for (int base = 0; base < nel; base += TW) {
    int k = base + t.tl;
    double gxk = 0.0, gyk = 0.0;
    if (k < nel) {
      int4 e = S.EN[c.eb + ne[k]];
      double g[3][5];
      quality_grad_c(e.x, e.y, e.z, load_vd(S, c.vb + e.x), load_vd(S, c.vb + e.y),
                     load_vd(S, c.vb + e.z), g);
      int i = (e.x == lv) ? 0 : (e.y == lv) ? 1 : 2;
      gxk = g[i][0];
      gyk = g[i][1];
    }
    int cnt = min(TW, nel - base);
    for (int j = 0; j < cnt; ++j) {
      gx = gx + tshfl(t, gxk, j);
      gy = gy + tshfl(t, gyk, j);
    }
  }
  double gn = sqrt(gx * gx + gy * gy);
  if (!(gn > 0.0)) return false;
  const int* nn = nn_row(S, v);
  int nnl = S.NNlen[v];
  double2 pv = S.xy[v];
  double lmin = 1e300;
  for (int k = t.tl; k < nnl; k += TW) {
    double2 pj = S.xy[c.vb + nn[k]];
    double dx = pj.x - pv.x;
    double dy = pj.y - pv.y;
    double l = sqrt(dx * dx + dy * dy);
    lmin = (l < lmin) ? l : lmin;
  }
  lmin = tmin(t, lmin);
  double qsum_old;
  double qmin_old = tile_ball_quality(t, S, c, ne, nel, &qsum_old);
  double alpha = (0.1 * lmin) / gn;
  for (int k = 0; k < 6; ++k) {
    double X = pv.x + alpha * gx;
    double Y = pv.y + alpha * gy;
    double4 Mn;
    if (tile_interpolate(t, S, c, ne, nel, X, Y, Mn)) {
      double qsum;
      if (tile_ball_after_move(t, S, c, lv, ne, nel, X, Y, Mn, qmin_old, false, qout, &qsum) &&
          qsum > qsum_old) {
        Xo = make_double2(X, Y);
        Mo = Mn;
        return true;
      }
    }
    alpha = alpha * 0.5;
  }
  return false;
}

// Evaluate and apply in one pass (one tile per member of S): members are
// pairwise non-adjacent, so no member reads a vertex another member moves.
__global__ void k_opt_apply(Store S, const int* Sl, const int* nSp, double* qball, int stamp) {
  advance_rounds(S);
  const int n = *nSp;
  const Tile t = tile_of();
  const int tiles_per_block = blockDim.x / TW;
  for (int j0 = blockIdx.x * tiles_per_block; j0 < n; j0 += gridDim.x * tiles_per_block) {
    int j = j0 + threadIdx.x / TW;
    bool moved = false;
    int mi = 0;
    if (j < n) {
      int v = Sl[j];
      MeshCtx c = ctx_of(S, v);
      mi = c.mi;
      double* qb = qball + (size_t)v * S.W;
      double2 X;
      double4 Mv;
      moved = tile_opt_eval(t, S, v, c, X, Mv, qb);
      __syncwarp(t.mask);
      if (moved && t.tl == 0) {
        S.xy[v] = X;
        S.M[v] = Mv;
        S.touch[v] = stamp;
        const int* ne = ne_row(S, v);
        int nel = S.NElen[v];
        for (int k = 0; k < nel; ++k) S.qK[c.eb + ne[k]] = qb[k];
        stamp_neighbours(S, nn_row(S, v), S.NNlen[v], c.vb, stamp);
      }
    }
    count_op(S, moved && t.tl == 0, mi);
  }
}

// Every listed vertex is a candidate of this round.
__global__ void k_stamp_list(Store S, const int* L, const int* nLp, int* cmark, int tag) {
  const int n = *nLp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int v = L[i];
    cmark[v] = tag;
    S.tab.had[mesh_of_vslot(S, v)] = 1;
  }
}

// ---- refinement (Sec. 2.4.2) -----------------------------------------------------

// Mark edges (a, b), a < b, longer than L_up: entry k of vmask[a] for NN entry k.
// A vertex unchanged since it was marked earlier in this pass keeps its mask;
// one unchanged since the end of an earlier complete pass has none.  The mask
// reads a's own row and the positions and metrics of a and its neighbours;
// inside one call vertices keep their positions and metrics until the
// operator loop ends (smoothing runs after it), so a's own stamp tells
// whether anything the mask read has changed: every change of a's row stamps a.
__global__ void k_refine_mark(Store S, int* cnt, RowMask* mask, int tag, int pass0, int lo) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    int mi = mesh_of_vslot(S, s);
    int vb = S.tab.vbase[mi];
    RowMask m;
    bool live = s - vb < S.tab.nv[mi] && S.tab.active[mi] && (S.vflag[s] & VF_ALIVE);
    const int et = live ? S.evr[s] : 0;
    const bool same = live && S.touch[s] <= et;
    if (same && et > pass0) {
      m = mask[s];  // kept as it is
    } else if (same && et > lo) {
      mask[s] = RowMask();
    } else if (live) {
      S.evr[s] = tag;
      int la = s - vb;
      const int* nn = nn_row(S, s);
      int nnl = S.NNlen[s];
      VD da = load_vd(S, s);
      const double L_up = S.tab.L_up[mi];
      const double4 band = S.tab.band[mi];
      // the row is sorted, so the neighbours above la form a suffix; four
      // lengths at a time so that their loads overlap
      int k0 = 0;
      while (k0 < nnl && nn[k0] <= la) ++k0;
#pragma unroll 4
      for (int k = k0; k < nnl; ++k)
        if (len_gt(metric_len2(da, load_vd(S, vb + nn[k])), band.z, band.w, L_up)) m.set(k);
      mask[s] = m;
    } else {
      mask[s] = RowMask();
    }
    cnt[s] = m.count();
  }
}

// Per-mesh number of new vertices (edges to split).
__global__ void k_refine_newcount(Store S, const int* vscan, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nmesh) return;
  int vb = S.tab.vbase[i];
  out[i] = vscan[vb + S.tab.nv[i]] - vscan[vb];
}

// A mesh that splits edges counts the round and its splits.
__global__ void k_refine_vtotals(Store S, const int* vscan) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nmesh) return;
  int vb = S.tab.vbase[i];
  int t = vscan[vb + S.tab.nv[i]] - vscan[vb];
  if (t > 0) {
    S.tab.r[i] += 1;
    S.tab.ops[i] += (unsigned long long)t;
  }
}

__device__ __forceinline__ int mid_id(const Store& S, int vb, int nv, const int* vscan,
                                      const RowMask* mask, int p, int q) {
  int a = p < q ? p : q, b = p < q ? q : p;
  const RowMask m = mask[vb + a];
  if (!m.any()) return -1;
  int k = row_find(nn_row(S, vb + a), S.NNlen[vb + a], b);
  if (k < 0 || !m.test(k)) return -1;
  int rank = m.below(k);
  return nv + (vscan[vb + a] - vscan[vb]) + rank;
}

__global__ void k_refine_newverts(Store S, const int* vscan, const RowMask* mask, int stamp,
                                  int4* owner) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    RowMask m = mask[s];
    if (!m.any()) continue;
    int mi = mesh_of_vslot(S, s);
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi], nv = S.tab.nv[mi];
    const int* nn = nn_row(S, s);
    const int* ne = ne_row(S, s);
    int nel = S.NElen[s];
    int base = nv + (vscan[s] - vscan[vb]);
    int rank = 0;
    VD da = load_vd(S, s);
    while (m.any()) {
      int b = nn[m.pop()];
      VD db = load_vd(S, vb + b);
      int slot = vb + base + rank;
      ++rank;
      S.xy[slot] = make_double2(0.5 * (da.x + db.x), 0.5 * (da.y + db.y));
      S.M[slot] = make_double4(0.5 * (da.m00 + db.m00), 0.5 * (da.m01 + db.m01),
                               0.5 * (da.m11 + db.m11), 0.0);
      bool bedge = count_elems_with(S, ne, nel, eb, b) == 1;
      S.vflag[slot] = (uint8_t)(VF_ALIVE | (bedge ? VF_BND : 0));
      if (S.lid) S.lid[slot] = (slot - vb) - S.voff[mi];
      S.touch[slot] = stamp;
      S.evc[slot] = S.evs[slot] = S.evm[slot] = S.evr[slot] = 0;
      owner[slot] = make_int4(s - vb, b, 0, 0);  // the split edge (a, b)
    }
  }
}

// Extra children per live element (0..3); an element that splits gets the
// midpoint ids of its edges and joins the split list.
__global__ void k_refine_count(Store S, const int* vscan, const RowMask* mask, int* ecnt,
                               int4* emid, int* elist, int* nel) {
  for (int i0 = blockIdx.x * blockDim.x; i0 < S.eused; i0 += gridDim.x * blockDim.x) {
    int s = i0 + threadIdx.x;
    int extra = 0;
    if (s < S.eused) {
      int mi = mesh_of_eslot(S, s);
      int eb = S.tab.ebase[mi];
      if (s - eb < S.tab.ne[mi] && S.tab.active[mi]) {
        int4 e = S.EN[s];
        if (e.w) {
          int vb = S.tab.vbase[mi], nv = S.tab.nv[mi];
          int m0 = mid_id(S, vb, nv, vscan, mask, e.x, e.y);
          int m1 = mid_id(S, vb, nv, vscan, mask, e.y, e.z);
          int m2 = mid_id(S, vb, nv, vscan, mask, e.z, e.x);
          extra = (m0 >= 0) + (m1 >= 0) + (m2 >= 0);
          if (extra) emid[s] = make_int4(m0, m1, m2, extra);
        }
      }
      ecnt[s] = extra;
    }
    warp_append(extra > 0, s, elist, nel);
  }
}

// Templates: one split -> (a,m,o),(m,b,o); two splits -> (m0,u1,m1) plus the
// trapezoid (u0,m0,m1,u2) cut along its metric-shorter diagonal; three
// splits -> four children.  The first child keeps the parent's slot, the rest
// take ne + scan(extra children) in parent order.  Every child slot joins
// the list whose qualities k_refine_quality computes.
__global__ void k_refine_split(Store S, const int* escan, const int4* emid, const int* elist,
                               const int* nelp, int* clist, int* ncl, int stamp) {
  const int n = *nelp;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    int i = i0 + threadIdx.x;
    int s = 0, nslot = 0, extra = 0;
    if (i < n) {
      s = elist[i];
      int mi = mesh_of_eslot(S, s);
      int eb = S.tab.ebase[mi];
      int4 e = S.EN[s];
      int4 md = emid[s];
      extra = md.w;
      int vb = S.tab.vbase[mi];
      nslot = eb + S.tab.ne[mi] + (escan[s] - escan[eb]);
      auto put = [&](int slot, int a, int b, int c) { S.EN[slot] = make_int4(a, b, c, 1); };
      int t[3] = {e.x, e.y, e.z};
      int mm[3] = {md.x, md.y, md.z};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        S.touch[vb + t[k]] = stamp;
        if (mm[k] >= 0) S.touch[vb + mm[k]] = stamp;
      }
      if (md.w == 1) {
        int j = (mm[0] >= 0) ? 0 : (mm[1] >= 0) ? 1 : 2;
        int a = t[j], b = t[(j + 1) % 3], o = t[(j + 2) % 3], m = mm[j];
        put(s, a, m, o);
        put(nslot, m, b, o);
      } else if (md.w == 2) {
        int j = (mm[0] < 0) ? 0 : (mm[1] < 0) ? 1 : 2;
        int q = (j + 1) % 3;
        int u0 = t[q], u1 = t[(q + 1) % 3], u2 = t[(q + 2) % 3];
        int m0 = mm[q], m1 = mm[(q + 1) % 3];
        put(s, m0, u1, m1);
        double d1 = metric_len(load_vd(S, vb + u0), load_vd(S, vb + m1));
        double d2 = metric_len(load_vd(S, vb + m0), load_vd(S, vb + u2));
        if (!dgt(d1, d2)) {
          put(nslot, u0, m0, m1);
          put(nslot + 1, u0, m1, u2);
        } else {
          put(nslot, u0, m0, u2);
          put(nslot + 1, m0, m1, u2);
        }
      } else {
        put(s, t[0], mm[0], mm[2]);
        put(nslot, mm[0], t[1], mm[1]);
        put(nslot + 1, mm[2], mm[1], t[2]);
        put(nslot + 2, mm[0], mm[1], mm[2]);
      }
    }
    warp_append(i < n, s, clist, ncl);
    for (int j = 0; j < 3; ++j) warp_append(j < extra, nslot + j, clist, ncl);
  }
}

// Cached quality of every listed element slot (one element per thread): the
// children of a refinement round, the elements a collapse round changed.
__global__ void k_refine_quality(Store S, const int* clist, const int* nclp,
                                 unsigned long long* work) {
  elem_quality_phase(S, clist, nclp, work);
}

// Children of parent element K (local id) of this round: K itself and, when
// split, the extra slots ne + (escan[K] - escan[eb]) onwards.
__device__ __forceinline__ int refine_children(const Store& S, int mi, int eb, const int* escan,
                                               int K, int* out) {
  int s = eb + K;
  int e0 = escan[s], extra = escan[s + 1] - e0;
  out[0] = K;
  int first = S.tab.ne[mi] + (e0 - escan[eb]);
  for (int j = 0; j < extra; ++j) out[1 + j] = first + j;
  return 1 + extra;
}

// New rows of every vertex whose elements changed in this refinement round
// (stamped), written to the spare buffer B: NE = the children of its old
// elements that contain it (a new vertex: the children of the elements of its
// split edge), NN = the other vertices of those, both sorted.
__global__ void k_refine_rows(Store S, Store B, int vend, const int* vscan, const int* escan,
                              const int4* owner, int stamp, DevStatus* st) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < vend; s += gridDim.x * blockDim.x) {
    if (S.touch[s] != stamp) continue;
    int mi = mesh_of_vslot(S, s);
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi], nv = S.tab.nv[mi];
    int lu = s - vb;
    // the old element row holding the parents: v's own, or for a new vertex
    // that of its split edge's first end (the children that contain the new
    // vertex are exactly those of the two parents on that edge)
    int src = (lu < nv) ? s : vb + owner[s].x;
    const int* ne = S.NE + (size_t)src * S.W;
    int nel = S.NElen[src];
    int eb_[MAXW], nb_[MAXW];
    int ne2 = 0, nn2 = 0;
    bool ok = true;
    for (int k = 0; k < nel; ++k) {
      int K = ne[k];
      int ch[4];
      int n = refine_children(S, mi, eb, escan, K, ch);
      for (int j = 0; j < n; ++j) {
        int4 e = S.EN[eb + ch[j]];
        if (e.x != lu && e.y != lu && e.z != lu) continue;
        ok &= sorted_insert(eb_, ne2, MAXW, ch[j]);
        int a = (e.x == lu) ? e.y : e.x;
        int b = (e.z == lu) ? e.y : e.z;
        ok &= sorted_insert(nb_, nn2, MAXW, a);
        ok &= sorted_insert(nb_, nn2, MAXW, b);
      }
    }
    if (!ok || ne2 > S.W || nn2 > S.W) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->maxdeg, max(ne2, nn2));
      continue;
    }
    int* wn = B.NN + (size_t)s * B.W;
    int* we = B.NE + (size_t)s * B.W;
    for (int k = 0; k < nn2; ++k) wn[k] = nb_[k];
    for (int k = 0; k < ne2; ++k) we[k] = eb_[k];
    B.NNlen[s] = nn2;
    B.NElen[s] = ne2;
  }
}

__global__ void k_refine_rows_copy(Store S, Store B, int vend, int stamp) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < vend; s += gridDim.x * blockDim.x) {
    if (S.touch[s] != stamp) continue;
    int a = B.NNlen[s], b = B.NElen[s];
    const int* nn = B.NN + (size_t)s * B.W;
    for (int k = 0; k < a; ++k) S.NN[(size_t)s * S.W + k] = nn[k];
    for (int k = 0; k < b; ++k) S.NE[(size_t)s * S.W + k] = B.NE[(size_t)s * B.W + k];
    S.NNlen[s] = a;
    S.NElen[s] = b;
    stamp_neighbours(S, nn, a, S.tab.vbase[mesh_of_vslot(S, s)], stamp);
  }
}

__global__ void k_refine_sizes(Store S, const int* vscan, const int* escan) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nmesh) return;
  int vb = S.tab.vbase[i], eb = S.tab.ebase[i];
  int nv = S.tab.nv[i], ne = S.tab.ne[i];
  S.tab.nv[i] = nv + (vscan[vb + nv] - vscan[vb]);
  S.tab.ne[i] = ne + (escan[eb + ne] - escan[eb]);
}

// ---- persistent rounds ------------------------------------------------------------
//
// Once a pass's dirty list is small, a round does little work and its cost is
// launch and synchronisation latency.  Such rounds run back to back inside one
// cooperative launch (every block resident), with a grid-wide barrier between
// the phases and one read-back when the launch ends.  A collapse round
// evaluates in one phase (coarsen_eval_phase) and takes three barriers;
// smoothing scans and evaluates in one tile-parallel phase when the list fits
// one pass of tiles (two barriers), else keeps the scan apart (three); flips
// scan, evaluate and pick in one tile-parallel phase when the list fits one
// pass of tiles (three barriers), else keep their scan, item-parallel gains
// and pick (five).  The launch
// returns when a round finds no candidate (the pass is complete), when the
// next round's list outgrows `limit`, on a row overflow or an error, or after
// `max_rounds` rounds.
//
// Counters are reset where no block can still read or write them: the
// candidate count alternates between two slots (C of even rounds, C2 of odd
// ones); the other slot and the lists a round fills are cleared by block 0
// at least one barrier before their first use and after their last read.

constexpr unsigned long long kBarrierNs = 2000000000ull;  // a barrier wait gives up after 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

// Grid-wide barrier on a counter of arrivals that only grows (zeroed before
// the launch): the k-th barrier waits for k * gridDim.x arrivals.  Thread 0
// of each block publishes the block's writes (__syncthreads, then a
// device-wide fence), arrives, waits, and fences again before the block
// reads what the other blocks wrote.  Returns false (the caller leaves the
// kernel) when the wait ran out (PM_ERR_TIMEOUT is recorded) or when any
// phase recorded an error.
__device__ bool grid_barrier(unsigned* bar, unsigned& target, DevStatus* st,
                             unsigned long long limit_ns = kBarrierNs) {
  __shared__ int s_ok;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if ((int)(arrived - target) < 0) {
      const volatile unsigned* vb = bar;
      const unsigned long long t0 = global_ns();
      while ((int)(*vb - target) < 0) {
        if (ld_volatile(&st->err) != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > limit_ns) {
          set_err(st, PM_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && ld_volatile(&st->err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Test support: every block waits at a barrier whose target lies one arrival
// beyond the grid, so the wait can only end by its time limit.
__global__ void k_selftest_barrier(unsigned* bar, DevStatus* st, unsigned long long limit_ns) {
  unsigned target = 1;
  grid_barrier(bar, target, st, limit_ns);
}

struct RoundArgs {
  Store S;
  Work w;
  DevStatus* st;
  unsigned* bar;       // barrier arrivals (zeroed before the launch)
  int* res;            // out: rounds run, list index after, pass complete
  int cur;             // list index the first round reads
  int tag0;            // tag of the first round (then +2 per round)
  int pass0;
  int max_rounds;
  int limit;           // leave when the next list holds more entries
  int icap;            // flips: capacity of the item list
  int ptag;            // smoothing: stamp of the next sweep's list
  int fuse;            // flips, smoothing: lists up to this size take the one-phase evaluation
  unsigned long long* work;  // counted FP64 work (measurement) or null
};

__device__ __forceinline__ int* cand_count(int* cnt, int r) {
  return cnt + ((r & 1) ? CN_C2 : CN_C);
}

__device__ __forceinline__ void finish_rounds(const RoundArgs& a, int r, int cur, bool complete) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.res[0] = r;
    a.res[1] = cur;
    a.res[2] = complete ? 1 : 0;
  }
}

// Rounds of collapses: [evaluate] B1 [select + apply] B2 [commit] B3; rounds
// of flips whose list fits one pass of the grid's tiles: [scan + gains +
// pick] B1 [select + apply] B2 [commit] B3; longer flip lists: [scan] B1
// [gains] [pick] [select + apply] [commit], five barriers.  Block 0 clears,
// before B1 of round r: A and the list round r
// fills (both last read before the last barrier of round r - 1); right after
// B1: the candidate slot of round r + 1 (last read before the last barrier of
// round r - 1); flips, after the pick: E and the item count (read by the pick
// and the gains).
template <bool FLIP>
__device__ __forceinline__ void topo_rounds(const RoundArgs& a) {
  const Work& w = a.w;
  int* cnt = w.counts;
  unsigned target = 0;
  int cur = a.cur, r = 0;
  bool complete = false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cand_count(cnt, 0) = 0;
    cnt[CN_E] = cnt[CN_I] = 0;
  }
  if (!grid_barrier(a.bar, target, a.st)) return;
  // a first list longer than the limit is left to the one-kernel-per-phase rounds
  const bool too_long = ld_volatile(cnt + cn_list(cur)) > a.limit;
  while (!too_long && r < a.max_rounds) {
    const int tag = a.tag0 + 2 * r, nxt = 1 - cur;
    int* nC = cand_count(cnt, r);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      cnt[CN_A] = 0;
      cnt[cn_list(nxt)] = 0;
      cnt[CN_CL] = 0;  // elements whose quality changes
    }
    if (FLIP && ld_volatile(cnt + cn_list(cur)) <= min(a.fuse, tcount())) {
      // the list fits one pass of tiles: scan, gains and pick in one phase
      // (the list is complete since the last barrier: every block decides alike)
      swap_scan_eval_phase(a.S, w.D[cur], cnt + cn_list(cur), w.opA, w.opK2, w.C, nC, w.cmark,
                           tag, a.pass0, a.work);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) *cand_count(cnt, r + 1) = 0;
    } else if (FLIP) {
      // a longer list keeps the three passes: item-parallel FP64 gains beat
      // two barriers saved
      swap_scan_phase(a.S, w.D[cur], cnt + cn_list(cur), w.opA, w.C, nC, w.cmark, tag, a.pass0,
                      w.E, cnt + CN_E, w.items, cnt + CN_I, a.icap, w.gains, a.st, true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) *cand_count(cnt, r + 1) = 0;
      swap_edge_phase(a.S, w.items, cnt + CN_I, w.gains, tag, a.work, true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      swap_pick_phase(a.S, w.E, cnt + CN_E, w.gains, w.opA, w.opK2, w.C, nC, w.cmark, tag, true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) cnt[CN_E] = cnt[CN_I] = 0;
    } else {
      coarsen_eval_phase(a.S, w.D[cur], cnt + cn_list(cur), w.target, w.cand, w.ncand, w.C, nC,
                         w.cmark, tag, a.pass0, a.work, true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) *cand_count(cnt, r + 1) = 0;
    }
    if (FLIP)
      swap_select_apply_phase(a.S, w.C, nC, w.cmark, w.smark, tag, w.opA, w.opK2, w.A,
                              cnt + CN_A, w.amark, w.D[nxt], cnt + cn_list(nxt), w.dmark, w.clist,
                              cnt + CN_CL, true);
    else
      coarsen_select_apply_phase(a.S, w.C, nC, w.cmark, w.smark, tag, w.target, w.A, cnt + CN_A,
                                 w.amark, w.D[nxt], cnt + cn_list(nxt), w.dmark, w.clist,
                                 cnt + CN_CL, true);
    if (!grid_barrier(a.bar, target, a.st)) return;
    const int nc = ld_volatile(nC), nd = ld_volatile(cnt + cn_list(nxt));
    advance_rounds(a.S);
    if (FLIP)
      swap_commit_phase(a.S, w.A, cnt + CN_A, w.opA, w.opK2, w.smark, tag, a.st, true);
    else
      coarsen_commit_phase(a.S, w.A, cnt + CN_A, w.target, w.smark, tag, a.st, true);
    elem_quality_phase(a.S, w.clist, cnt + CN_CL, a.work, true);
    if (!grid_barrier(a.bar, target, a.st)) return;
    ++r;
    if (nc == 0) {
      complete = true;
      break;
    }
    cur = nxt;
    if (ld_volatile(&a.st->overflow) != 0 || nd > a.limit) break;
  }
  // the host reads the candidates of the last round from the C slot
  if (blockIdx.x == 0 && threadIdx.x == 0 && r > 0)
    cnt[CN_C] = ld_volatile(cand_count(cnt, r - 1));
  finish_rounds(a, r, cur, complete);
}

__global__ void __launch_bounds__(256) k_coarsen_rounds(RoundArgs a) { topo_rounds<false>(a); }

__global__ void __launch_bounds__(256) k_swap_rounds(RoundArgs a) { topo_rounds<true>(a); }

// Rounds of smoothing moves.  A round whose list fits one pass of the grid's
// tiles: [scan + evaluate] B1 [select + apply] B2; a longer one: [scan] B1
// [evaluate] B1' [select + apply] B2 (its tiles then go to the vertices that
// need an evaluation only).  Block 0 clears, before B1 of round r: the list
// round r fills (last read by round r - 1's scan and by its decision, both
// before B1 of round r); after B1: the candidate slot of round r + 1 (last
// read after B2 of round r - 1); after B1': E (read by the evaluation before
// B1').  The round counters advance after B2 from the flag set of the round's
// parity, so that round r + 1's evaluation can set the other set meanwhile.
__global__ void __launch_bounds__(256) k_smooth_rounds(RoundArgs a) {
  const Work& w = a.w;
  int* cnt = w.counts;
  unsigned target = 0;
  int cur = a.cur, r = 0;
  bool complete = false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cand_count(cnt, 0) = 0;
    cnt[CN_E] = 0;
  }
  if (!grid_barrier(a.bar, target, a.st)) return;
  // a first list longer than the limit is left to the one-kernel-per-phase rounds
  const bool too_long = ld_volatile(cnt + cn_list(cur)) > a.limit;
  const int tiles = gridDim.x * (blockDim.x / TW);
  while (!too_long && r < a.max_rounds) {
    const int tag = a.tag0 + 2 * r, nxt = 1 - cur;
    int* nC = cand_count(cnt, r);
    Store S = a.S;
    S.tab.had = a.S.tab.had + (r & 1) * S.nmesh;
    // the list is complete since B2 of the last round: every block decides alike
    const bool fused = ld_volatile(cnt + cn_list(cur)) <= min(a.fuse, tiles);
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[cn_list(nxt)] = 0;
    if (fused) {
      smooth_scan_eval_phase(S, w.D[cur], cnt + cn_list(cur), w.mvxy, w.mvM, w.gains, w.C, nC,
                             w.cmark, tag, a.pass0, a.work);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) *cand_count(cnt, r + 1) = 0;
    } else {
      smooth_scan_phase(S, w.D[cur], cnt + cn_list(cur), w.mvM, w.C, nC, w.cmark, tag, a.pass0,
                        w.E, cnt + CN_E, true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) *cand_count(cnt, r + 1) = 0;
      smooth_eval_phase(S, w.E, cnt + CN_E, w.mvxy, w.mvM, w.gains, w.C, nC, w.cmark, tag, a.work,
                        true);
      if (!grid_barrier(a.bar, target, a.st)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) cnt[CN_E] = 0;
    }
    smooth_select_apply_phase(S, w.C, nC, w.cmark, w.smark, tag, w.D[nxt], cnt + cn_list(nxt),
                              w.dmark, w.mvxy, w.mvM, w.gains, w.P, cnt + CN_P, w.pmark, a.ptag,
                              tag + 1, true);
    if (!grid_barrier(a.bar, target, a.st)) return;
    const int nc = ld_volatile(nC), nd = ld_volatile(cnt + cn_list(nxt));
    advance_rounds(S);
    ++r;
    if (nc == 0) {
      complete = true;
      break;
    }
    cur = nxt;
    if (nd > a.limit) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && r > 0)
    cnt[CN_C] = ld_volatile(cand_count(cnt, r - 1));
  finish_rounds(a, r, cur, complete);
}

// ---- host helpers --------------------------------------------------------------

struct RoundIO {
  int nC;
  int overflow;
  int err;
};

RoundIO read_round(MeshSet& m) {
  cudaMemcpyAsync(m.hcounts, m.w.counts, CN_NUM * sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(m.hst, m.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, m.stream);
  cudaError_t e = cudaStreamSynchronize(m.stream);
  RoundIO io;
  io.nC = m.hcounts[CN_C];
  io.overflow = m.hst->overflow;
  io.err = (e != cudaSuccess) ? PM_ERR_CUDA : m.hst->err;
  if (e != cudaSuccess) set_last_error(std::string("CUDA: ") + cudaGetErrorString(e));
  return io;
}

void zero_counts(MeshSet& m, int first, int num) {
  cudaMemsetAsync(m.w.counts + first, 0, num * sizeof(int), m.stream);
}

// Colours every active mesh whose parameters ask for colour-class sets, at
// the start of a collapse, flip or smoothing pass: speculative rounds until
// no vertex is left uncoloured (each round keeps at least the proposal of
// the highest priority; the cap is far beyond any mesh's rounds).
int colour_set(MeshSet& m) {
  bool any = false;
  for (int x : m.select) any |= x == PM_SELECT_COLOUR;
  if (!any) return PM_OK;
  Work& w = m.w;
  const int g = grid_for(m, m.S.vused);
  zero_counts(m, CN_D0, 1);
  PM_LAUNCH(k_colour_init, g, BLOCK, 0, m.stream, m.S, w.D[0], w.counts + CN_D0);
  int cur = 0;
  for (int it = 0; it < (1 << 20); ++it) {
    const int nxt = 1 - cur;
    const int rt = (m.tag += 2);
    zero_counts(m, cn_list(nxt), 1);
    PM_LAUNCH(k_colour_propose, g, BLOCK, 0, m.stream, m.S, w.D[cur], w.counts + cn_list(cur),
              w.cprop, w.cstamp, rt);
    PM_LAUNCH(k_colour_resolve, g, BLOCK, 0, m.stream, m.S, w.D[cur], w.counts + cn_list(cur),
              w.cprop, w.cstamp, rt, w.D[nxt], w.counts + cn_list(nxt));
    RoundIO io = read_round(m);
    if (io.err) return io.err;
    if (m.hcounts[cn_list(nxt)] == 0) return PM_OK;
    cur = nxt;
  }
  set_last_error("colouring did not finish");
  return PM_ERR_INVALID_MESH;
}

// The counters of a new round (C, S, A, E, I, I2) and of the list it fills
// (D[nxt]); the list it reads keeps its count.
void zero_round(MeshSet& m, int nxt) {
  static_assert(CN_D0 == 0 && CN_C == 1 && CN_I2 == 6 && CN_D1 == 7, "counter layout");
  zero_counts(m, nxt == 0 ? CN_D0 : CN_C, 7);
}

// A row overflow leaves some rows unwritten and the neighbour stamps of the
// rebuilt rows unset: rows are rebuilt from the elements and no evaluation
// made before is reused (every lo_* and the callers' pass start move to now).
int after_overflow(MeshSet& m) {
  int err = rebuild_adjacency(m, false, false);
  m.lo_coarsen = m.lo_swap = m.lo_refine = m.tag;
  return err;
}

int after_round(MeshSet& m, const RoundIO& io) {
  if (io.err) return io.err;
  if (io.overflow) return after_overflow(m);
  return PM_OK;
}

// Persistent rounds take over once a pass's list holds at most
// Tuning::rounds_limit vertices (and hand back when the next list outgrows
// it); default 131072 for each operator, measured best of 8k to 1M on the
// 2M workload.
constexpr int kRoundsThreads = 256;

// Blocks of a cooperative launch of the persistent round kernel `which`
// (0 collapse, 1 flip, 2 smoothing) on this device: the tuning's blocks per
// SM (Tuning::rounds_blocks_per_sm, at most what its registers allow) on
// every SM, or 0 when the device cannot run it cooperatively (rounds stay one
// kernel per phase).
int rounds_grid(MeshSet& m, int which) {
  static std::mutex mu;
  static int occ[64][3];
  static bool known[64];
  const int dev = m.device;
  if (dev < 0 || dev >= 64 || which < 0 || which > 2) return 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!known[dev]) {
      int coop = 0;
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
      const void* ks[] = {(const void*)k_coarsen_rounds, (const void*)k_swap_rounds,
                          (const void*)k_smooth_rounds};
      for (int k = 0; k < 3; ++k) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ks[k], kRoundsThreads, 0) !=
            cudaSuccess)
          b = 0;
        occ[dev][k] = coop ? b : 0;
      }
      cudaGetLastError();
      known[dev] = true;
    }
  }
  const int b = std::min(occ[dev][which], tuning().rounds_blocks_per_sm[which]);
  return b >= 1 ? m.num_sms * b : 0;
}

RoundArgs round_args(MeshSet& m, int cur, int pass0, long long max_rounds) {
  RoundArgs a;
  a.S = m.S;
  a.w = m.w;
  a.st = m.st;
  a.bar = (unsigned*)(m.w.counts + CN_BAR);
  a.res = m.w.counts + CN_RES;
  a.cur = cur;
  a.tag0 = m.tag + 2;
  a.pass0 = pass0;
  a.max_rounds = (int)std::min<long long>(max_rounds, 1 << 30);
  a.limit = tuning().rounds_limit[0];
  a.icap = 0;
  a.ptag = 0;
  a.fuse = 0;
  a.work = nullptr;
  return a;
}

struct RoundsOut {
  int rounds = 0;    // rounds run, the last one empty when the pass completed
  int cur = 0;       // list the next round reads
  int complete = 0;
  RoundIO io{0, 0, 0};
};

// One cooperative launch of persistent rounds, then the read-back of every
// counter and the status.  Advances the tag past the rounds that ran.
int run_rounds(MeshSet& m, int which, const void* kernel, const char* name, RoundArgs& a,
               RoundsOut& out) {
  a.work = prof_work(name);
  void* args[] = {&a};
  cudaMemsetAsync(a.bar, 0, sizeof(unsigned), m.stream);
  __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED);
  int slot = g_prof_on ? prof_begin(name, m.stream) : -1;
  cudaError_t e = cudaLaunchCooperativeKernel(kernel, dim3(rounds_grid(m, which)),
                                              dim3(kRoundsThreads), args, 0, m.stream);
  if (slot >= 0) prof_end(slot, m.stream);
  if (e != cudaSuccess) {
    set_last_error(std::string("cooperative launch: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  out.io = read_round(m);
  if (out.io.err) return out.io.err;
  out.rounds = m.hcounts[CN_RES];
  out.cur = m.hcounts[CN_RES + 1];
  out.complete = m.hcounts[CN_RES + 2];
  m.tag += 2 * out.rounds;
  return PM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Operator loops (host)
// ---------------------------------------------------------------------------

void zero_ops(MeshSet& m) {
  cudaMemsetAsync(m.S.tab.ops, 0, m.nmesh * sizeof(unsigned long long), m.stream);
}

cudaError_t fetch_ops(MeshSet& m, std::vector<unsigned long long>& ops) {
  ops.resize(m.nmesh);
  cudaError_t e = cudaMemcpyAsync(ops.data(), m.S.tab.ops, m.nmesh * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, m.stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(m.stream);
}

// Rounds of collapses until no dirty vertex has a valid collapse.  The first
// round's list leaves out vertices whose last collapse evaluation found
// nothing and whose inputs have not changed since.
int op_coarsen(MeshSet& m, int max_rounds) {
  if (int err = colour_set(m)) return err;
  const Tuning tu = tuning();
  const int bs = tu.block[TO_COARSEN], bps = tu.blocks_per_sm[TO_COARSEN];
  const int rlimit = tu.rounds_limit[0];
  Work& w = m.w;
  const int gv = grid_tuned(m, m.S.vused, bs, bps);
  int pass0 = m.tag;
  const bool persist = rounds_grid(m, 0) > 0;
  zero_counts(m, 0, CN_NUM);
  PM_LAUNCH(k_init_list, gv, bs, 0, m.stream, m.S, 0, w.D[0], w.counts + CN_D0, m.S.evc,
            m.lo_coarsen);
  // entries of the list the next round reads; unknown (0) at first: the
  // persistent launch itself hands a long first list back
  int nlist = 0;
  int cur = 0;
  bool complete = false;
  for (long long nr = 0; max_rounds == 0 || nr < max_rounds;) {
    if (m.lo_coarsen > pass0) pass0 = m.lo_coarsen;  // rows were rebuilt after an overflow
    if (persist && nlist >= 0 && nlist <= rlimit) {
      RoundArgs a = round_args(m, cur, pass0, max_rounds == 0 ? (1LL << 30) : max_rounds - nr);
      a.limit = rlimit;
      RoundsOut o;
      int err = run_rounds(m, 0, (const void*)k_coarsen_rounds, "k_coarsen_rounds", a, o);
      if (err) return err;
      nr += o.rounds - o.complete;
      cur = o.cur;
      if (o.complete) {
        complete = true;
        break;
      }
      if ((err = after_round(m, o.io))) return err;
      nlist = m.hcounts[cn_list(cur)];
      continue;
    }
    int tag = (m.tag += 2);
    int nxt = 1 - cur;
    zero_round(m, nxt);
    PM_LAUNCH(k_coarsen_scan, gv, bs, 0, m.stream, m.S, w.D[cur], w.counts + cn_list(cur),
              w.target, w.cand, w.ncand, w.C, w.counts + CN_C, w.cmark, tag, pass0, w.items,
              w.counts + CN_I, w.gains);
    // one dense wave checking every vertex's best candidate, then the
    // remaining candidates of the vertices whose best one failed
    PM_LAUNCH(k_coarsen_check, gv, bs, 0, m.stream, m.S, w.items, w.counts + CN_I, w.items2,
              w.counts + CN_I2, w.target, w.cand, w.ncand, w.C, w.counts + CN_C, w.cmark, tag, 0,
              prof_work("k_coarsen_check"));
    PM_LAUNCH(k_coarsen_check, gv, bs, 0, m.stream, m.S, w.items2, w.counts + CN_I2, w.items,
              w.counts + CN_I, w.target, w.cand, w.ncand, w.C, w.counts + CN_C, w.cmark, tag, 1,
              prof_work("k_coarsen_check"));
    zero_counts(m, CN_CL, 1);
    PM_LAUNCH(k_coarsen_select_apply, gv, bs, 0, m.stream, m.S, w.C, w.counts + CN_C, w.cmark,
              w.smark, tag, w.target, w.A, w.counts + CN_A, w.amark, w.D[nxt],
              w.counts + cn_list(nxt), w.dmark, w.clist, w.counts + CN_CL,
              (unsigned*)(w.counts + CN_DONE));
    PM_LAUNCH(k_coarsen_commit, gv, bs, 0, m.stream, m.S, w.A, w.counts + CN_A, w.target,
              w.smark, tag, m.st);
    PM_LAUNCH(k_refine_quality, gv, bs, 0, m.stream, m.S, w.clist, w.counts + CN_CL, nullptr);
    RoundIO io = read_round(m);
    if (io.err) return io.err;
    if (io.nC == 0) {
      complete = true;
      break;
    }
    int err = after_round(m, io);
    if (err) return err;
    cur = nxt;
    ++nr;
    nlist = m.hcounts[cn_list(cur)];
  }
  if (!complete) m.lo_coarsen = m.tag;  // some vertex may still have a collapse
  return PM_OK;
}

// Rounds of flips until no dirty vertex has an improving flip.
int op_swap(MeshSet& m, int max_rounds) {
  if (int err = colour_set(m)) return err;
  const Tuning tu = tuning();
  const int bs = tu.block[TO_SWAP], bps = tu.blocks_per_sm[TO_SWAP];
  const int rlimit = tu.rounds_limit[1];
  Work& w = m.w;
  const int gv = grid_tuned(m, m.S.vused, bs, bps);
  int pass0 = m.tag;
  const int icap = m.S.vslots * 6 + 64;
  const bool persist = rounds_grid(m, 1) > 0;
  zero_counts(m, 0, CN_NUM);
  PM_LAUNCH(k_init_list, gv, bs, 0, m.stream, m.S, 0, w.D[0], w.counts + CN_D0, m.S.evs,
            m.lo_swap);
  int nlist = 0;  // unknown at first (see op_coarsen)
  int cur = 0;
  bool complete = false;
  for (long long nr = 0; max_rounds == 0 || nr < max_rounds;) {
    if (m.lo_swap > pass0) pass0 = m.lo_swap;  // rows were rebuilt after an overflow
    if (persist && nlist >= 0 && nlist <= rlimit) {
      RoundArgs a = round_args(m, cur, pass0, max_rounds == 0 ? (1LL << 30) : max_rounds - nr);
      a.icap = icap;
      a.limit = rlimit;
      a.fuse = tu.fuse_limit[0];
      RoundsOut o;
      int err = run_rounds(m, 1, (const void*)k_swap_rounds, "k_swap_rounds", a, o);
      if (err) return err;
      nr += o.rounds - o.complete;
      cur = o.cur;
      if (o.complete) {
        complete = true;
        break;
      }
      if ((err = after_round(m, o.io))) return err;
      nlist = m.hcounts[cn_list(cur)];
      continue;
    }
    int tag = (m.tag += 2);
    int nxt = 1 - cur;
    zero_round(m, nxt);
    PM_LAUNCH(k_swap_scan, gv, bs, 0, m.stream, m.S, w.D[cur], w.counts + cn_list(cur), w.opA,
              w.C, w.counts + CN_C, w.cmark, tag, pass0, w.E, w.counts + CN_E, w.items,
              w.counts + CN_I, icap, w.gains, m.st);
    PM_LAUNCH(k_swap_edge, grid_tuned(m, 6LL * m.S.vslots, bs, bps), bs, 0, m.stream, m.S, w.items,
              w.counts + CN_I, w.gains, tag, prof_work("k_swap_edge"));
    PM_LAUNCH(k_swap_pick, gv, bs, 0, m.stream, m.S, w.E, w.counts + CN_E, w.gains, w.opA,
              w.opK2, w.C, w.counts + CN_C, w.cmark, tag);
    zero_counts(m, CN_CL, 1);
    PM_LAUNCH(k_swap_select_apply, gv, bs, 0, m.stream, m.S, w.C, w.counts + CN_C, w.cmark,
              w.smark, tag, w.opA, w.opK2, w.A, w.counts + CN_A, w.amark, w.D[nxt],
              w.counts + cn_list(nxt), w.dmark, w.clist, w.counts + CN_CL,
              (unsigned*)(w.counts + CN_DONE));
    PM_LAUNCH(k_swap_commit, gv, bs, 0, m.stream, m.S, w.A, w.counts + CN_A, w.opA, w.opK2,
              w.smark, tag, m.st);
    PM_LAUNCH(k_refine_quality, gv, bs, 0, m.stream, m.S, w.clist, w.counts + CN_CL, nullptr);
    RoundIO io = read_round(m);
    if (io.err) return io.err;
    if (io.nC == 0) {
      complete = true;
      break;
    }
    int err = after_round(m, io);
    if (err) return err;
    cur = nxt;
    ++nr;
    nlist = m.hcounts[cn_list(cur)];
  }
  if (!complete) m.lo_swap = m.tag;
  return PM_OK;
}

// Rounds of splits until no edge is longer than L_up.  Capacity is checked
// (and grown) before any new vertex or element is written.
int op_refine(MeshSet& m, int max_rounds) {
  const Tuning tu = tuning();
  const int bs = tu.block[TO_REFINE], bps = tu.blocks_per_sm[TO_REFINE];
  Work& w = m.w;
  int pass0 = m.tag;
  bool complete = false;
  for (long long nr = 0; max_rounds == 0 || nr < max_rounds; ++nr) {
    const int gv = grid_tuned(m, m.S.vused, bs, bps);
    const int ge = grid_tuned(m, m.S.eused, bs, bps);
    int tag = (m.tag += 2);
    if (m.lo_refine > pass0) pass0 = m.lo_refine;  // storage was regrown
    PM_LAUNCH(k_refine_mark, gv, bs, 0, m.stream, m.S, w.vcnt, w.vmask, tag, pass0,
              m.lo_refine);
    scan_exclusive(w.vcnt, w.vscan, m.S.vused, m.scan, m.st, m.stream);
    int* tot = w.counts + CN_NUM;
    std::vector<int> newv(m.nmesh);
    PM_LAUNCH(k_refine_newcount, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, w.vscan, tot);
    cudaMemcpyAsync(m.hcounts + CN_NUM, tot, m.nmesh * sizeof(int), cudaMemcpyDeviceToHost,
                    m.stream);
    {
      int err = sync_status(m);
      if (err) return err;
    }
    for (int i = 0; i < m.nmesh; ++i) newv[i] = m.hcounts[CN_NUM + i];
    // A growth moves every mesh of the set, so when one mesh needs room,
    // every mesh that is splitting gets twice what this round needs (the
    // next rounds of a refinement pass usually split again).
    long long total = 0;
    bool need_grow = false;
    for (int i = 0; i < m.nmesh; ++i) {
      total += newv[i];
      if ((long long)m.nv[i] + newv[i] > m.vcap[i] || (long long)m.ne[i] + 2LL * newv[i] > m.ecap[i])
        need_grow = true;
    }
    std::vector<int> vcap = m.vcap, ecap = m.ecap;
    for (int i = 0; need_grow && i < m.nmesh; ++i) {
      if (newv[i] == 0) continue;
      long long vneed = (long long)m.nv[i] + newv[i];
      long long eneed = (long long)m.ne[i] + 2LL * newv[i];
      if (2 * vneed > m.vcap[i])
        vcap[i] = (int)std::min<long long>(std::max<long long>(2LL * m.vcap[i], 2 * vneed),
                                           (1LL << 30));
      if (2 * eneed > m.ecap[i])
        ecap[i] = (int)std::min<long long>(std::max<long long>(2LL * m.ecap[i], 2 * eneed),
                                           (1LL << 30));
    }
    if (total == 0) {
      complete = true;
      break;
    }
    if (need_grow) {
      cudaError_t e = grow(m, vcap, ecap, m.S.W);
      if (e != cudaSuccess) {
        set_last_error(std::string("growing mesh storage: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
      }
      --nr;  // redo this round on the new layout
      continue;
    }
    const int stamp = tag + 1;
    const int vend = m.vbase.back() + m.nv.back() + newv.back();  // above every new vertex
    PM_LAUNCH(k_refine_vtotals, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, w.vscan);
    PM_LAUNCH(k_refine_newverts, gv, bs, 0, m.stream, m.S, w.vscan, w.vmask, stamp, w.opA);
    zero_counts(m, CN_EL, 2);
    PM_LAUNCH(k_refine_count, ge, bs, 0, m.stream, m.S, w.vscan, w.vmask, w.ecnt, w.emid,
              w.elist, w.counts + CN_EL);
    scan_exclusive(w.ecnt, w.escan, m.S.eused, m.scan, m.st, m.stream);
    PM_LAUNCH(k_refine_split, ge, bs, 0, m.stream, m.S, w.escan, w.emid, w.elist,
              w.counts + CN_EL, w.clist, w.counts + CN_CL, stamp);
    PM_LAUNCH(k_refine_quality, ge, bs, 0, m.stream, m.S, w.clist, w.counts + CN_CL, nullptr);
    // rows of the vertices whose elements changed, through the spare buffer
    PM_LAUNCH(k_refine_rows, grid_tuned(m, vend, bs, bps), bs, 0, m.stream, m.S, m.B, vend, w.vscan,
              w.escan, w.opA, stamp, m.st);
    PM_LAUNCH(k_refine_rows_copy, grid_tuned(m, vend, bs, bps), bs, 0, m.stream, m.S, m.B, vend, stamp);
    PM_LAUNCH(k_refine_sizes, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, w.vscan, w.escan);
    // the new sizes and the status in one read-back
    int* hsz = m.hcounts + CN_NUM;
    cudaMemcpyAsync(hsz, m.S.tab.nv, 2 * m.nmesh * sizeof(int), cudaMemcpyDeviceToHost, m.stream);
    int err = sync_status(m);
    if (err) return err;
    for (int i = 0; i < m.nmesh; ++i) {
      m.nv[i] = hsz[i];
      m.ne[i] = hsz[m.nmesh + i];
    }
    set_used(m);
    if (m.hst->overflow) {  // a row outgrew W: rebuild every row with wider ones
      err = after_overflow(m);
      if (err) return err;
    }
  }
  if (!complete) m.lo_refine = m.tag;
  return PM_OK;
}

// Laplacian sweeps, each a sequence of rounds over the sweep's pending set.
int op_smooth(MeshSet& m, int max_sweeps, int max_rounds) {
  // smoothing changes no topology: one colouring serves every sweep
  if (int err = colour_set(m)) return err;
  const Tuning tu = tuning();
  const int bs = tu.block[TO_SMOOTH], bps = tu.blocks_per_sm[TO_SMOOTH];
  const int rlimit = tu.rounds_limit[2];
  Work& w = m.w;
  const int gv = grid_tuned(m, m.S.vused, bs, bps);
  const int pass0 = m.tag;
  const bool persist = rounds_grid(m, 2) > 0;
  zero_counts(m, 0, CN_NUM);
  PM_LAUNCH(k_init_list, gv, bs, 0, m.stream, m.S, 1, w.D[0], w.counts + CN_D0, nullptr, 0);
  int nlist = 0;  // unknown at first (see op_coarsen)
  long long nr = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int ptag = (m.tag += 2);  // stamp of the next sweep's pending list
    zero_counts(m, CN_P, 1);
    int cur = 0;
    bool moved = false;
    while (max_rounds == 0 || nr < max_rounds) {
      if (persist && nlist >= 0 && nlist <= rlimit) {
        RoundArgs a = round_args(m, cur, pass0, max_rounds == 0 ? (1LL << 30) : max_rounds - nr);
        a.ptag = ptag;
        a.limit = rlimit;
        a.fuse = tu.fuse_limit[1];
        RoundsOut o;
        int err = run_rounds(m, 2, (const void*)k_smooth_rounds, "k_smooth_rounds", a, o);
        if (err) return err;
        nr += o.rounds - o.complete;
        if (o.rounds - o.complete > 0) moved = true;
        cur = o.cur;
        nlist = m.hcounts[cn_list(cur)];
        if (o.complete) break;
        continue;
      }
      int tag = (m.tag += 2);
      int nxt = 1 - cur;
      zero_round(m, nxt);
      PM_LAUNCH(k_smooth_scan, gv, bs, 0, m.stream, m.S, w.D[cur], w.counts + cn_list(cur),
                w.mvM, w.C, w.counts + CN_C, w.cmark, tag, pass0, w.E, w.counts + CN_E);
      PM_LAUNCH(k_smooth_eval, grid_tuned(m, (long long)m.S.vused * TW, bs, bps), bs, 0, m.stream, m.S,
                w.E, w.counts + CN_E, w.mvxy, w.mvM, w.gains, w.C, w.counts + CN_C, w.cmark, tag,
                prof_work("k_smooth_eval"));
      PM_LAUNCH(k_smooth_select_apply, gv, bs, 0, m.stream, m.S, w.C, w.counts + CN_C,
                w.cmark, w.smark, tag, w.D[nxt], w.counts + cn_list(nxt), w.dmark, w.mvxy, w.mvM,
                w.gains, w.P, w.counts + CN_P, w.pmark, ptag, tag + 1,
                (unsigned*)(w.counts + CN_DONE));
      RoundIO io = read_round(m);
      if (io.err) return io.err;
      if (io.nC == 0) break;
      ++nr;
      moved = true;
      cur = nxt;
      nlist = m.hcounts[cn_list(cur)];
    }
    if (!moved) break;
    // the next sweep's pending list becomes the current list
    std::swap(w.D[0], w.P);
    cudaMemcpyAsync(w.counts + CN_D0, w.counts + CN_P, sizeof(int), cudaMemcpyDeviceToDevice,
                    m.stream);
    nlist = m.hcounts[CN_P];
  }
  return PM_OK;
}

// Rounds of optimisation-based smoothing over all interior vertices.
int op_opt_smooth(MeshSet& m, int nrounds, int max_rounds) {
  const Tuning tu = tuning();
  const int bs = tu.block[TO_SMOOTH], bps = tu.blocks_per_sm[TO_SMOOTH];
  Work& w = m.w;
  const int gv = grid_tuned(m, m.S.vused, bs, bps);
  zero_counts(m, 0, CN_NUM);
  PM_LAUNCH(k_init_list, gv, bs, 0, m.stream, m.S, 1, w.C, w.counts + CN_C, nullptr, 0);
  for (int it = 0; it < nrounds && (max_rounds == 0 || it < max_rounds); ++it) {
    int tag = (m.tag += 2);
    zero_counts(m, CN_S, 1);
    PM_LAUNCH(k_stamp_list, gv, bs, 0, m.stream, m.S, w.C, w.counts + CN_C, w.cmark, tag);
    PM_LAUNCH(k_select, gv, bs, 0, m.stream, m.S, w.C, w.counts + CN_C, w.cmark, w.smark, tag,
              w.Sl, w.counts + CN_S, nullptr, nullptr, nullptr);
    PM_LAUNCH(k_opt_apply, grid_tuned(m, (long long)m.S.vused * TW, bs, bps), bs, 0, m.stream, m.S, w.Sl,
              w.counts + CN_S, w.gains, tag + 1);
  }
  return sync_status(m);
}

}  // namespace pm

// Test support (see pm.h): a grid barrier that nothing completes gives up
// after limit_ms and reports PM_ERR_TIMEOUT through the status word.
extern "C" pm_status pm_selftest_wait_timeout(double limit_ms, int32_t* device_status,
                                              double* elapsed_ms) {
  using namespace pm;
  if (!device_status || !elapsed_ms || !(limit_ms > 0.0) || !(limit_ms <= 2000.0))
    return PM_ERR_INVALID_ARG;
  int dev = 0, sms = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
    return PM_ERR_CUDA;
  if (!coop || sms < 1) return PM_ERR_CUDA;
  unsigned* bar = nullptr;
  DevStatus* st = nullptr;
  if (cudaMalloc(&bar, sizeof(unsigned)) != cudaSuccess) return PM_ERR_OOM;
  if (cudaMalloc(&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaFree(bar);
    return PM_ERR_OOM;
  }
  cudaMemset(bar, 0, sizeof(unsigned));
  cudaMemset(st, 0, sizeof(DevStatus));
  unsigned long long limit_ns = (unsigned long long)(limit_ms * 1e6);
  void* args[] = {&bar, &st, &limit_ns};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_selftest_barrier, dim3(sms),
                                              dim3(256), args, 0, 0);
  cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(bar);
  cudaFree(st);
  if (e != cudaSuccess) return PM_ERR_CUDA;
  *device_status = h.err;
  *elapsed_ms = ms;
  return PM_OK;
}
