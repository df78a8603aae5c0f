// Mesh storage: allocation, growth, adjacency construction, validation,
// renumbering and compacted output.
//
// Adjacency (Sec. 3.1, "adjacency list of a vertex"): every vertex slot owns
// two fixed-capacity rows of W int32 entries, NN (neighbour vertices) and NE
// (incident elements), each kept sorted.  Rows are rebuilt from the element
// list here; between rebuilds the operators keep them current through the
// deferred-update commit (pm_ops.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pm_internal.cuh"

namespace pm {

namespace {

// Pinned host memory for per-round read-backs, shared by all mesh sets of the
// process: page-locking is slow and gets slower after many allocate/free
// cycles, so slots of one arena are handed out and recycled instead.
constexpr size_t kPinnedSlot = 16384;
// staging per mesh of upload_tab: band (double4), L_low/L_up/q_thresh, seven
// ints, the seed
constexpr size_t kTabUploadBytes = sizeof(double4) + 3 * sizeof(double) + 7 * sizeof(int) +
                                   sizeof(uint32_t);
constexpr size_t kPinnedBlock = 64 * kPinnedSlot;
std::mutex g_pin_mu;
std::vector<void*> g_pin_free;

void* pinned_get() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    char* blk = nullptr;
    if (cudaMallocHost((void**)&blk, kPinnedBlock) != cudaSuccess) return nullptr;
    for (size_t i = 0; i < kPinnedBlock / kPinnedSlot; ++i)
      g_pin_free.push_back(blk + i * kPinnedSlot);
  }
  void* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_put(void* p) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

// One device allocation per store, carved into 256-byte aligned arrays:
// pools fragmented by many small blocks make each allocation slow, so a mesh
// set asks for one block instead of one per array.
// Only the arrays that are read before they are first written (stamps,
// marks, counters, scan state) are cleared: clearing a whole store of many
// gigabytes at every growth cost more than the growth itself.
struct Carver {
  struct Req {
    void** p;
    size_t bytes;
    bool zero;
  };
  std::vector<Req> req;
  template <class T>
  void add(T** p, size_t count, bool zero = false) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    req.push_back({(void**)p, (bytes + 255) & ~size_t(255), zero});
  }
  cudaError_t commit(MeshSet& m) {
    size_t total = 0;
    for (auto& r : req) total += r.bytes;
    char* base = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&base, total, m.stream);
    if (e != cudaSuccess) return e;
    m.allocs.push_back(base);
    size_t off = 0, zoff = 0, zlen = 0;  // adjacent cleared arrays share one memset
    for (auto& r : req) {
      *r.p = base + off;
      if (r.zero && zoff + zlen == off) {
        zlen += r.bytes;
      } else if (r.zero) {
        if (zlen && (e = cudaMemsetAsync(base + zoff, 0, zlen, m.stream))) return e;
        zoff = off;
        zlen = r.bytes;
      }
      off += r.bytes;
    }
    if (zlen) e = cudaMemsetAsync(base + zoff, 0, zlen, m.stream);
    return e;
  }
};

template <class T>
cudaError_t dalloc(MeshSet& m, T** p, size_t count, bool zero) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMallocAsync((void**)p, bytes, m.stream);
  if (e != cudaSuccess) return e;
  m.allocs.push_back(*p);
  if (zero) e = cudaMemsetAsync(*p, 0, bytes, m.stream);
  return e;
}

__device__ __forceinline__ bool vslot_used(const Store& S, int slot, int& mi) {
  mi = mesh_of_vslot(S, slot);
  return slot - S.tab.vbase[mi] < S.tab.nv[mi];
}

__device__ __forceinline__ bool eslot_used(const Store& S, int slot, int& mi) {
  mi = mesh_of_eslot(S, slot);
  return slot - S.tab.ebase[mi] < S.tab.ne[mi];
}

// Mesh of every slot of the layout (binary search over the sorted bases),
// once per allocation.
__global__ void k_mesh_index(int n, const int* base, int slots, int* out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (base[mid] <= s) lo = mid; else hi = mid - 1;
    }
    out[s] = lo;
  }
}

// ---- relayout (growth) ------------------------------------------------------

// Per-slot data of every used vertex slot into its place in the new layout.
__global__ void k_relayout_v(Store A, Store B) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(A, s, mi)) continue;
    int ns = B.tab.vbase[mi] + (s - A.tab.vbase[mi]);
    B.xy[ns] = A.xy[s];
    B.M[ns] = A.M[s];
    B.vflag[ns] = A.vflag[s];
    B.touch[ns] = A.touch[s];
    B.ntouch[ns] = A.ntouch[s];
    B.evc[ns] = A.evc[s];
    B.evs[ns] = A.evs[s];
    B.evm[ns] = A.evm[s];
    B.evr[ns] = A.evr[s];
    if (A.lid && B.lid) B.lid[ns] = A.lid[s];
    B.NNlen[ns] = A.NNlen[s];
    B.NElen[ns] = A.NElen[s];
  }
}

// The rows: thread t copies 16-byte chunk t % (W/4) of row t / (W/4), so a
// warp moves consecutive chunks (whole rows when W = 16); chunks past the
// row's length are not copied (nothing reads them).  W of both layouts is a
// multiple of 4 and the new one is at least the old one.
__global__ void k_relayout_rows(Store A, Store B) {
  const int cpr = A.W >> 2;
  const long long total = (long long)A.vused * cpr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int s = (int)(t / cpr), c = (int)(t - (long long)s * cpr);
    int mi;
    if (!vslot_used(A, s, mi)) continue;
    int ns = B.tab.vbase[mi] + (s - A.tab.vbase[mi]);
    if (4 * c < A.NNlen[s])
      reinterpret_cast<int4*>(B.NN + (size_t)ns * B.W)[c] =
          reinterpret_cast<const int4*>(A.NN + (size_t)s * A.W)[c];
    if (4 * c < A.NElen[s])
      reinterpret_cast<int4*>(B.NE + (size_t)ns * B.W)[c] =
          reinterpret_cast<const int4*>(A.NE + (size_t)s * A.W)[c];
  }
}

__global__ void k_relayout_e(Store A, Store B) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(A, s, mi)) continue;
    int ns = B.tab.ebase[mi] + (s - A.tab.ebase[mi]);
    B.EN[ns] = A.EN[s];
    B.qK[ns] = A.qK[s];
  }
}

// ---- adjacency build ----------------------------------------------------------

__global__ void k_zero_nelen(Store S) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    S.NElen[s] = 0;
  }
}

__global__ void k_fill_ne(Store S, DevStatus* st) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(S, s, mi)) continue;
    int4 e = S.EN[s];
    if (!e.w) continue;
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi];
    int K = s - eb;
    int vs[3] = {e.x, e.y, e.z};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      int slot = vb + vs[i];
      int pos = atomicAdd(S.NElen + slot, 1);
      if (pos < S.W) S.NE[(size_t)slot * S.W + pos] = K;
      else atomicExch(&st->overflow, 1);
    }
  }
}

// Sort the NE row, derive the NN row (sorted union of the other vertices of
// the incident elements), check manifoldness, optionally derive the boundary
// flag (a vertex is on the boundary when it has one more neighbour than
// incident elements).
__global__ void k_finish_rows(Store S, int derive, DevStatus* st) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(S, s, mi)) continue;
    uint8_t f = S.vflag[s];
    if (!(f & VF_ALIVE)) {
      S.NNlen[s] = 0;
      S.NElen[s] = 0;
      continue;
    }
    int nel = S.NElen[s];
    if (nel > S.W) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->maxdeg, nel);
      continue;
    }
    int* ne = S.NE + (size_t)s * S.W;
    int buf[MAXW];
    for (int k = 0; k < nel; ++k) buf[k] = ne[k];
    for (int k = 1; k < nel; ++k) {  // insertion sort
      int x = buf[k];
      int j = k - 1;
      while (j >= 0 && buf[j] > x) {
        buf[j + 1] = buf[j];
        --j;
      }
      buf[j + 1] = x;
    }
    for (int k = 0; k < nel; ++k) ne[k] = buf[k];
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi];
    int lv = s - vb;
    int nnb[MAXW];
    int nn = 0;
    int nxt[MAXW];
    int nnx = 0;
    bool ok = true;
    for (int k = 0; k < nel; ++k) {
      int4 e = S.EN[eb + buf[k]];
      int i = (e.x == lv) ? 0 : (e.y == lv) ? 1 : 2;
      int vv[3] = {e.x, e.y, e.z};
      int a = vv[(i + 1) % 3], b = vv[(i + 2) % 3];
      if (!sorted_insert(nnb, nn, MAXW, a) || !sorted_insert(nnb, nn, MAXW, b)) ok = false;
      // the outgoing directed edge lv->a must be unique (no overlapping elements)
      int before = nnx;
      if (!sorted_insert(nxt, nnx, MAXW, a)) ok = false;
      if (nnx == before && derive) set_err(st, PM_ERR_INVALID_MESH);
    }
    if (!ok || nn > S.W) {
      atomicExch(&st->overflow, 1);
      atomicMax(&st->maxdeg, nn);
      continue;
    }
    atomicMax(&st->maxdeg, nn);
    int* row = S.NN + (size_t)s * S.W;
    for (int k = 0; k < nn; ++k) row[k] = nnb[k];
    S.NNlen[s] = nn;
    if (derive) {
      int d = nn - nel;
      if (nel == 0 || (d != 0 && d != 1)) set_err(st, PM_ERR_INVALID_MESH);
      S.vflag[s] = (uint8_t)((f & ~VF_BND) | (d == 1 ? VF_BND : 0));
    }
  }
}

__device__ __forceinline__ int edge_elements(const Store& S, int slot, int eb, int lw) {
  const int* ne = S.NE + (size_t)slot * S.W;
  int nel = S.NElen[slot];
  int c = 0;
  for (int k = 0; k < nel; ++k) {
    int4 e = S.EN[eb + ne[k]];
    if (e.x == lw || e.y == lw || e.z == lw) ++c;
  }
  return c;
}

// Corners: boundary vertices whose two boundary neighbours are not collinear
// with them, or (given) the caller's flags, already set in vflag by the ingest.
__global__ void k_corners(Store S, int given) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(S, s, mi)) continue;
    uint8_t f = S.vflag[s];
    if (!(f & VF_ALIVE)) continue;
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi];
    bool c = false;
    if (given) {
      c = (f & VF_CORNER) != 0;
    } else if (f & VF_BND) {
      const int* nn = S.NN + (size_t)s * S.W;
      int nnl = S.NNlen[s];
      int bn[2];
      int k2 = 0;
      for (int k = 0; k < nnl; ++k) {
        if (edge_elements(S, s, eb, nn[k]) == 1 && k2 < 2) bn[k2++] = nn[k];
      }
      if (k2 < 2) {
        c = true;
      } else {
        int lo = bn[0] < bn[1] ? bn[0] : bn[1];
        int hi = bn[0] < bn[1] ? bn[1] : bn[0];
        c = orient_sign(load_vd(S, vb + lo), load_vd(S, s), load_vd(S, vb + hi)) != 0;
      }
    }
    S.vflag[s] = (uint8_t)((f & ~VF_CORNER) | (c ? VF_CORNER : 0));
  }
}

// Every used vertex slot holds finite coordinates (PM_ERR_INVALID_ARG).
__global__ void k_validate_coords(Store S, DevStatus* st) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    const int mi = mesh_of_vslot(S, s);
    if (s - S.tab.vbase[mi] >= S.tab.nv[mi]) continue;
    const double2 p = S.xy[s];
    if (!isfinite(p.x) || !isfinite(p.y)) set_err(st, PM_ERR_INVALID_ARG);
  }
}

// Ids in range, distinct, and every element counter-clockwise (canonical).
__global__ void k_validate_elems(Store S, DevStatus* st) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(S, s, mi)) continue;
    int4 e = S.EN[s];
    if (!e.w) continue;
    int nv = S.tab.nv[mi], vb = S.tab.vbase[mi];
    if (e.x < 0 || e.y < 0 || e.z < 0 || e.x >= nv || e.y >= nv || e.z >= nv || e.x == e.y ||
        e.y == e.z || e.x == e.z) {
      set_err(st, PM_ERR_INVALID_MESH);
      continue;
    }
    if (orient_sign(load_vd(S, vb + e.x), load_vd(S, vb + e.y), load_vd(S, vb + e.z)) <= 0)
      set_err(st, PM_ERR_INVALID_MESH);
  }
}

// Quality of every live element into the cache.
__global__ void k_qcache_all(Store S) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(S, s, mi)) continue;
    int4 e = S.EN[s];
    if (!e.w) continue;
    int vb = S.tab.vbase[mi];
    S.qK[s] = quality_c(e.x, e.y, e.z, load_vd(S, vb + e.x), load_vd(S, vb + e.y),
                        load_vd(S, vb + e.z));
  }
}

// ---- renumbering -----------------------------------------------------------

// The compacted counts become the used slots of every mesh.
__global__ void k_set_sizes(Store S, const int* tot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nmesh) return;
  S.tab.nv[i] = tot[2 * i];
  S.tab.ne[i] = tot[2 * i + 1];
}

// Live counts of every mesh; with `changed`, records whether any mesh has a
// dead slot (its compaction is not the identity).
__global__ void k_mesh_totals(Store S, const int* vscan, const int* escan, int* out,
                              int* changed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nmesh) return;
  int vb = S.tab.vbase[i], eb = S.tab.ebase[i];
  out[2 * i] = vscan[vb + S.tab.nv[i]] - vscan[vb];
  out[2 * i + 1] = escan[eb + S.tab.ne[i]] - escan[eb];
  if (changed && (out[2 * i] != S.tab.nv[i] || out[2 * i + 1] != S.tab.ne[i]))
    atomicOr(changed, 1);
}

// One slot per thread.  Rows move in 16-byte chunks (W is a multiple of 4 and
// rows start W-aligned); entries past the row length read as -1.
__device__ __forceinline__ void renum_row(const int* row, int len, int* out, const int* scan,
                                          int base, int first) {
  for (int k = 0; k < len; k += 4) {
    int4 q = *reinterpret_cast<const int4*>(row + k);
    int4 r;
    r.x = scan[base + q.x] - first;
    r.y = (k + 1 < len) ? scan[base + q.y] - first : -1;
    r.z = (k + 2 < len) ? scan[base + q.z] - first : -1;
    r.w = (k + 3 < len) ? scan[base + q.w] - first : -1;
    *reinterpret_cast<int4*>(out + k) = r;
  }
}

__global__ void k_renum_v(Store A, Store B, const int* vscan, const int* escan,
                          const int* changed) {
  if (!*changed) return;  // nothing died since the last compaction
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(A, s, mi)) continue;
    if (!(A.vflag[s] & VF_ALIVE)) continue;
    int vb = A.tab.vbase[mi], eb = A.tab.ebase[mi];
    int v0 = vscan[vb], e0 = escan[eb];
    int ns = vb + (vscan[s] - v0);
    B.xy[ns] = A.xy[s];
    B.M[ns] = A.M[s];
    B.vflag[ns] = A.vflag[s];
    B.touch[ns] = A.touch[s];
    B.ntouch[ns] = A.ntouch[s];
    B.evc[ns] = A.evc[s];
    B.evs[ns] = A.evs[s];
    B.evm[ns] = A.evm[s];
    B.evr[ns] = A.evr[s];
    int a = A.NNlen[s], b = A.NElen[s];
    renum_row(A.NN + (size_t)s * A.W, a, B.NN + (size_t)ns * B.W, vscan, vb, v0);
    renum_row(A.NE + (size_t)s * A.W, b, B.NE + (size_t)ns * B.W, escan, eb, e0);
    B.NNlen[ns] = a;
    B.NElen[ns] = b;
  }
}

// Renumbering in place: every live vertex's id becomes its rank among the
// live slots of its mesh; ids of slots appended later skip the dead slots.
__global__ void k_renum_ids(Store S, const int* vscan, const int* tot, int* lid, int* voff) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(S, s, mi)) continue;
    if (!(S.vflag[s] & VF_ALIVE)) continue;
    int vb = S.tab.vbase[mi];
    lid[s] = vscan[s] - vscan[vb];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nmesh; i += gridDim.x * blockDim.x)
    voff[i] = S.tab.nv[i] - tot[2 * i];
}

__global__ void k_renum_e(Store A, Store B, const int* vscan, const int* escan,
                          const int* changed) {
  if (!*changed) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(A, s, mi)) continue;
    int4 e = A.EN[s];
    if (!e.w) continue;
    int vb = A.tab.vbase[mi], eb = A.tab.ebase[mi];
    int v0 = vscan[vb];
    int ns = eb + (escan[s] - escan[eb]);
    B.EN[ns] = make_int4(vscan[vb + e.x] - v0, vscan[vb + e.y] - v0, vscan[vb + e.z] - v0, 1);
    B.qK[ns] = A.qK[s];
  }
}

// Compacted output of one mesh (canonical rotation of every triangle).
__global__ void k_out_v(Store S, int mesh, const int* vscan, double* xy, double* mt) {
  int vb = S.tab.vbase[mesh], nv = S.tab.nv[mesh];
  int v0 = vscan[vb];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nv; l += gridDim.x * blockDim.x) {
    int s = vb + l;
    if (!(S.vflag[s] & VF_ALIVE)) continue;
    int o = vscan[s] - v0;
    double2 p = S.xy[s];
    double4 m = S.M[s];
    if (xy) {
      xy[2 * o] = p.x;
      xy[2 * o + 1] = p.y;
    }
    if (mt) {
      mt[3 * o] = m.x;
      mt[3 * o + 1] = m.y;
      mt[3 * o + 2] = m.z;
    }
  }
}

__global__ void k_out_e(Store S, int mesh, const int* vscan, const int* escan, int32_t* tri) {
  int vb = S.tab.vbase[mesh], eb = S.tab.ebase[mesh], ne = S.tab.ne[mesh];
  int v0 = vscan[vb], e0 = escan[eb];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ne; l += gridDim.x * blockDim.x) {
    int s = eb + l;
    int4 e = S.EN[s];
    if (!e.w) continue;
    int o = escan[s] - e0;
    int a = vscan[vb + e.x] - v0, b = vscan[vb + e.y] - v0, c = vscan[vb + e.z] - v0;
    if (b < a && b < c) {
      int t = a; a = b; b = c; c = t;
    } else if (c < a && c < b) {
      int t = c; c = b; b = a; a = t;
    }
    tri[3 * o] = a;
    tri[3 * o + 1] = b;
    tri[3 * o + 2] = c;
  }
}

// Element count each mesh's metric asks for, before the factor 4/sqrt(3):
// the sum over live elements of area * mean sqrt(det M) of its vertices (the
// number of unit equilateral metric triangles that tile the mesh).  Only
// sizes storage, so the order of the atomic sums does not matter.
__global__ void k_estimate(Store S, double* est) {
  const int lane = threadIdx.x & 31;
  for (int s0 = blockIdx.x * blockDim.x; s0 < S.eused; s0 += gridDim.x * blockDim.x) {
    const int s = s0 + (int)threadIdx.x;
    int mi = -1;
    double x = 0.0;
    if (s < S.eused && eslot_used(S, s, mi)) {
      int4 e = S.EN[s];
      if (e.w) {
        int vb = S.tab.vbase[mi];
        VD a = load_vd(S, vb + e.x), b = load_vd(S, vb + e.y), c = load_vd(S, vb + e.z);
        double area = 0.5 * fabs(orient3(a, b, c));
        double sd = sqrt(fmax(a.m00 * a.m11 - a.m01 * a.m01, 0.0)) +
                    sqrt(fmax(b.m00 * b.m11 - b.m01 * b.m01, 0.0)) +
                    sqrt(fmax(c.m00 * c.m11 - c.m01 * c.m01, 0.0));
        x = area * sd / 3.0;
      }
    }
    // a warp whose slots all belong to one mesh (meshes are contiguous runs
    // of slots) adds its sum with one atomic
    const int m0 = __shfl_sync(0xffffffffu, mi, 0);
    if (__all_sync(0xffffffffu, mi == m0) && m0 >= 0) {
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) atomicAdd(est + m0, x);
    } else if (mi >= 0) {
      atomicAdd(est + mi, x);
    }
  }
}

// Output offsets of every mesh: exclusive prefix sums over the meshes of the
// live counts tot[2i] (vertices) and tot[2i+1] (elements) into pre (vertex
// offsets pre[0..n], element offsets pre[n+1..2n+1]).  One block: each
// thread sums a contiguous chunk of meshes, thread 0 scans the chunk sums.
__global__ void k_out_prefix(int n, const int* tot, int* pre) {
  __shared__ long long part[2][1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int a = t * per, b = min(n, a + per);
  long long sv = 0, se = 0;
  for (int i = a; i < b; ++i) {
    sv += tot[2 * i];
    se += tot[2 * i + 1];
  }
  part[0][t] = sv;
  part[1][t] = se;
  __syncthreads();
  if (t == 0) {
    long long cv = 0, ce = 0;
    for (int k = 0; k < T; ++k) {
      long long x = part[0][k], y = part[1][k];
      part[0][k] = cv;
      part[1][k] = ce;
      cv += x;
      ce += y;
    }
    pre[n] = (int)cv;
    pre[n + 1 + n] = (int)ce;
  }
  __syncthreads();
  long long cv = part[0][t], ce = part[1][t];
  for (int i = a; i < b; ++i) {
    pre[i] = (int)cv;
    pre[n + 1 + i] = (int)ce;
    cv += tot[2 * i];
    ce += tot[2 * i + 1];
  }
}

// Compacted output of every mesh of the set, meshes one after the other
// (offsets in S.tab.pre); vertex ids in the triangles are local to the mesh.
__global__ void k_out_v_set(Store S, const int* vscan, double* xy, double* mt) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.vused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!vslot_used(S, s, mi)) continue;
    if (!(S.vflag[s] & VF_ALIVE)) continue;
    int vb = S.tab.vbase[mi];
    int o = S.tab.pre[mi] + (vscan[s] - vscan[vb]);
    double2 p = S.xy[s];
    double4 m = S.M[s];
    if (xy) {
      xy[2 * (size_t)o] = p.x;
      xy[2 * (size_t)o + 1] = p.y;
    }
    if (mt) {
      mt[3 * (size_t)o] = m.x;
      mt[3 * (size_t)o + 1] = m.y;
      mt[3 * (size_t)o + 2] = m.z;
    }
  }
}

__global__ void k_out_e_set(Store S, const int* vscan, const int* escan, int32_t* tri) {
  const int n = S.nmesh;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.eused; s += gridDim.x * blockDim.x) {
    int mi;
    if (!eslot_used(S, s, mi)) continue;
    int4 e = S.EN[s];
    if (!e.w) continue;
    int vb = S.tab.vbase[mi], eb = S.tab.ebase[mi];
    int v0 = vscan[vb];
    int o = S.tab.pre[n + 1 + mi] + (escan[s] - escan[eb]);
    int a = vscan[vb + e.x] - v0, b = vscan[vb + e.y] - v0, c = vscan[vb + e.z] - v0;
    if (b < a && b < c) {
      int t = a; a = b; b = c; c = t;
    } else if (c < a && c < b) {
      int t = c; c = b; b = a; a = t;
    }
    tri[3 * (size_t)o] = a;
    tri[3 * (size_t)o + 1] = b;
    tri[3 * (size_t)o + 2] = c;
  }
}

}  // namespace

// ---------------------------------------------------------------------------

// Bounds below which every used slot lies (from the host mirror).
void set_used(MeshSet& m) {
  int last = m.nmesh - 1;
  m.S.vused = m.vbase[last] + m.nv[last];
  m.S.eused = m.ebase[last] + m.ne[last];
  m.B.vused = m.S.vused;
  m.B.eused = m.S.eused;
}

cudaError_t upload_tab(MeshSet& m) {
  const int n = m.nmesh;
  set_used(m);
  // staging in pinned memory (no stream synchronisation); the previous upload
  // of this set has normally long left it
  if (m.upev) cudaEventSynchronize(m.upev);
  double4* band = (double4*)m.hup;
  double* dbl = (double*)(band + n);
  int* ints = (int*)(dbl + 3 * n);
  uint32_t* seed = (uint32_t*)(ints + 7 * n);
  for (int i = 0; i < n; ++i) {
    ints[i] = m.vbase[i];
    ints[n + i] = m.vcap[i];
    ints[2 * n + i] = m.ebase[i];
    ints[3 * n + i] = m.ecap[i];
    ints[4 * n + i] = m.nv[i];
    ints[5 * n + i] = m.ne[i];
    ints[6 * n + i] = m.select.empty() ? 0 : m.select[i];
    seed[i] = m.seed[i];
    dbl[i] = m.L_low[i];
    dbl[n + i] = m.L_up[i];
    dbl[2 * n + i] = m.q_thresh[i];
    double a = m.L_low[i], b = m.L_up[i];
    double alo = a * (1.0 - 1e-9), ahi = a * (1.0 + 1e-9);
    double blo = b * (1.0 - 1e-9), bhi = b * (1.0 + 1e-9);
    band[i] = make_double4(alo * alo, ahi * ahi, blo * blo, bhi * bhi);
  }
  cudaError_t e = cudaMemcpyAsync(m.S.tab.vbase, ints, 7 * n * sizeof(int), cudaMemcpyHostToDevice,
                                  m.stream);
  if (!e) e = cudaMemcpyAsync(m.S.tab.seed, seed, n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                              m.stream);
  if (!e) e = cudaMemcpyAsync(m.S.tab.L_low, dbl, 3 * n * sizeof(double), cudaMemcpyHostToDevice,
                              m.stream);
  if (!e) e = cudaMemcpyAsync(m.S.tab.band, band, n * sizeof(double4), cudaMemcpyHostToDevice,
                              m.stream);
  if (!e && m.upev) e = cudaEventRecord(m.upev, m.stream);
  if (!e && !m.mesh_index_ok) {
    PM_LAUNCH(k_mesh_index, grid_for(m, m.S.vslots), BLOCK, 0, m.stream, n,
              (const int*)m.S.tab.vbase, m.S.vslots, m.S.tab.vmesh);
    PM_LAUNCH(k_mesh_index, grid_for(m, m.S.eslots), BLOCK, 0, m.stream, n,
              (const int*)m.S.tab.ebase, m.S.eslots, m.S.tab.emesh);
    m.mesh_index_ok = true;
    e = cudaGetLastError();
  }
  return e;
}

// Read back the per-mesh used-slot counts (nv, ne) into the host mirror.
cudaError_t refresh_sizes(MeshSet& m) {
  std::vector<int> t(2 * m.nmesh);
  cudaError_t e = cudaMemcpyAsync(t.data(), m.S.tab.nv, 2 * m.nmesh * sizeof(int),
                                  cudaMemcpyDeviceToHost, m.stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(m.stream);
  for (int i = 0; i < m.nmesh; ++i) {
    m.nv[i] = t[i];
    m.ne[i] = t[m.nmesh + i];
  }
  set_used(m);
  return e;
}

static void carve_store(Carver& cv, Store& S) {
  size_t V = S.vslots, E = S.eslots, W = S.W;
  cv.add(&S.xy, V);
  cv.add(&S.M, V);
  cv.add(&S.EN, E);
  cv.add(&S.qK, E);
  cv.add(&S.NN, V * W);
  cv.add(&S.NE, V * W);
  // cleared: flags, row lengths and stamps
  cv.add(&S.vflag, V, true);
  cv.add(&S.NNlen, V, true);
  cv.add(&S.NElen, V, true);
  cv.add(&S.touch, V, true);
  cv.add(&S.ntouch, V, true);
  cv.add(&S.evc, V, true);
  cv.add(&S.evs, V, true);
  cv.add(&S.evm, V, true);
  cv.add(&S.evr, V, true);
}

cudaError_t set_alloc(MeshSet& m, const std::vector<int>& vcap, const std::vector<int>& ecap,
                      int W) {
  int n = m.nmesh;
  m.vcap = vcap;
  m.ecap = ecap;
  m.vbase.assign(n, 0);
  m.ebase.assign(n, 0);
  long long vs = 0, es = 0;
  for (int i = 0; i < n; ++i) {
    m.vbase[i] = (int)vs;
    m.ebase[i] = (int)es;
    vs += vcap[i];
    es += ecap[i];
  }
  if (vs >= (1LL << 31) - 4 || es >= (1LL << 31) - 4 || vs * (long long)W >= (1LL << 40))
    return cudaErrorMemoryAllocation;
  cudaError_t e;
  Store& S = m.S;
  S.nmesh = n;
  S.W = W;
  S.vslots = (int)vs;
  S.eslots = (int)es;
  S.lid = S.voff = nullptr;
  m.B = S;
  Carver cv;
  carve_store(cv, S);
  carve_store(cv, m.B);
  size_t tab_bytes = (size_t)n * (8 * sizeof(int) + 2 * sizeof(uint32_t) + 3 * sizeof(int) +
                                  2 * sizeof(unsigned long long) + 3 * sizeof(double) +
                                  sizeof(double4)) +
                     2 * ((size_t)n + 1) * sizeof(int) + 64;
  char* t = nullptr;
  cv.add(&t, tab_bytes, true);
  int* vmesh = nullptr;
  int* emesh = nullptr;
  if (n > 1) {
    cv.add(&vmesh, vs);
    cv.add(&emesh, es);
  }
  int* col = nullptr;
  cv.add(&col, vs);
  Work& w = m.w;
  cv.add(&w.D[0], vs);
  cv.add(&w.D[1], vs);
  cv.add(&w.C, vs);
  cv.add(&w.Sl, vs);
  cv.add(&w.A, vs);
  cv.add(&w.P, vs);
  cv.add(&w.target, vs);
  cv.add(&w.opA, vs);
  cv.add(&w.opK2, vs);
  cv.add(&w.mvxy, vs);
  cv.add(&w.mvM, vs);
  cv.add(&w.dmark, vs, true);
  cv.add(&w.amark, vs, true);
  cv.add(&w.cmark, vs, true);
  cv.add(&w.smark, vs, true);
  cv.add(&w.pmark, vs, true);
  cv.add(&w.vcnt, vs + 1);
  cv.add(&w.vscan, vs + 1);
  cv.add(&w.vmask, vs);
  cv.add(&w.ecnt, es + 1);
  cv.add(&w.escan, es + 1);
  cv.add(&w.emid, es);
  cv.add(&w.elist, es);
  cv.add(&w.clist, es);
  cv.add(&w.E, vs);
  // each interior edge gives at most two items and a planar mesh has < 3V edges
  cv.add(&w.items, (size_t)vs * 6 + 64);
  cv.add(&w.gains, (size_t)vs * W);
  cv.add(&w.items2, vs);
  cv.add(&w.cand, (size_t)vs * W);
  cv.add(&w.ncand, vs);
  cv.add(&w.counts, CN_NUM + 2 * n + 8, true);
  cv.add(&w.cprop, vs);
  cv.add(&w.cstamp, vs, true);
  cv.add(&m.lidbuf, vs);
  cv.add(&m.voffbuf, n);
  int tiles = scan_tiles((int)std::max(vs, es) + 1);
  cv.add(&m.scan.state, tiles, true);
  cv.add(&m.scan.ticket, 1, true);
  m.scan.tiles_cap = tiles;
  if ((e = cv.commit(m))) return e;
  m.tabmem = t;
  MeshTab& T = S.tab;
  // 32-byte, then 8-byte aligned members first
  T.band = (double4*)t; t += n * sizeof(double4);
  T.L_low = (double*)t; t += n * sizeof(double);
  T.L_up = (double*)t; t += n * sizeof(double);
  T.q_thresh = (double*)t; t += n * sizeof(double);
  T.ops = (unsigned long long*)t; t += n * sizeof(unsigned long long);
  T.iter_ops = (unsigned long long*)t; t += n * sizeof(unsigned long long);
  T.vbase = (int*)t; t += n * sizeof(int);
  T.vcap = (int*)t; t += n * sizeof(int);
  T.ebase = (int*)t; t += n * sizeof(int);
  T.ecap = (int*)t; t += n * sizeof(int);
  T.nv = (int*)t; t += n * sizeof(int);
  T.ne = (int*)t; t += n * sizeof(int);
  T.select = (int*)t; t += n * sizeof(int);
  T.ncol = (int*)t; t += n * sizeof(int);
  T.seed = (uint32_t*)t; t += n * sizeof(uint32_t);
  T.r = (uint32_t*)t; t += n * sizeof(uint32_t);
  T.had = (int*)t; t += 2 * n * sizeof(int);  // two sets: persistent rounds alternate
  T.active = (int*)t; t += n * sizeof(int);
  T.pre = (int*)t; t += 2 * ((size_t)n + 1) * sizeof(int);
  T.vmesh = vmesh;
  T.emesh = emesh;
  T.col = col;
  m.mesh_index_ok = n == 1;
  m.B.tab = T;
  if (!m.st) {
    if ((e = cudaMallocAsync((void**)&m.st, sizeof(DevStatus), m.stream))) return e;
    if ((e = cudaMemsetAsync(m.st, 0, sizeof(DevStatus), m.stream))) return e;
    const size_t counts_bytes = (CN_NUM + 2 * (size_t)std::max(n, 1024) + 8) * sizeof(int);
    const size_t ops_off = 64 + ((counts_bytes + 7) & ~size_t(7));
    const size_t up_off = (ops_off + 3 * (size_t)n * sizeof(unsigned long long) + 63) & ~size_t(63);
    size_t need = up_off + (size_t)n * kTabUploadBytes;
    if (need <= kPinnedSlot) {
      m.pinned = pinned_get();
      if (!m.pinned) return cudaErrorMemoryAllocation;
      m.pinned_own = false;
    } else {
      if ((e = cudaMallocHost(&m.pinned, need))) return e;
      m.pinned_own = true;
    }
    m.hst = (DevStatus*)m.pinned;
    m.hcounts = (int*)((char*)m.pinned + 64);
    m.hops = (unsigned long long*)((char*)m.pinned + ops_off);
    m.hup = (char*)m.pinned + up_off;
    if ((e = cudaEventCreateWithFlags(&m.upev, cudaEventDisableTiming))) return e;
  }
  return cudaSuccess;
}

void set_free(MeshSet& m) {
  for (void* p : m.allocs) cudaFreeAsync(p, m.stream);
  m.allocs.clear();
}

void set_release(MeshSet& m) {
  if (m.st) cudaFreeAsync(m.st, m.stream);
  cudaStreamSynchronize(m.stream);
  if (m.pinned) {
    if (m.pinned_own) cudaFreeHost(m.pinned);
    else pinned_put(m.pinned);
  }
  if (m.upev) cudaEventDestroy(m.upev);
  m.st = nullptr;
  m.pinned = nullptr;
  m.hst = nullptr;
  m.hcounts = nullptr;
  m.hops = nullptr;
  m.hup = nullptr;
  m.upev = nullptr;
}

// Move the meshes into new regions of capacity vcap/ecap and row width W.
cudaError_t grow(MeshSet& m, const std::vector<int>& vcap, const std::vector<int>& ecap, int W) {
  MeshSet n2;
  n2.device = m.device;
  n2.stream = m.stream;
  n2.nmesh = m.nmesh;
  n2.nv = m.nv;
  n2.ne = m.ne;
  n2.seed = m.seed;
  n2.L_low = m.L_low;
  n2.L_up = m.L_up;
  n2.q_thresh = m.q_thresh;
  n2.select = m.select;
  n2.st = m.st;
  n2.hst = m.hst;
  n2.hcounts = m.hcounts;
  n2.hops = m.hops;
  n2.hup = m.hup;
  n2.upev = m.upev;
  n2.num_sms = m.num_sms;
  cudaError_t e = set_alloc(n2, vcap, ecap, W);
  if (e != cudaSuccess) {
    set_free(n2);
    return e;
  }
  if ((e = upload_tab(n2))) {
    set_free(n2);
    return e;
  }
  // carry the per-call round counters and op counts
  int nm = m.nmesh;
  cudaMemcpyAsync(n2.S.tab.r, m.S.tab.r, nm * sizeof(uint32_t), cudaMemcpyDeviceToDevice, m.stream);
  cudaMemcpyAsync(n2.S.tab.active, m.S.tab.active, nm * sizeof(int), cudaMemcpyDeviceToDevice,
                  m.stream);
  cudaMemcpyAsync(n2.S.tab.ops, m.S.tab.ops, 2 * nm * sizeof(unsigned long long),
                  cudaMemcpyDeviceToDevice, m.stream);
  if (m.S.lid) {  // ids that are not slot offsets move with their slots
    n2.S.lid = n2.lidbuf;
    n2.S.voff = n2.voffbuf;
    cudaMemcpyAsync(n2.voffbuf, m.S.voff, nm * sizeof(int), cudaMemcpyDeviceToDevice, m.stream);
  }
  PM_LAUNCH(k_relayout_v, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, n2.S);
  PM_LAUNCH(k_relayout_rows, grid_for(m, (long long)m.S.vused * (m.S.W / 4)), BLOCK, 0, m.stream,
            m.S, n2.S);
  PM_LAUNCH(k_relayout_e, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, n2.S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  set_free(m);
  m.vbase = n2.vbase;
  m.vcap = n2.vcap;
  m.ebase = n2.ebase;
  m.ecap = n2.ecap;
  m.S = n2.S;
  m.B = n2.B;
  m.w = n2.w;
  m.scan = n2.scan;
  m.tabmem = n2.tabmem;
  m.lidbuf = n2.lidbuf;
  m.voffbuf = n2.voffbuf;
  m.allocs = n2.allocs;
  n2.allocs.clear();
  // per-round stamp arrays start at zero, below every later tag; scratch that
  // held evaluation results is fresh, so earlier evaluations are stale
  m.lo_coarsen = m.lo_swap = m.lo_refine = m.tag;
  return cudaSuccess;
}

// Widen the adjacency rows to W (contents are rebuilt by the caller); every
// other array, worklist and stamp keeps its place.
// Frees `p` only when it is an allocation of its own (arrays carved from the
// store's block go with the block).
static void free_if_own(MeshSet& m, void* p) {
  auto it = std::find(m.allocs.begin(), m.allocs.end(), p);
  if (it == m.allocs.end()) return;
  cudaFreeAsync(p, m.stream);
  m.allocs.erase(it);
}

cudaError_t grow_rows(MeshSet& m, int W) {
  void* ptrs[4] = {m.S.NN, m.S.NE, m.B.NN, m.B.NE};
  for (void* p : ptrs) free_if_own(m, p);
  size_t n = (size_t)m.S.vslots * W;
  cudaError_t e;
  if ((e = dalloc(m, &m.S.NN, n, false))) return e;
  if ((e = dalloc(m, &m.S.NE, n, false))) return e;
  if ((e = dalloc(m, &m.B.NN, n, false))) return e;
  if ((e = dalloc(m, &m.B.NE, n, false))) return e;
  m.S.W = W;
  m.B.W = W;
  free_if_own(m, m.w.gains);
  free_if_own(m, m.w.cand);
  if ((e = dalloc(m, &m.w.cand, n, false))) return e;
  return dalloc(m, &m.w.gains, n, false);
}

int sync_status(MeshSet& m) {
  cudaError_t e = cudaMemcpyAsync(m.hst, m.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, m.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m.stream);
  if (e != cudaSuccess) {
    set_last_error(std::string("CUDA: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  return m.hst->err;
}

// Build NN and NE from the element list for every mesh of the set.  With
// `derive_flags` (creation) also derive boundary and corner flags and check
// manifoldness.  Grows W (rebuilding) when a row does not fit.
int rebuild_adjacency(MeshSet& m, bool derive_flags, bool corners_given) {
  for (;;) {
    cudaMemsetAsync(&m.st->overflow, 0, 2 * sizeof(int), m.stream);
    PM_LAUNCH(k_zero_nelen, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S);
    PM_LAUNCH(k_fill_ne, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, m.st);
    PM_LAUNCH(k_finish_rows, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, derive_flags ? 1 : 0,
                                                                  m.st);
    int err = sync_status(m);
    if (err) return err;
    if (!m.hst->overflow) break;
    int need = std::max(m.hst->maxdeg, m.S.W + 1);
    int W = m.S.W;
    while (W < need) W *= 2;
    if (W > MAXW) {
      set_last_error("adjacency row longer than the supported maximum of 128 entries");
      return PM_ERR_CAPACITY;
    }
    cudaError_t e = grow_rows(m, W);
    if (e != cudaSuccess) {
      set_last_error(std::string("growing adjacency rows: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
    }
  }
  if (derive_flags) {
    PM_LAUNCH(k_corners, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, corners_given ? 1 : 0);
    return sync_status(m);
  }
  return PM_OK;
}

int refresh_quality(MeshSet& m) {
  PM_LAUNCH(k_qcache_all, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S);
  m.qvalid = true;
  return sync_status(m);
}

int ensure_quality(MeshSet& m) { return m.qvalid ? PM_OK : refresh_quality(m); }

int validate_mesh(MeshSet& m) {
  PM_LAUNCH(k_validate_coords, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, m.st);
  int err = sync_status(m);
  if (err) return err;  // orientations of non-finite points mean nothing
  PM_LAUNCH(k_validate_elems, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, m.st);
  return sync_status(m);
}

// Renumbering of every mesh: live vertices and elements in ascending slot
// order take consecutive ids (adjacency keeps its order: the map is monotone).
// The final renumbering of a call, or one that finds many dead slots, moves
// the live slots together (compaction); the others leave every slot in place
// and record the new vertex ids (only the priorities read id values; every
// other use of an id is an order, which both numberings share).
int renumber(MeshSet& m, bool final) {
  Work& w = m.w;
  scan_alive_vertices(m.S, w.vscan, m.S.vused, m.scan, m.st, m.stream);
  scan_alive_elements(m.S, w.escan, m.S.eused, m.scan, m.st, m.stream);
  int* tot = w.counts + CN_NUM;
  int* changed = w.counts + CN_RENUM;
  cudaMemsetAsync(changed, 0, sizeof(int), m.stream);
  PM_LAUNCH(k_mesh_totals, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, w.vscan, w.escan, tot,
            changed);
  // compaction into the second buffer set (skipped on the device when no
  // slot died); the host swaps the sets afterwards
  auto compact = [&] {
    // the second buffer's flags must read "dead" beyond the new counts
    cudaMemsetAsync(m.B.vflag, 0, m.S.vslots, m.stream);
    PM_LAUNCH(k_renum_v, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, m.B, w.vscan, w.escan,
              changed);
    PM_LAUNCH(k_renum_e, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, m.B, w.vscan, w.escan,
              changed);
    PM_LAUNCH(k_set_sizes, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, tot);
  };
  if (final) compact();  // queued before the read-back: one synchronisation
  cudaMemcpyAsync(m.hcounts, tot, 2 * m.nmesh * sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(m.hcounts + 2 * m.nmesh, changed, sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  int err = sync_status(m);
  if (err) return err;
  if (!m.hcounts[2 * m.nmesh]) return PM_OK;  // no dead slot: every id stays
  if (!final) {
    long long vdead = 0, edead = 0;
    for (int i = 0; i < m.nmesh; ++i) {
      vdead += m.nv[i] - m.hcounts[2 * i];
      edead += m.ne[i] - m.hcounts[2 * i + 1];
    }
    if (8 * vdead <= m.S.vused && 8 * edead <= m.S.eused) {
      m.S.lid = m.lidbuf;
      m.S.voff = m.voffbuf;
      PM_LAUNCH(k_renum_ids, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, w.vscan, tot,
                m.lidbuf, m.voffbuf);
      return PM_OK;
    }
    compact();
  }
  for (int i = 0; i < m.nmesh; ++i) {
    m.nv[i] = m.hcounts[2 * i];
    m.ne[i] = m.hcounts[2 * i + 1];
  }
  std::swap(m.S.xy, m.B.xy);
  std::swap(m.S.M, m.B.M);
  std::swap(m.S.vflag, m.B.vflag);
  std::swap(m.S.EN, m.B.EN);
  std::swap(m.S.qK, m.B.qK);
  std::swap(m.S.NN, m.B.NN);
  std::swap(m.S.NNlen, m.B.NNlen);
  std::swap(m.S.NE, m.B.NE);
  std::swap(m.S.NElen, m.B.NElen);
  std::swap(m.S.touch, m.B.touch);
  std::swap(m.S.ntouch, m.B.ntouch);
  std::swap(m.S.evc, m.B.evc);
  std::swap(m.S.evs, m.B.evs);
  std::swap(m.S.evm, m.B.evm);
  std::swap(m.S.evr, m.B.evr);
  m.S.lid = m.S.voff = nullptr;  // ids are the slot offsets again
  set_used(m);
  return PM_OK;
}

// Compacted, canonically rotated copy of mesh `mesh` into device buffers
// (each may be null).  Writes the live counts.
int compact_out(MeshSet& m, int mesh, double* xy, int32_t* tri, double* mt, int* nv_out,
                int* ne_out) {
  Work& w = m.w;
  scan_alive_vertices(m.S, w.vscan, m.S.vused, m.scan, m.st, m.stream);
  scan_alive_elements(m.S, w.escan, m.S.eused, m.scan, m.st, m.stream);
  int* tot = w.counts + CN_NUM;
  PM_LAUNCH(k_mesh_totals, (m.nmesh + 127) / 128, 128, 0, m.stream, m.S, w.vscan, w.escan, tot,
            (int*)nullptr);
  if (xy || mt)
    PM_LAUNCH(k_out_v, grid_for(m, m.nv[mesh]), BLOCK, 0, m.stream, m.S, mesh, w.vscan, xy, mt);
  if (tri)
    PM_LAUNCH(k_out_e, grid_for(m, m.ne[mesh]), BLOCK, 0, m.stream, m.S, mesh, w.vscan, w.escan,
              tri);
  cudaMemcpyAsync(m.hcounts, tot, 2 * m.nmesh * sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  int err = sync_status(m);
  if (err) return err;
  *nv_out = m.hcounts[2 * mesh];
  *ne_out = m.hcounts[2 * mesh + 1];
  return PM_OK;
}

// Compacted, canonically rotated copy of every mesh of the set, one after
// the other in mesh order, into device buffers (each may be null).  Writes
// each mesh's live counts into nv_out[nmesh] and ne_out[nmesh].
int compact_out_set(MeshSet& m, double* xy, int32_t* tri, double* mt, int* nv_out, int* ne_out) {
  Work& w = m.w;
  const int n = m.nmesh;
  scan_alive_vertices(m.S, w.vscan, m.S.vused, m.scan, m.st, m.stream);
  scan_alive_elements(m.S, w.escan, m.S.eused, m.scan, m.st, m.stream);
  int* tot = w.counts + CN_NUM;
  PM_LAUNCH(k_mesh_totals, (n + 127) / 128, 128, 0, m.stream, m.S, w.vscan, w.escan, tot,
            (int*)nullptr);
  if (xy || mt || tri) {
    PM_LAUNCH(k_out_prefix, 1, 1024, 0, m.stream, n, (const int*)tot, m.S.tab.pre);
    if (xy || mt)
      PM_LAUNCH(k_out_v_set, grid_for(m, m.S.vused), BLOCK, 0, m.stream, m.S, w.vscan, xy, mt);
    if (tri)
      PM_LAUNCH(k_out_e_set, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, w.vscan, w.escan,
                tri);
  }
  cudaMemcpyAsync(m.hcounts, tot, 2 * n * sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  int err = sync_status(m);
  if (err) return err;
  for (int i = 0; i < n; ++i) {
    nv_out[i] = m.hcounts[2 * i];
    ne_out[i] = m.hcounts[2 * i + 1];
  }
  return PM_OK;
}

// Capacity for the adaptation ahead, in one growth: while adapting, a mesh
// holds at most about 2.2 times the larger of its element count and the
// element count its metric asks for (refinement overshoots before the
// collapses that follow), so every mesh below 2.5 times the estimate grows
// now, together, instead of round after round of refinement.
int presize(MeshSet& m) {
  const int n = m.nmesh;
  double* est = m.w.gains;  // scratch: no evaluation is kept across calls
  cudaMemsetAsync(est, 0, n * sizeof(double), m.stream);
  PM_LAUNCH(k_estimate, grid_for(m, m.S.eused), BLOCK, 0, m.stream, m.S, est);
  std::vector<double> h(n);
  cudaError_t e = cudaMemcpyAsync(h.data(), est, n * sizeof(double), cudaMemcpyDeviceToHost,
                                  m.stream);
  if (!e) e = cudaStreamSynchronize(m.stream);
  if (e) {
    set_last_error(std::string("estimating sizes: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  std::vector<int> vcap = m.vcap, ecap = m.ecap;
  bool need = false;
  long long vt = 0, et = 0;
  for (int i = 0; i < n; ++i) {
    const double ne_est = 4.0 / std::sqrt(3.0) * h[i];
    const double want_e = 2.5 * std::max(ne_est, (double)m.ne[i]);
    if (std::isfinite(want_e) && want_e > ecap[i] && want_e < (double)(1 << 29)) {
      ecap[i] = (int)want_e + 64;
      vcap[i] = std::max(vcap[i], (int)(0.6 * want_e) + 64);
      need = true;
    }
    vt += vcap[i];
    et += ecap[i];
  }
  if (!need || vt >= (1LL << 31) - 4 || et >= (1LL << 31) - 4) return PM_OK;
  e = grow(m, vcap, ecap, m.S.W);
  if (e) {
    set_last_error(std::string("growing mesh storage: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
  }
  return PM_OK;
}

}  // namespace pm
