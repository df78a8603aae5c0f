// Element quality functional (Sec. 2.2, Vasilevskii et al.) summed over a
// mesh, and its gradient with respect to vertex coordinates and metric
// entries (hand-written reverse mode, see quality_grad_c).
//
// Two passes: one thread per element writes q and the 15 partial derivatives
// of its three vertices; one thread per vertex then sums its elements'
// contributions in ascending element id, so the result does not depend on
// thread timing.  The sum of q is a fixed-shape two-level reduction.
#include <algorithm>

#include "pm_internal.cuh"

namespace pm {

namespace {

constexpr int RED_BLOCKS = 256;
constexpr int RED_THREADS = 256;

struct EGrad {
  double g[15];
};

__global__ void k_elem_qgrad_store(Store S, int mesh, double* qel, EGrad* eg) {
  int vb = S.tab.vbase[mesh], eb = S.tab.ebase[mesh], ne = S.tab.ne[mesh];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ne; l += gridDim.x * blockDim.x) {
    int4 e = S.EN[eb + l];
    if (!e.w) {
      qel[l] = 0.0;
      continue;
    }
    double g[3][5];
    double q = quality_grad_c(e.x, e.y, e.z, load_vd(S, vb + e.x), load_vd(S, vb + e.y),
                              load_vd(S, vb + e.z), g);
    qel[l] = q;
    if (eg) {
      EGrad out;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 5; ++j) out.g[5 * k + j] = g[k][j];
      eg[l] = out;
    }
  }
}

__global__ void k_vgather_store(Store S, int mesh, const EGrad* eg, double* dxy, double* dm) {
  int vb = S.tab.vbase[mesh], eb = S.tab.ebase[mesh], nv = S.tab.nv[mesh];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nv; l += gridDim.x * blockDim.x) {
    int s = vb + l;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (S.vflag[s] & VF_ALIVE) {
      const int* ne = S.NE + (size_t)s * S.W;
      int nel = S.NElen[s];
      for (int k = 0; k < nel; ++k) {
        int K = ne[k];
        int4 e = S.EN[eb + K];
        int i = (e.x == l) ? 0 : (e.y == l) ? 1 : 2;
        const double* g = eg[K].g + 5 * i;
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] = acc[j] + g[j];
      }
    }
    if (dxy) {
      dxy[2 * l] = acc[0];
      dxy[2 * l + 1] = acc[1];
    }
    if (dm) {
      dm[3 * l] = acc[2];
      dm[3 * l + 1] = acc[3];
      dm[3 * l + 2] = acc[4];
    }
  }
}

// ---- arrays (no mesh handle) ----------------------------------------------------

__device__ __forceinline__ VD arr_vd(const double* xy, const double* m, int v) {
  return VD{xy[2 * v], xy[2 * v + 1], m[3 * v], m[3 * v + 1], m[3 * v + 2]};
}

// An element with a vertex id outside [0, nv) records PM_ERR_INVALID_MESH
// and contributes NaN (nothing is read through a bad id).
__global__ void k_elem_qgrad_arr(const double* xy, const double* m, const int* tri, int ne,
                                 int nv, double* qel, EGrad* eg, DevStatus* st) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    int a = tri[3 * K], b = tri[3 * K + 1], c = tri[3 * K + 2];
    if ((unsigned)a >= (unsigned)nv || (unsigned)b >= (unsigned)nv || (unsigned)c >= (unsigned)nv) {
      set_err(st, PM_ERR_INVALID_MESH);
      qel[K] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    double g[3][5];
    double q = quality_grad_c(a, b, c, arr_vd(xy, m, a), arr_vd(xy, m, b), arr_vd(xy, m, c), g);
    qel[K] = q;
    if (eg) {
      EGrad out;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 5; ++j) out.g[5 * k + j] = g[k][j];
      eg[K] = out;
    }
  }
}

// Corners per vertex (ids outside [0, nv) are skipped: the element pass has
// recorded them).
__global__ void k_corner_count(const int* tri, int ne, int nv, int* cnt) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x)
    for (int i = 0; i < 3; ++i) {
      int v = tri[3 * K + i];
      if ((unsigned)v < (unsigned)nv) atomicAdd(cnt + v, 1);
    }
}

// Corner list per vertex: entry = 3 * element + corner position; nothing is
// written after a device error (the offsets may be unwritten) and no entry
// leaves its vertex's range.
__global__ void k_corner_fill(const int* tri, int ne, int nv, const int* off, int* fill, int* col,
                              const DevStatus* st) {
  if (st->err) return;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    for (int i = 0; i < 3; ++i) {
      int v = tri[3 * K + i];
      if ((unsigned)v >= (unsigned)nv) continue;
      int p = atomicAdd(fill + v, 1);
      if (off[v] + p < off[v + 1]) col[off[v] + p] = 3 * K + i;
    }
  }
}

// Per vertex: its corners in ascending element id, contributions summed in
// that order.  After a device error every output entry is NaN.
__global__ void k_vgather_arr(const int* off, int* col, const EGrad* eg, int nv, double* dxy,
                              double* dm, const DevStatus* st) {
  const bool bad = st->err != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (bad) {
#pragma unroll
      for (int j = 0; j < 5; ++j) acc[j] = nan;
    } else {
      int a = off[v], b = off[v + 1];
      for (int k = a + 1; k < b; ++k) {  // ascending element id
        int x = col[k];
        int j = k - 1;
        while (j >= a && col[j] > x) {
          col[j + 1] = col[j];
          --j;
        }
        col[j + 1] = x;
      }
      for (int k = a; k < b; ++k) {
        int x = col[k];
        const double* g = eg[x / 3].g + 5 * (x % 3);
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] = acc[j] + g[j];
      }
    }
    if (dxy) {
      dxy[2 * v] = acc[0];
      dxy[2 * v + 1] = acc[1];
    }
    if (dm) {
      dm[3 * v] = acc[2];
      dm[3 * v + 1] = acc[3];
      dm[3 * v + 2] = acc[4];
    }
  }
}

// ---- deterministic sum -------------------------------------------------------------

__global__ void k_sum_stage1(const double* x, int n, double* part) {
  __shared__ double sh[RED_THREADS];
  long long chunk = ((long long)n + gridDim.x - 1) / gridDim.x;
  long long a = chunk * blockIdx.x, b = a + chunk < n ? a + chunk : n;
  double s = 0.0;
  for (long long i = a + threadIdx.x; i < b; i += blockDim.x) s = s + x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_stage2(const double* part, int n, double* out) {
  __shared__ double sh[RED_BLOCKS];
  sh[threadIdx.x] = threadIdx.x < n ? part[threadIdx.x] : 0.0;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

void dsum(const double* x, int n, double* part, double* out, cudaStream_t s) {
  PM_LAUNCH(k_sum_stage1, RED_BLOCKS, RED_THREADS, 0, s, x, n, part);
  PM_LAUNCH(k_sum_stage2, 1, RED_BLOCKS, 0, s, part, RED_BLOCKS, out);
}

int gridn(long long n) {
  long long g = (n + 127) / 128;
  return (int)std::max<long long>(1, std::min<long long>(g, 152 * 16));
}

}  // namespace

// Quality sum and gradient of mesh 0 of the set, written to host arrays
// indexed by vertex slot (dxy[2*nv], dm[3*nv]; each may be null).
int quality_mesh(MeshSet& m, double* qsum_host, double* dxy_host, double* dm_host) {
  cudaStream_t s = m.stream;
  int ne = m.ne[0], nv = m.nv[0];
  bool grad = dxy_host || dm_host;
  double *qel = nullptr, *part = nullptr, *out = nullptr, *dxy = nullptr, *dm = nullptr;
  EGrad* eg = nullptr;
  cudaError_t e = cudaMallocAsync(&qel, std::max(ne, 1) * sizeof(double), s);
  if (!e) e = cudaMallocAsync(&part, (RED_BLOCKS + 1) * sizeof(double), s);
  if (!e && grad) e = cudaMallocAsync(&eg, std::max(ne, 1) * sizeof(EGrad), s);
  if (!e && grad) e = cudaMallocAsync(&dxy, std::max(nv, 1) * 2 * sizeof(double), s);
  if (!e && grad) e = cudaMallocAsync(&dm, std::max(nv, 1) * 3 * sizeof(double), s);
  int status = PM_OK;
  if (e) {
    set_last_error(std::string("quality workspace: ") + cudaGetErrorString(e));
    status = PM_ERR_OOM;
  } else {
    out = part + RED_BLOCKS;
    PM_LAUNCH(k_elem_qgrad_store, gridn(ne), 128, 0, s, m.S, 0, qel, eg);
    dsum(qel, ne, part, out, s);
    if (grad) PM_LAUNCH(k_vgather_store, gridn(nv), 128, 0, s, m.S, 0, eg, dxy, dm);
    cudaMemcpyAsync(qsum_host, out, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (dxy_host)
      cudaMemcpyAsync(dxy_host, dxy, nv * 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (dm_host) cudaMemcpyAsync(dm_host, dm, nv * 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  for (void* p : {(void*)qel, (void*)part, (void*)eg, (void*)dxy, (void*)dm})
    if (p) cudaFreeAsync(p, s);
  int err = sync_status(m);
  return status ? status : err;
}

// Quality sum (and gradient) on plain device arrays.  Temporaries come from
// one stream-ordered allocation; the call waits for its stream and returns
// the device status (PM_ERR_INVALID_MESH for a vertex id outside [0, nv),
// PM_ERR_TIMEOUT when the scan's bounded wait gave up; the outputs then hold
// NaN).
int quality_arrays(const double* xy, const double* mt, int nv, const int* tri, int ne,
                   double* qsum, double* dxy, double* dm, cudaStream_t s) {
  const bool grad = dxy || dm;
  const int tiles = scan_tiles(nv + 1);
  auto r256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_qel = r256(std::max(ne, 1) * sizeof(double));
  const size_t b_part = r256(RED_BLOCKS * sizeof(double));
  const size_t b_st = r256(sizeof(DevStatus));
  const size_t b_eg = grad ? r256(std::max(ne, 1) * sizeof(EGrad)) : 0;
  const size_t b_cnt = grad ? r256(2 * ((size_t)nv + 1) * sizeof(int)) : 0;
  const size_t b_off = grad ? r256(((size_t)nv + 1) * sizeof(int)) : 0;
  const size_t b_col = grad ? r256(std::max(3LL * ne, 1LL) * sizeof(int)) : 0;
  const size_t b_state = grad ? r256((size_t)tiles * sizeof(unsigned long long)) : 0;
  const size_t b_ticket = grad ? r256(sizeof(int)) : 0;
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, b_qel + b_part + b_st + b_eg + b_cnt + b_off +
                                                     b_col + b_state + b_ticket, s);
  if (e != cudaSuccess) {
    set_last_error(std::string("quality workspace: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
  }
  char* p = base;
  double* qel = (double*)p; p += b_qel;
  double* part = (double*)p; p += b_part;
  DevStatus* st = (DevStatus*)p; p += b_st;
  EGrad* eg = grad ? (EGrad*)p : nullptr; p += b_eg;
  int* cnt = (int*)p; p += b_cnt;
  int* off = (int*)p; p += b_off;
  int* col = (int*)p; p += b_col;
  ScanWork sw;
  sw.state = (unsigned long long*)p; p += b_state;
  sw.ticket = (int*)p;
  sw.tiles_cap = tiles;
  e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  if (!e && grad) e = cudaMemsetAsync(cnt, 0, 2 * ((size_t)nv + 1) * sizeof(int), s);
  if (!e && grad) e = cudaMemsetAsync(sw.state, 0, b_state, s);
  if (!e) {
    PM_LAUNCH(k_elem_qgrad_arr, gridn(ne), 128, 0, s, xy, mt, tri, ne, nv, qel, eg, st);
    dsum(qel, ne, part, qsum, s);
    if (grad) {
      int* fill = cnt + (nv + 1);
      PM_LAUNCH(k_corner_count, gridn(ne), 128, 0, s, tri, ne, nv, cnt);
      scan_exclusive(cnt, off, nv, sw, st, s);
      PM_LAUNCH(k_corner_fill, gridn(ne), 128, 0, s, tri, ne, nv, (const int*)off, fill, col,
                (const DevStatus*)st);
      PM_LAUNCH(k_vgather_arr, gridn(nv), 128, 0, s, (const int*)off, col, (const EGrad*)eg, nv,
                dxy, dm, (const DevStatus*)st);
    }
    e = cudaGetLastError();
  }
  DevStatus h{};
  if (!e) e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(std::string("CUDA: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  if (h.err == PM_ERR_INVALID_MESH) set_last_error("vertex id outside [0, nv) in tri");
  if (h.err == PM_ERR_TIMEOUT) set_last_error("the gradient's scan gave up waiting");
  return h.err;
}

}  // namespace pm
