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

__global__ void k_elem_qgrad_arr(const double* xy, const double* m, const int* tri, int ne,
                                 double* qel, EGrad* eg) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    int a = tri[3 * K], b = tri[3 * K + 1], c = tri[3 * K + 2];
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

__global__ void k_corner_count(const int* tri, int ne, int* cnt) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    atomicAdd(cnt + tri[3 * K], 1);
    atomicAdd(cnt + tri[3 * K + 1], 1);
    atomicAdd(cnt + tri[3 * K + 2], 1);
  }
}

// Corner list per vertex: entry = 3 * element + corner position.
__global__ void k_corner_fill(const int* tri, int ne, const int* off, int* fill, int* col) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    for (int i = 0; i < 3; ++i) {
      int v = tri[3 * K + i];
      int p = atomicAdd(fill + v, 1);
      col[off[v] + p] = 3 * K + i;
    }
  }
}

__global__ void k_vgather_arr(const int* off, int* col, const EGrad* eg, int nv, double* dxy,
                              double* dm) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
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
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = a; k < b; ++k) {
      int x = col[k];
      const double* g = eg[x / 3].g + 5 * (x % 3);
#pragma unroll
      for (int j = 0; j < 5; ++j) acc[j] = acc[j] + g[j];
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

// Quality sum (and gradient) on plain device arrays; stream-ordered, no
// synchronisation.  Temporary memory comes from the stream-ordered pool.
int quality_arrays(const double* xy, const double* mt, int nv, const int* tri, int ne,
                   double* qsum, double* dxy, double* dm, cudaStream_t s) {
  bool grad = dxy || dm;
  double *qel = nullptr, *part = nullptr;
  EGrad* eg = nullptr;
  int *cnt = nullptr, *off = nullptr, *col = nullptr;
  cudaError_t e = cudaMallocAsync(&qel, std::max(ne, 1) * sizeof(double), s);
  if (!e) e = cudaMallocAsync(&part, RED_BLOCKS * sizeof(double), s);
  if (!e && grad) e = cudaMallocAsync(&eg, std::max(ne, 1) * sizeof(EGrad), s);
  if (!e && grad) e = cudaMallocAsync(&cnt, (nv + 1) * sizeof(int) * 2, s);
  if (!e && grad) e = cudaMallocAsync(&off, (nv + 1) * sizeof(int), s);
  if (!e && grad) e = cudaMallocAsync(&col, std::max(3LL * ne, 1LL) * sizeof(int), s);
  int status = PM_OK;
  if (e) {
    set_last_error(std::string("quality workspace: ") + cudaGetErrorString(e));
    status = PM_ERR_OOM;
  } else {
    PM_LAUNCH(k_elem_qgrad_arr, gridn(ne), 128, 0, s, xy, mt, tri, ne, qel, eg);
    dsum(qel, ne, part, qsum, s);
    if (grad) {
      int* fill = cnt + (nv + 1);
      cudaMemsetAsync(cnt, 0, (nv + 1) * sizeof(int) * 2, s);
      PM_LAUNCH(k_corner_count, gridn(ne), 128, 0, s, tri, ne, cnt);
      ScanWork sw;
      cudaMallocAsync(&sw.state, (size_t)scan_tiles(nv + 1) * sizeof(unsigned long long), s);
      cudaMallocAsync(&sw.ticket, sizeof(int), s);
      cudaMemsetAsync(sw.state, 0, (size_t)scan_tiles(nv + 1) * sizeof(unsigned long long), s);
      DevStatus* st = nullptr;
      cudaMallocAsync(&st, sizeof(DevStatus), s);
      cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
      scan_exclusive(cnt, off, nv, sw, st, s);
      PM_LAUNCH(k_corner_fill, gridn(ne), 128, 0, s, tri, ne, off, fill, col);
      PM_LAUNCH(k_vgather_arr, gridn(nv), 128, 0, s, off, col, eg, nv, dxy, dm);
      cudaFreeAsync(sw.state, s);
      cudaFreeAsync(sw.ticket, s);
      cudaFreeAsync(st, s);
    }
  }
  for (void* p : {(void*)qel, (void*)part, (void*)eg, (void*)cnt, (void*)off, (void*)col})
    if (p) cudaFreeAsync(p, s);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess && !status) {
    set_last_error(std::string("CUDA: ") + cudaGetErrorString(le));
    status = PM_ERR_CUDA;
  }
  return status;
}

}  // namespace pm
