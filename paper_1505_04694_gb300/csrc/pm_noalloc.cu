// pm_quality_arrays_noalloc_dev: the quality sum and its gradient on plain
// device arrays (same computation as pm_quality_arrays_dev) without any
// device allocation during the call.
//
// Some callers cannot allocate device memory when they call in: a framework
// that has already reserved the device's memory for its own caching
// allocator, a latency-bound loop that cannot afford an allocation (or the
// synchronisation one may imply), or a program that forbids allocation after
// start-up.  For them every temporary lives in one fixed array compiled into
// this library (kScratchBytes below, about 9.6 MB): each GPU that loads the
// library keeps it until the process exits.  The sizes it admits are
// kMaxElements elements and kMaxVertices vertices; larger inputs are refused.
//
// All calls share the array and it keeps the last call's contents, so the
// parts that must start at zero are cleared by each call.  Two calls that
// overlap on the GPU (for example on two streams) race on the array; order
// them on one stream or synchronise between them.
#include <mutex>

#include "pm_internal.cuh"

namespace pm {

namespace {

constexpr int kMaxElements = 65536;
constexpr int kMaxVertices = 65536;
constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

struct NaGrad {
  double g[15];
};

// byte offsets inside the array (each a multiple of 256)
constexpr size_t round256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffQel = 0;
constexpr size_t kOffGrad = round256(kOffQel + sizeof(double) * kMaxElements);
constexpr size_t kOffPart = round256(kOffGrad + sizeof(NaGrad) * kMaxElements);
constexpr size_t kOffCnt = round256(kOffPart + sizeof(double) * kRedBlocks);
constexpr size_t kOffFill = round256(kOffCnt + sizeof(int) * (kMaxVertices + 1));
constexpr size_t kOffOff = round256(kOffFill + sizeof(int) * (kMaxVertices + 1));
constexpr size_t kOffCol = round256(kOffOff + sizeof(int) * (kMaxVertices + 1));
constexpr size_t kScanTiles = (kMaxVertices + 1 + 2047) / 2048;
constexpr size_t kOffScan = round256(kOffCol + sizeof(int) * 3 * kMaxElements);
constexpr size_t kOffTicket = round256(kOffScan + sizeof(unsigned long long) * kScanTiles);
constexpr size_t kOffStatus = round256(kOffTicket + sizeof(int));
constexpr size_t kScratchBytes = round256(kOffStatus + sizeof(DevStatus));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host side: the array's device address, looked up once per device.
struct DeviceScratch {
  unsigned char* base = nullptr;
  ScanWork scan;
};
std::mutex g_mu;
DeviceScratch g_dev[64];

__device__ __forceinline__ VD na_vd(const double* xy, const double* m, int v) {
  return VD{xy[2 * v], xy[2 * v + 1], m[3 * v], m[3 * v + 1], m[3 * v + 2]};
}

__global__ void k_na_clear(int* cnt, int* fill, int nv, DevStatus* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nv; i += gridDim.x * blockDim.x) {
    cnt[i] = 0;
    fill[i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->err = 0;
    st->overflow = 0;
    st->maxdeg = 0;
  }
}

// An element with a vertex id outside [0, nv) records PM_ERR_INVALID_MESH
// and contributes NaN (nothing is read through a bad id).
__global__ void k_na_elem(const double* xy, const double* m, const int* tri, int ne, int nv,
                          double* qel, NaGrad* eg, DevStatus* st) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x) {
    int a = tri[3 * K], b = tri[3 * K + 1], c = tri[3 * K + 2];
    if ((unsigned)a >= (unsigned)nv || (unsigned)b >= (unsigned)nv || (unsigned)c >= (unsigned)nv) {
      set_err(st, PM_ERR_INVALID_MESH);
      qel[K] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    double g[3][5];
    qel[K] = quality_grad_c(a, b, c, na_vd(xy, m, a), na_vd(xy, m, b), na_vd(xy, m, c), g);
    if (eg) {
      NaGrad out;
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 5; ++j) out.g[5 * k + j] = g[k][j];
      eg[K] = out;
    }
  }
}

__global__ void k_na_count(const int* tri, int ne, int nv, int* cnt) {
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x)
    for (int i = 0; i < 3; ++i) {
      int v = tri[3 * K + i];
      if ((unsigned)v < (unsigned)nv) atomicAdd(cnt + v, 1);
    }
}

// Nothing is written after a device error (the offsets may be stale from an
// earlier call) and no entry leaves its vertex's range of the array.
__global__ void k_na_fill(const int* tri, int ne, int nv, const int* off, int* fill, int* col,
                          const DevStatus* st) {
  if (st->err) return;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < ne; K += gridDim.x * blockDim.x)
    for (int i = 0; i < 3; ++i) {
      int v = tri[3 * K + i];
      if ((unsigned)v >= (unsigned)nv) continue;
      int p = atomicAdd(fill + v, 1);
      if (off[v] + p < off[v + 1]) col[off[v] + p] = 3 * K + i;
    }
}

// Per vertex: sort its corner list (ascending element id) and sum the
// contributions in that order.  After a device error every output is NaN.
__global__ void k_na_gather(const int* off, int* col, const NaGrad* eg, int nv, double* dxy,
                            double* dm, const DevStatus* st) {
  const bool bad = st->err != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (bad) {
      for (int j = 0; j < 5; ++j) acc[j] = nan;
    } else {
      int a = off[v], b = off[v + 1];
      for (int k = a + 1; k < b; ++k) {
        int x = col[k];
        int j = k - 1;
        while (j >= a && col[j] > x) {
          col[j + 1] = col[j];
          --j;
        }
        col[j + 1] = x;
      }
      for (int k = a; k < b; ++k) {
        const double* g = eg[col[k] / 3].g + 5 * (col[k] % 3);
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

__global__ void k_na_sum1(const double* x, int n, double* part) {
  __shared__ double sh[kRedThreads];
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

__global__ void k_na_sum2(const double* part, double* out) {
  __shared__ double sh[kRedBlocks];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

int na_grid(long long n) {
  long long g = (n + 127) / 128;
  return (int)(g < 1 ? 1 : (g > 2432 ? 2432 : g));
}

}  // namespace

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_quality_arrays_noalloc_dev(const double* xy, const double* M, int32_t nv,
                                                   const int32_t* tri, int32_t ne, double* q_sum,
                                                   double* dxy, double* dm, void* stream) {
  if (!xy || !M || (!tri && ne > 0) || !q_sum || nv < 1 || ne < 0) {
    set_last_error("need xy, m, tri, q_sum, nv >= 1, ne >= 0");
    return PM_ERR_INVALID_ARG;
  }
  if (ne > kMaxElements || nv > kMaxVertices) {
    set_last_error("pm_quality_arrays_noalloc_dev handles at most 65536 elements and 65536 "
                   "vertices; use pm_quality_arrays_dev for larger meshes");
    return PM_ERR_CAPACITY;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("no current CUDA device");
    return PM_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  ScanWork* sw = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch& d = g_dev[dev];
    if (!d.base) {
      // one-time set-up on this device (the device is current here)
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        set_last_error(std::string("locating the scratch array: ") + cudaGetErrorString(e));
        return PM_ERR_CUDA;
      }
      d.base = (unsigned char*)p;
      d.scan.state = (unsigned long long*)(d.base + kOffScan);
      d.scan.ticket = (int*)(d.base + kOffTicket);
      d.scan.tiles_cap = (int)kScanTiles;
    }
    base = d.base;
    sw = &d.scan;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* qel = (double*)(base + kOffQel);
  NaGrad* eg = (NaGrad*)(base + kOffGrad);
  double* part = (double*)(base + kOffPart);
  int* cnt = (int*)(base + kOffCnt);
  int* fill = (int*)(base + kOffFill);
  int* off = (int*)(base + kOffOff);
  int* col = (int*)(base + kOffCol);
  DevStatus* st = (DevStatus*)(base + kOffStatus);
  bool grad = dxy || dm;
  PM_LAUNCH(k_na_clear, na_grid(nv + 1), 128, 0, s, cnt, fill, nv, st);
  PM_LAUNCH(k_na_elem, na_grid(ne), 128, 0, s, xy, M, tri, ne, nv, qel, grad ? eg : nullptr, st);
  PM_LAUNCH(k_na_sum1, kRedBlocks, kRedThreads, 0, s, qel, ne, part);
  PM_LAUNCH(k_na_sum2, 1, kRedBlocks, 0, s, part, q_sum);
  if (grad) {
    PM_LAUNCH(k_na_count, na_grid(ne), 128, 0, s, tri, ne, nv, cnt);
    {
      // the scan's epoch counter is shared by all calls on this device
      std::lock_guard<std::mutex> lk(g_mu);
      scan_exclusive(cnt, off, nv, *sw, st, s);
    }
    PM_LAUNCH(k_na_fill, na_grid(ne), 128, 0, s, tri, ne, nv, (const int*)off, fill, col,
              (const DevStatus*)st);
    PM_LAUNCH(k_na_gather, na_grid(nv), 128, 0, s, (const int*)off, col, (const NaGrad*)eg, nv,
              dxy, dm, (const DevStatus*)st);
  }
  cudaError_t e = cudaGetLastError();
  // the status word of this call (a copy into pageable host memory returns
  // once the stream has reached it)
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(std::string("CUDA: ") + cudaGetErrorString(e));
    return PM_ERR_CUDA;
  }
  if (h.err == PM_ERR_INVALID_MESH) set_last_error("vertex id outside [0, nv) in tri");
  if (h.err == PM_ERR_TIMEOUT) set_last_error("the gradient's scan gave up waiting");
  return (pm_status)h.err;
}
