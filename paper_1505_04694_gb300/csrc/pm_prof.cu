// Launch counting and per-kernel event timing for measurement.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

unsigned long long g_launches = 0;
bool g_prof_on = false;

namespace {

struct ProfEvent {
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::string g_filter;
unsigned long long* g_work = nullptr;  // device counter of the profiled kernel's work
std::vector<ProfEvent> g_pool;
size_t g_used = 0;

// Eight independent chains per thread, each step one multiplication and one
// addition (the library is compiled without contraction): the FP64 pipe is
// the only limit.  `out` keeps the result alive.
__global__ void k_fp64_peak(int iters, double seed, double* out) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + j + threadIdx.x * 1e-3;
  const double m = 0.999999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = a[j] * m + c;
  }
  double t = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) t += a[j];
  if (t == 12345.678) out[0] = t;  // never true; keeps the chains
}

// Test support: out[i] = div3(x[i]), the quotient by three the quality
// functional uses for its means.
__global__ void k_selftest_div3(const double* x, double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = div3(x[i]);
}

// Test support: out[i] = exact orientation sign of points pts[6i .. 6i+5]
// = (px, py, qx, qy, rx, ry), the predicate every validity decision uses.
__global__ void k_selftest_orient(const double* pts, int* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double* t = pts + 6 * i;
    VD p{t[0], t[1], 0.0, 0.0, 0.0}, q{t[2], t[3], 0.0, 0.0, 0.0}, r{t[4], t[5], 0.0, 0.0, 0.0};
    out[i] = orient_sign(p, q, r);
  }
}

}  // namespace

int prof_begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_prof_on || g_filter.empty() || !std::strstr(name, g_filter.c_str())) return -1;
  if (g_used == g_pool.size()) {
    ProfEvent e;
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return -1;
    g_pool.push_back(e);
  }
  int slot = (int)g_used++;
  cudaEventRecord(g_pool[slot].a, s);
  return slot;
}

unsigned long long* prof_work(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_prof_on || g_filter.empty() || !std::strstr(name, g_filter.c_str())) return nullptr;
  return g_work;
}

void prof_end(int slot, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_pool[slot].b, s);
}

}  // namespace pm

using namespace pm;

extern "C" {

uint64_t pm_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

pm_status pm_profile_enable(const char* kernel_substring) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_used = 0;
  if (!kernel_substring || !*kernel_substring) {
    g_prof_on = false;
    g_filter.clear();
  } else {
    g_prof_on = true;
    g_filter = kernel_substring;
    if (!g_work && cudaMalloc(&g_work, sizeof(unsigned long long)) != cudaSuccess) {
      g_work = nullptr;
      return PM_ERR_CUDA;
    }
    if (cudaMemset(g_work, 0, sizeof(unsigned long long)) != cudaSuccess) return PM_ERR_CUDA;
  }
  return PM_OK;
}

pm_status pm_fp64_peak(double* gops) {
  if (!gops) return PM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PM_ERR_CUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return PM_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    k_fp64_peak<<<blocks, threads>>>(iters, 1.0 + rep, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
  const double ops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *gops = ops / (best * 1e-3) / 1e9;
  return PM_OK;
}

pm_status pm_selftest_div3_dev(const double* x, double* out, int64_t n, void* stream) {
  if (!x || !out || n < 0) return PM_ERR_INVALID_ARG;
  if (n == 0) return PM_OK;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  PM_LAUNCH(k_selftest_div3, dim3((unsigned)blocks), dim3(256), 0, (cudaStream_t)stream, x, out,
            (long long)n);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

pm_status pm_selftest_orient_dev(const double* pts, int32_t* out, int64_t n, void* stream) {
  if (!pts || !out || n < 0) return PM_ERR_INVALID_ARG;
  if (n == 0) return PM_OK;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  PM_LAUNCH(k_selftest_orient, dim3((unsigned)blocks), dim3(256), 0, (cudaStream_t)stream, pts,
            out, (long long)n);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

pm_status pm_profile_read(double* total_ms, int64_t* launches, double* work) {
  if (!total_ms || !launches) return PM_ERR_INVALID_ARG;
  if (work) {
    unsigned long long wv = 0;
    if (g_work && cudaMemcpy(&wv, g_work, sizeof(wv), cudaMemcpyDeviceToHost) != cudaSuccess)
      return PM_ERR_CUDA;
    *work = (double)wv;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0.0;
  for (size_t i = 0; i < g_used; ++i) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_pool[i].b) != cudaSuccess) return PM_ERR_CUDA;
    if (cudaEventElapsedTime(&ms, g_pool[i].a, g_pool[i].b) != cudaSuccess) return PM_ERR_CUDA;
    t += ms;
  }
  *total_ms = t;
  *launches = (int64_t)g_used;
  return PM_OK;
}

}  // extern "C"
