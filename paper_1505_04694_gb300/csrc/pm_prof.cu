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
std::vector<ProfEvent> g_pool;
size_t g_used = 0;

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
  }
  return PM_OK;
}

pm_status pm_profile_read(double* total_ms, int64_t* launches) {
  if (!total_ms || !launches) return PM_ERR_INVALID_ARG;
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
