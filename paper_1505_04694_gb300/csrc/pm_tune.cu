// Launch shapes of the operators and the tuning cache.
//
// The operators' one-kernel-per-phase rounds run grid-stride loops over
// their worklists; how many threads a block has and how many blocks an SM
// takes set how much of a list each thread walks (the worklist chunk).
// Below a list size the rounds of collapses, flips and smoothing run inside
// one persistent launch instead (small rounds are bound by launch and
// synchronisation latency).  None of these choices changes any result: they
// only decide which thread does which item and in which launch.  The GPU
// counterpart of the paper's load balancing (Sec. 3.5: work-stealing for
// loops) is hardware block scheduling over these grids; the tuner picks the
// shapes per operator by measurement.
//
// A tuning cache is a JSON file written by the package's autotuner:
//   {"format": 1, "entries": {"<GPU name>|<build id>": {"block": [4 ints],
//    "blocks_per_sm": [4 ints], "rounds_limit": [3 ints],
//    "rounds_blocks_per_sm": [3 ints], "fuse_limit": [2 ints], ...}}}
// An entry applies only to the GPU model and the library build it was
// measured on.
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "pm_internal.cuh"

#ifndef PM_BUILD_ID
#define PM_BUILD_ID "unversioned"
#endif

namespace pm {

namespace {

constexpr Tuning kDefaults = {{128, 128, 128, 128}, {16, 16, 16, 16}, {131072, 131072, 131072},
                               {1, 1, 1}, {0, 1 << 30}};

std::mutex g_tmu;
Tuning g_tune = kDefaults;
std::string g_source = "default";
bool g_auto_done = false;

bool valid(const Tuning& t) {
  for (int i = 0; i < 4; ++i) {
    if (t.block[i] != 64 && t.block[i] != 128 && t.block[i] != 256) return false;
    if (t.blocks_per_sm[i] < 1 || t.blocks_per_sm[i] > 32) return false;
  }
  for (int i = 0; i < 3; ++i) {
    if (t.rounds_limit[i] < 0 || t.rounds_limit[i] > (1 << 30)) return false;
    if (t.rounds_blocks_per_sm[i] < 1 || t.rounds_blocks_per_sm[i] > 2) return false;
  }
  for (int i = 0; i < 2; ++i)
    if (t.fuse_limit[i] < 0 || t.fuse_limit[i] > (1 << 30)) return false;
  return true;
}

// The text between the brace that opens after position `from` and its
// matching brace (strings skipped); empty when there is none.
std::string object_after(const std::string& s, size_t from) {
  size_t a = s.find('{', from);
  if (a == std::string::npos) return "";
  int depth = 0;
  bool str = false;
  for (size_t i = a; i < s.size(); ++i) {
    char ch = s[i];
    if (str) {
      if (ch == '\\') ++i;
      else if (ch == '"') str = false;
      continue;
    }
    if (ch == '"') str = true;
    else if (ch == '{') ++depth;
    else if (ch == '}' && --depth == 0) return s.substr(a, i - a + 1);
  }
  return "";
}

// The integer array of key `name` in object text `o`: exactly n entries.
bool int_array(const std::string& o, const char* name, int* out, int n) {
  std::string key = std::string("\"") + name + "\"";
  size_t p = o.find(key);
  if (p == std::string::npos) return false;
  p = o.find(':', p + key.size());
  if (p == std::string::npos) return false;
  p = o.find_first_not_of(" \t\r\n", p + 1);
  if (p == std::string::npos || o[p] != '[') return false;
  ++p;
  for (int i = 0; i < n; ++i) {
    char* end = nullptr;
    long v = std::strtol(o.c_str() + p, &end, 10);
    if (end == o.c_str() + p) return false;
    out[i] = (int)v;
    p = end - o.c_str();
    p = o.find_first_not_of(" \t\r\n", p);
    if (p == std::string::npos) return false;
    if (i + 1 < n) {
      if (o[p] != ',') return false;
      ++p;
    } else if (o[p] != ']') {
      return false;
    }
  }
  return true;
}

pm_status load_locked(const char* path, const char* gpu_name) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return PM_ERR_INVALID_ARG;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
  std::fclose(f);
  const std::string key = std::string("\"") + gpu_name + "|" + PM_BUILD_ID + "\"";
  size_t p = text.find(key);
  if (p == std::string::npos) return PM_ERR_INVALID_ARG;
  std::string o = object_after(text, p + key.size());
  Tuning t;
  if (o.empty() || !int_array(o, "block", t.block, 4) ||
      !int_array(o, "blocks_per_sm", t.blocks_per_sm, 4) ||
      !int_array(o, "rounds_limit", t.rounds_limit, 3) ||
      !int_array(o, "rounds_blocks_per_sm", t.rounds_blocks_per_sm, 3) ||
      !int_array(o, "fuse_limit", t.fuse_limit, 2) || !valid(t))
    return PM_ERR_INVALID_ARG;
  g_tune = t;
  g_source = std::string("cache ") + path;
  return PM_OK;
}

std::string device_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  return p.name;
}

}  // namespace

Tuning tuning() {
  std::lock_guard<std::mutex> lk(g_tmu);
  return g_tune;
}

// First mesh of the process: the first of these caches that holds an entry
// for this GPU and build applies -- the file named by PM_TUNING_CACHE,
// tuning.json beside the library, tuning.json in the directory above it
// (the package's own cache); otherwise the defaults stay.
void tuning_autoload() {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (g_auto_done) return;
  g_auto_done = true;
  const std::string name = device_name();
  if (name.empty()) return;
  if (const char* env = std::getenv("PM_TUNING_CACHE")) {
    if (load_locked(env, name.c_str()) == PM_OK) return;
  }
  Dl_info info;
  if (!dladdr((void*)&tuning_autoload, &info) || !info.dli_fname) return;
  std::string dir = info.dli_fname;
  size_t slash = dir.rfind('/');
  dir = slash == std::string::npos ? std::string(".") : dir.substr(0, slash);
  if (load_locked((dir + "/tuning.json").c_str(), name.c_str()) == PM_OK) return;
  load_locked((dir + "/../tuning.json").c_str(), name.c_str());
}

}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_set_tuning(const pm_tuning* t) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_auto_done = true;  // an explicit choice is not replaced by the cache
  if (!t) {
    g_tune = kDefaults;
    g_source = "default";
    return PM_OK;
  }
  Tuning n;
  std::memcpy(n.block, t->block, sizeof n.block);
  std::memcpy(n.blocks_per_sm, t->blocks_per_sm, sizeof n.blocks_per_sm);
  std::memcpy(n.rounds_limit, t->rounds_limit, sizeof n.rounds_limit);
  std::memcpy(n.rounds_blocks_per_sm, t->rounds_blocks_per_sm, sizeof n.rounds_blocks_per_sm);
  std::memcpy(n.fuse_limit, t->fuse_limit, sizeof n.fuse_limit);
  if (!valid(n)) return PM_ERR_INVALID_ARG;
  g_tune = n;
  g_source = "set";
  return PM_OK;
}

pm_status pm_get_tuning(pm_tuning* t) {
  if (!t) return PM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tmu);
  std::memcpy(t->block, g_tune.block, sizeof t->block);
  std::memcpy(t->blocks_per_sm, g_tune.blocks_per_sm, sizeof t->blocks_per_sm);
  std::memcpy(t->rounds_limit, g_tune.rounds_limit, sizeof t->rounds_limit);
  std::memcpy(t->rounds_blocks_per_sm, g_tune.rounds_blocks_per_sm, sizeof t->rounds_blocks_per_sm);
  std::memcpy(t->fuse_limit, g_tune.fuse_limit, sizeof t->fuse_limit);
  return PM_OK;
}

const char* pm_tuning_source(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  static thread_local std::string copy;
  copy = g_source;
  return copy.c_str();
}

pm_status pm_tuning_load(const char* path, const char* gpu_name) {
  if (!path) return PM_ERR_INVALID_ARG;
  std::string name = gpu_name ? std::string(gpu_name) : device_name();
  if (name.empty()) return PM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tmu);
  g_auto_done = true;
  return load_locked(path, name.c_str());
}

const char* pm_build_id(void) { return PM_BUILD_ID; }

}  // extern "C"
