// Host-side structures of the library (one translation unit per subsystem
// shares these declarations).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "pm_common.cuh"

namespace pm {

constexpr int MAXW = 128;         // largest supported adjacency row (a vertex's degree)
constexpr int BLOCK = 128;        // threads per block of the round kernels

struct ScanWork {
  unsigned long long* state = nullptr;  // one word per tile
  int* ticket = nullptr;
  unsigned epoch = 0;
  int tiles_cap = 0;
};

int scan_tiles(int n);
void scan_exclusive(const int* in, int* out, int n, ScanWork& w, DevStatus* st, cudaStream_t s);
void scan_alive_vertices(const Store& S, int* out, int n, ScanWork& w, DevStatus* st,
                         cudaStream_t s);
void scan_alive_elements(const Store& S, int* out, int n, ScanWork& w, DevStatus* st,
                         cudaStream_t s);

// Per-round worklists and marks (slot-indexed scratch, sized with the store).
struct Work {
  int* D[2] = {nullptr, nullptr};  // dirty / pending lists (ping-pong)
  int* C = nullptr;                // candidates
  int* Sl = nullptr;               // independent set
  int* A = nullptr;                // vertices whose rows change (commit owners)
  int* P = nullptr;                // next-sweep list (smoothing)
  int* target = nullptr;           // collapse target (local id) per vertex
  int4* opA = nullptr;             // flip record (w, c, d, K1) per vertex
  int* opK2 = nullptr;
  double2* mvxy = nullptr;         // smoothing move per vertex
  double4* mvM = nullptr;
  int* dmark = nullptr;            // per-round stamps
  int* amark = nullptr;
  int* cmark = nullptr;
  int* smark = nullptr;
  int* pmark = nullptr;
  int* vcnt = nullptr;             // per-vertex counts (refine / renumber), vslots + 1
  int* vscan = nullptr;            // vslots + 1
  RowMask* vmask = nullptr;        // refine: marked NN entries
  int* ecnt = nullptr;             // per-element counts, eslots + 1
  int* escan = nullptr;
  int4* emid = nullptr;            // refine: midpoint ids per element edge
  int* elist = nullptr;            // refine: elements split this round, eslots
  int* clist = nullptr;            // refine: their children's slots, eslots
  int* E = nullptr;                // vertices evaluated in full this round
  int2* items = nullptr;           // flip candidates (vertex, edge slots) of this round
  double* gains = nullptr;         // gain of each (vertex, ball-element slot), vslots * W
  int2* items2 = nullptr;          // second wave list (vertex, candidate rank)
  int* cand = nullptr;             // collapse candidates of each vertex by (length, id), vslots * W
  int* ncand = nullptr;
  int* counts = nullptr;           // device counters (see CountIdx)
  int* cprop = nullptr;            // colouring: proposed colour per vertex slot
  int* cstamp = nullptr;           // colouring: round in which the slot was uncoloured
};

// The per-round counters sit between the two dirty-list counts so that one
// memset clears them together with the next round's list (zero_round).
enum CountIdx {
  CN_D0 = 0, CN_C = 1, CN_S = 2, CN_A = 3, CN_E = 4, CN_I = 5, CN_I2 = 6, CN_D1 = 7,
  CN_P = 8, CN_EL = 9, CN_CL = 10, CN_DONE = 11,
  CN_RES = 12,  // persistent rounds: rounds run, list index after, pass complete (3)
  CN_BAR = 15,  // persistent rounds: grid barrier arrivals
  CN_C2 = 16,   // persistent rounds: candidates of odd rounds
  CN_RENUM = 17,  // renumbering: 1 when some mesh's compaction is not the identity
  CN_NUM = 18
};
constexpr int cn_list(int i) { return i == 0 ? CN_D0 : CN_D1; }

// Everything the library keeps on the device for a set of meshes.
struct MeshSet {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nmesh = 0;
  // host mirror of the per-mesh table
  std::vector<int> vbase, vcap, ebase, ecap, nv, ne;
  std::vector<uint32_t> seed;
  std::vector<double> L_low, L_up, q_thresh;
  std::vector<int> select;  // PM_SELECT_* per mesh
  Store S{};          // device arrays (S.tab points into tabmem)
  Store B{};          // second buffer set for renumbering
  Work w{};
  ScanWork scan{};
  DevStatus* st = nullptr;     // device
  DevStatus* hst = nullptr;    // pinned host
  int* hcounts = nullptr;      // pinned host copy of w.counts
  unsigned long long* hops = nullptr;  // pinned: operation counts of three operators (3 * nmesh)
  char* hup = nullptr;                 // pinned: staging of the per-mesh table for upload_tab
  cudaEvent_t upev = nullptr;          // the last table upload has left the staging
  void* pinned = nullptr;      // slot of the process-wide pinned arena (hst, hcounts)
  bool pinned_own = false;     // slot too small: a private pinned allocation
  void* tabmem = nullptr;      // device block holding MeshTab arrays
  int* lidbuf = nullptr;       // S.lid and S.voff when in use (vslots, nmesh)
  int* voffbuf = nullptr;
  int tag = 0;                 // per-round tag (even); the round's change stamp is tag + 1
  // evaluations with tags at or below these are stale for that operator
  int lo_coarsen = 0, lo_swap = 0, lo_refine = 0;
  int num_sms = 152;
  bool qvalid = false;         // the element quality cache matches the current metric
  bool mesh_index_ok = false;  // S.tab.vmesh / emesh describe the current layout
  std::vector<void*> allocs;   // device allocations owned by the set
};

// ---- mesh storage (pm_mesh.cu) ----
cudaError_t set_alloc(MeshSet& m, const std::vector<int>& vcap, const std::vector<int>& ecap,
                      int W);
void set_free(MeshSet& m);
// Release the status word and the pinned read-back slot of a set.
void set_release(MeshSet& m);
cudaError_t upload_tab(MeshSet& m);
void set_used(MeshSet& m);
cudaError_t grow(MeshSet& m, const std::vector<int>& vcap, const std::vector<int>& ecap, int W);
int rebuild_adjacency(MeshSet& m, bool derive_flags, bool corners_given);
int presize(MeshSet& m);
int renumber(MeshSet& m, bool final);
int compact_out(MeshSet& m, int mesh, double* xy, int32_t* tri, double* mt, int* nv_out,
                int* ne_out);
int compact_out_set(MeshSet& m, double* xy, int32_t* tri, double* mt, int* nv_out, int* ne_out);
int sync_status(MeshSet& m);
int validate_mesh(MeshSet& m);
int refresh_quality(MeshSet& m);
// The quality cache of every element, computed now when it is stale (a mesh
// whose metric was never set gets it at its first operator call).
int ensure_quality(MeshSet& m);
cudaError_t refresh_sizes(MeshSet& m);

// ---- operators (pm_ops.cu) ----
int op_coarsen(MeshSet& m, int max_rounds);
int op_swap(MeshSet& m, int max_rounds);
int op_refine(MeshSet& m, int max_rounds);
int op_smooth(MeshSet& m, int max_sweeps, int max_rounds);
int op_opt_smooth(MeshSet& m, int nrounds, int max_rounds);
void zero_ops(MeshSet& m);
cudaError_t fetch_ops(MeshSet& m, std::vector<unsigned long long>& ops);

// ---- quality (pm_quality.cu) ----
int quality_mesh(MeshSet& m, double* qsum_host, double* dxy_host, double* dm_host);
int quality_arrays(const double* xy, const double* mt, int nv, const int* tri, int ne,
                   double* qsum, double* dxy, double* dm, cudaStream_t s);

// ---- errors (pm_capi.cu) ----
void set_last_error(const std::string& msg);

// ---- launches (pm_prof.cu) ----
// Every kernel of the library is launched through PM_LAUNCH: it counts the
// launch and, while profiling is on for a matching kernel name, brackets it
// with CUDA events on its own stream.
extern unsigned long long g_launches;
extern bool g_prof_on;
int prof_begin(const char* name, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);
// Device counter of algorithmic work (FP64 operations) for the kernel being
// profiled, or null when `name` is not being profiled.
unsigned long long* prof_work(const char* name);

template <class K, class... A>
inline void launch(const char* name, K kern, dim3 g, dim3 b, size_t sh, cudaStream_t s,
                   A... args) {
  __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED);
  int slot = g_prof_on ? prof_begin(name, s) : -1;
  kern<<<g, b, sh, s>>>(args...);
  if (slot >= 0) prof_end(slot, s);
}

#define PM_LAUNCH(k, g, b, sh, s, ...) ::pm::launch(#k, k, g, b, sh, s, __VA_ARGS__)

// ---- launch shapes (pm_tune.cu) ----
// Per operator (collapse, flip, split, smoothing): threads per block and the
// cap on blocks per SM of the one-kernel-per-phase grids; per operator
// (collapse, flip, smoothing): the largest list whose rounds run in one
// persistent launch, the blocks per SM of that launch, and (flips,
// smoothing) the list size up to which its rounds evaluate in one phase.
// No choice changes a result.
enum TuneOp { TO_COARSEN = 0, TO_SWAP = 1, TO_REFINE = 2, TO_SMOOTH = 3 };
struct Tuning {
  int block[4];
  int blocks_per_sm[4];
  int rounds_limit[3];
  int rounds_blocks_per_sm[3];  // resident blocks per SM of the persistent round kernels
  int fuse_limit[2];            // flips, smoothing: one-phase evaluation up to this list size
};
Tuning tuning();
void tuning_autoload();

// Blocks of `block` threads for n items, at most per_sm blocks per SM.
inline int grid_tuned(const MeshSet& m, long long n, int block, int per_sm) {
  long long want = (n + block - 1) / block;
  long long cap = (long long)m.num_sms * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

inline int grid_for(const MeshSet& m, long long n, int per_sm = 16) {
  long long want = (n + BLOCK - 1) / BLOCK;
  long long cap = (long long)m.num_sms * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

}  // namespace pm
