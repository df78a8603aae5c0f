// Single-pass exclusive scan with decoupled look-back (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016), written
// for this library.  Tiles take their position from an atomic ticket (the
// fetch-and-add worklist idea of Sec. 3.4), which guarantees that every tile a
// block waits for is already running; each wait is bounded and reports
// PM_ERR_TIMEOUT through the status word instead of spinning forever.
//
// The scan gives new vertex and element ids in index order, so ids are
// reproducible regardless of thread timing (the prefix-sum worklist of
// Sec. 3.4, here without its synchronisation cost).
#include "pm_internal.cuh"

namespace pm {

namespace {

constexpr int SCAN_THREADS = 128;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr long long SPIN_LIMIT = 1LL << 22;

// state word: [63:34] epoch, [33:32] flag (1 aggregate, 2 inclusive), [31:0] value
__device__ __forceinline__ unsigned long long pack(unsigned epoch, unsigned flag, unsigned val) {
  return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | val;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan(const int* __restrict__ in, int* __restrict__ out, int n, unsigned long long* state,
       int* ticket, unsigned epoch, DevStatus* st) {
  __shared__ int s_items[SCAN_TILE];
  __shared__ int s_warp[SCAN_THREADS / 32];
  __shared__ int s_tile;
  __shared__ int s_excl;
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(ticket, 1);
    s_fail = 0;
  }
  __syncthreads();
  const int tile = s_tile;
  const long long base = (long long)tile * SCAN_TILE;
  // coalesced load into shared memory
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
    long long g = base + k;
    s_items[k] = (g < n) ? in[g] : 0;
  }
  __syncthreads();
  int local[SCAN_ITEMS];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    local[j] = sum;
    sum += s_items[threadIdx.x * SCAN_ITEMS + j];
  }
  // block scan of thread sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  int wpre = 0, total = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    int x = s_warp[w];
    if (w < wid) wpre += x;
    total += x;
  }
  const int texcl = wpre + incl - sum;
  // decoupled look-back by thread 0
  if (threadIdx.x == 0) {
    int excl = 0;
    if (tile == 0) {
      atomicExch(state + tile, pack(epoch, 2, (unsigned)total));
    } else {
      atomicExch(state + tile, pack(epoch, 1, (unsigned)total));
      int j = tile - 1;
      while (j >= 0) {
        unsigned long long w;
        long long spins = 0;
        for (;;) {
          w = *((volatile unsigned long long*)(state + j));
          if ((unsigned)(w >> 34) == (epoch & 0x3FFFFFFFu) && ((w >> 32) & 3u) != 0) break;
          if (++spins > SPIN_LIMIT) break;
          if (spins > 64) __nanosleep(64);
        }
        if (spins > SPIN_LIMIT) {
          s_fail = 1;
          break;
        }
        excl += (int)(unsigned)(w & 0xFFFFFFFFu);
        if (((w >> 32) & 3u) == 2u) break;
        --j;
      }
      if (!s_fail) {
        __threadfence();
        atomicExch(state + tile, pack(epoch, 2, (unsigned)(excl + total)));
      }
    }
    s_excl = excl;
  }
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0) set_err(st, PM_ERR_TIMEOUT);
    return;
  }
  const int off = s_excl + texcl;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) s_items[threadIdx.x * SCAN_ITEMS + j] = off + local[j];
  __syncthreads();
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
    long long g = base + k;
    if (g < n) out[g] = s_items[k];
  }
  // the last tile also writes the grand total at out[n]
  if (threadIdx.x == 0 && base + SCAN_TILE >= n) out[n] = s_excl + total;
}

}  // namespace

int scan_tiles(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// Exclusive scan of in[0..n) into out[0..n]; out[n] holds the total.
// `state` needs scan_tiles(n) words and is never cleared (epochs tell runs
// apart); `ticket` is reset here.
void scan_exclusive(const int* in, int* out, int n, ScanWork& w, DevStatus* st, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int), s);
    return;
  }
  int tiles = scan_tiles(n);
  cudaMemsetAsync(w.ticket, 0, sizeof(int), s);
  w.epoch = (w.epoch + 1) & 0x3FFFFFFFu;
  if (w.epoch == 0) w.epoch = 1;
  PM_LAUNCH(k_scan, tiles, SCAN_THREADS, 0, s, in, out, n, w.state, w.ticket, w.epoch, st);
}

}  // namespace pm
