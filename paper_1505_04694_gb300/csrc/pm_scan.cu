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

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;  // per thread, consecutive (four int4 loads)
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr long long SPIN_LIMIT = 1LL << 22;

// state word: [63:34] epoch, [33:32] flag (1 aggregate, 2 inclusive), [31:0] value
__device__ __forceinline__ unsigned long long pack(unsigned epoch, unsigned flag, unsigned val) {
  return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | val;
}

__device__ __forceinline__ unsigned long long load_state(const unsigned long long* p) {
  return *((volatile const unsigned long long*)p);
}

// Inputs of the scan: an int array, or the 0/1 alive flags of the used
// vertex or element slots of a store (read directly, no flag array).
struct IntInput {
  const int* in;
  __device__ __forceinline__ void load16(long long first, long long n, int* v) const {
    if (first + SCAN_ITEMS <= n) {
      const int4* p = reinterpret_cast<const int4*>(in + first);
#pragma unroll
      for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
        int4 x = p[q];
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < SCAN_ITEMS; ++j) v[j] = (first + j < n) ? in[first + j] : 0;
    }
  }
};

struct VertexAlive {
  Store S;
  __device__ __forceinline__ void load16(long long first, long long n, int* v) const {
    uint4 f = make_uint4(0, 0, 0, 0);
    if (first + SCAN_ITEMS <= n) f = *reinterpret_cast<const uint4*>(S.vflag + first);
    const unsigned w[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      const long long s = first + j;
      unsigned flag = (first + SCAN_ITEMS <= n) ? (w[j >> 2] >> (8 * (j & 3))) & 0xFFu
                                                : (s < n ? S.vflag[s] : 0u);
      int alive = 0;
      if (s < n && (flag & VF_ALIVE)) {
        const int mi = mesh_of_vslot(S, (int)s);
        alive = (int)s - S.tab.vbase[mi] < S.tab.nv[mi];
      }
      v[j] = alive;
    }
  }
};

struct ElementAlive {
  Store S;
  __device__ __forceinline__ void load16(long long first, long long n, int* v) const {
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      const long long s = first + j;
      int alive = 0;
      if (s < n && S.EN[s].w) {
        const int mi = mesh_of_eslot(S, (int)s);
        alive = (int)s - S.tab.ebase[mi] < S.tab.ne[mi];
      }
      v[j] = alive;
    }
  }
};

template <class Input>
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan(Input input, int* __restrict__ out, int n, unsigned long long* state, int* ticket,
       unsigned epoch, DevStatus* st) {
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
  const long long first = (long long)tile * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  input.load16(first, n, v);
  int sum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int x = v[j];
    v[j] = sum;
    sum += x;
  }
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
  // decoupled look-back by warp 0, 32 predecessors at a time
  if (wid == 0) {
    int excl = 0;
    if (tile == 0) {
      if (lane == 0) atomicExch(state, pack(epoch, 2, (unsigned)total));
    } else {
      if (lane == 0) atomicExch(state + tile, pack(epoch, 1, (unsigned)total));
      int j = tile - 1;  // newest predecessor not yet added
      bool done = false, fail = false;
      while (!done && !fail) {
        int idx = j - lane;
        unsigned flag = 3u;  // lanes beyond tile 0 act as an inclusive zero
        unsigned val = 0;
        if (idx >= 0) {
          long long spins = 0;
          for (;;) {
            unsigned long long w = load_state(state + idx);
            flag = ((unsigned)(w >> 34) == (epoch & 0x3FFFFFFFu)) ? (unsigned)((w >> 32) & 3u) : 0u;
            if (flag != 0u) {
              val = (unsigned)(w & 0xFFFFFFFFu);
              break;
            }
            if (++spins > SPIN_LIMIT) break;
            if (spins > 32) __nanosleep(64);
          }
          if (flag == 0u) fail = true;
        }
        fail = __any_sync(0xffffffffu, fail);
        if (fail) break;
        // the nearest predecessor holding an inclusive prefix ends the walk
        unsigned incl_mask = __ballot_sync(0xffffffffu, flag >= 2u);
        int stop = incl_mask ? (__ffs(incl_mask) - 1) : 32;
        int add = (lane <= stop && lane < 32 && idx >= 0) ? (int)val : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
        excl += add;
        if (incl_mask) done = true;
        else j -= 32;
      }
      if (fail) {
        if (lane == 0) s_fail = 1;
      } else if (lane == 0) {
        __threadfence();
        atomicExch(state + tile, pack(epoch, 2, (unsigned)(excl + total)));
      }
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0) set_err(st, PM_ERR_TIMEOUT);
    return;
  }
  const int off = s_excl + wpre + incl - sum;
  if (first + SCAN_ITEMS <= n) {
    int4* p = reinterpret_cast<int4*>(out + first);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS / 4; ++q)
      p[q] = make_int4(off + v[4 * q], off + v[4 * q + 1], off + v[4 * q + 2], off + v[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
      if (first + j < n) out[first + j] = off + v[j];
  }
  // the last tile also writes the grand total at out[n]
  if (threadIdx.x == 0 && (long long)tile * SCAN_TILE + SCAN_TILE >= n) out[n] = s_excl + total;
}

}  // namespace

int scan_tiles(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

namespace {

template <class Input>
void scan_run(Input input, int* out, int n, ScanWork& w, DevStatus* st, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int), s);
    return;
  }
  int tiles = scan_tiles(n);
  cudaMemsetAsync(w.ticket, 0, sizeof(int), s);
  w.epoch = (w.epoch + 1) & 0x3FFFFFFFu;
  if (w.epoch == 0) w.epoch = 1;
  PM_LAUNCH(k_scan<Input>, tiles, SCAN_THREADS, 0, s, input, out, n, w.state, w.ticket, w.epoch,
            st);
}

}  // namespace

// Exclusive scan of in[0..n) into out[0..n]; out[n] holds the total.
// `state` needs scan_tiles(n) words and is never cleared (epochs tell runs
// apart); `ticket` is reset here.
void scan_exclusive(const int* in, int* out, int n, ScanWork& w, DevStatus* st, cudaStream_t s) {
  scan_run(IntInput{in}, out, n, w, st, s);
}

// The same over the alive flags of the used vertex (element) slots [0, n).
void scan_alive_vertices(const Store& S, int* out, int n, ScanWork& w, DevStatus* st,
                         cudaStream_t s) {
  scan_run(VertexAlive{S}, out, n, w, st, s);
}

void scan_alive_elements(const Store& S, int* out, int n, ScanWork& w, DevStatus* st,
                         cudaStream_t s) {
  scan_run(ElementAlive{S}, out, n, w, st, s);
}

}  // namespace pm
