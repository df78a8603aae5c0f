// C interface (include/pm.h): argument checks, device selection, and the
// drivers that sequence the operators (Algorithm 1 of Sec. 2.3, batching).
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pm_internal.cuh"

struct pm_mesh {
  pm::MeshSet set;
};

namespace pm {

namespace {

thread_local std::string g_last_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

pm_status fail(pm_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

// Calls that read or write one mesh's arrays take a one-mesh handle.
pm_status single_only(const pm_mesh* h, const char* what) {
  if (h->set.nmesh == 1) return PM_OK;
  return fail(PM_ERR_INVALID_ARG,
              std::string(what) + " takes a one-mesh handle (use the pm_batch_ calls)");
}

pm_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PM_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
}

pm_status check_params(const pm_params* p) {
  if (!p) return fail(PM_ERR_INVALID_ARG, "params is null");
  if (!std::isfinite(p->L_low) || !std::isfinite(p->L_up) || !(p->L_low > 0.0) ||
      !(p->L_up > p->L_low))
    return fail(PM_ERR_INVALID_ARG, "need 0 < L_low < L_up, both finite");
  if (!std::isfinite(p->q_thresh) || !(p->q_thresh >= 0.0))
    return fail(PM_ERR_INVALID_ARG, "q_thresh must be finite and >= 0");
  if (p->max_iter < 0 || p->max_smooth_sweeps < 0 || p->opt_smooth_rounds < 0 ||
      p->max_rounds < 0)
    return fail(PM_ERR_INVALID_ARG, "iteration, sweep and round limits must be >= 0");
  if (p->select != PM_SELECT_HASH && p->select != PM_SELECT_COLOUR)
    return fail(PM_ERR_INVALID_ARG, "select must be PM_SELECT_HASH or PM_SELECT_COLOUR");
  return PM_OK;
}

// Concatenated inputs into the slots of every mesh: input vertex g of mesh
// i (offsets in S.tab.pre) goes to slot vbase_i + (g - pre_i), with the
// identity metric and, when the caller flags it, the corner bit.
__global__ void k_ingest(Store S, const double* xy, const int* tri, const uint8_t* corner,
                         int nv, int ne) {
  const int n = S.nmesh;
  const int* pv = S.tab.pre;
  const int* pe = S.tab.pre + n + 1;
  int top = ne > nv ? ne : nv;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < top; g += gridDim.x * blockDim.x) {
    if (g < nv) {
      int mi = seg_of(pv, n, g);
      int slot = S.tab.vbase[mi] + (g - pv[mi]);
      S.xy[slot] = make_double2(xy[2 * (size_t)g], xy[2 * (size_t)g + 1]);
      S.M[slot] = make_double4(1.0, 0.0, 1.0, 0.0);
      S.vflag[slot] = (uint8_t)(VF_ALIVE | ((corner && corner[g]) ? VF_CORNER : 0));
    }
    if (g < ne) {
      int mi = seg_of(pe, n, g);
      S.EN[S.tab.ebase[mi] + (g - pe[mi])] =
          make_int4(tri[3 * (size_t)g], tri[3 * (size_t)g + 1], tri[3 * (size_t)g + 2], 1);
    }
  }
}

__global__ void k_metric_check(const double* m, int nv, DevStatus* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    double a = m[3 * i], b = m[3 * i + 1], c = m[3 * i + 2];
    bool ok = isfinite(a) && isfinite(b) && isfinite(c) && a > 0.0 && a * c - b * b > 0.0;
    if (!ok) set_err(st, PM_ERR_INVALID_ARG);
  }
}

// Concatenated metric (mesh after mesh, each in its used-slot order; offsets
// in S.tab.pre) into the slots.
__global__ void k_metric_set(Store S, const double* m, int nv) {
  const int n = S.nmesh;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nv; g += gridDim.x * blockDim.x) {
    int mi = seg_of(S.tab.pre, n, g);
    int slot = S.tab.vbase[mi] + (g - S.tab.pre[mi]);
    S.M[slot] = make_double4(m[3 * (size_t)g], m[3 * (size_t)g + 1], m[3 * (size_t)g + 2], 0.0);
  }
}

int sms_of(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

void set_mem_pool_retain(int dev) {
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
}

// Exclusive prefix sums of per-mesh vertex and element counts into the
// device table (S.tab.pre), for kernels that map a concatenated array onto
// the meshes' slots.
cudaError_t upload_prefix(MeshSet& m, const std::vector<int>& nv, const std::vector<int>& ne) {
  const int n = m.nmesh;
  std::vector<int> pre(2 * ((size_t)n + 1));
  for (int i = 0; i < n; ++i) {
    pre[i + 1] = pre[i] + nv[i];
    pre[n + 1 + i + 1] = pre[n + 1 + i] + ne[i];
  }
  // a copy from pageable memory is staged before the call returns
  return cudaMemcpyAsync(m.S.tab.pre, pre.data(), pre.size() * sizeof(int),
                         cudaMemcpyHostToDevice, m.stream);
}

// Shared body of pm_mesh_create / pm_batch_create and their _dev forms.
// Inputs are host or device pointers: nmesh meshes concatenated (vertex ids
// local to each mesh), per-mesh sizes nv[i], ne[i] on the host.
pm_status create_set(const double* xy, const int32_t* nv, const int32_t* tri, const int32_t* ne,
                     int nmesh, const uint8_t* corner, int cap_factor, int dev,
                     cudaStream_t stream, bool own_stream, bool host, pm_mesh** out) {
  tuning_autoload();
  pm_mesh* h = new pm_mesh();
  MeshSet& m = h->set;
  m.device = dev;
  m.stream = stream;
  m.own_stream = own_stream;
  m.nmesh = nmesh;
  m.num_sms = sms_of(dev);
  m.nv.assign(nv, nv + nmesh);
  m.ne.assign(ne, ne + nmesh);
  m.seed.assign(nmesh, 1u);
  m.L_low.assign(nmesh, 0.4);
  m.L_up.assign(nmesh, std::sqrt(2.0));
  m.q_thresh.assign(nmesh, 0.7);
  m.select.assign(nmesh, 0);
  std::vector<int> vcap(nmesh), ecap(nmesh);
  long long nvt = 0, net = 0;
  for (int i = 0; i < nmesh; ++i) {
    long long vc = std::max<long long>((long long)nv[i] * cap_factor, (long long)nv[i] + 64);
    long long ec = std::max<long long>((long long)ne[i] * cap_factor, (long long)ne[i] + 64);
    if (vc >= (1LL << 30) || ec >= (1LL << 30)) {
      delete h;
      return fail(PM_ERR_CAPACITY, "mesh too large for 32-bit slot ids");
    }
    vcap[i] = (int)vc;
    ecap[i] = (int)ec;
    nvt += nv[i];
    net += ne[i];
  }
  cudaError_t e = set_alloc(m, vcap, ecap, 16);
  pm_status s = cuda_status(e, "allocating mesh");
  char* tmp = nullptr;
  const double* dxy = xy;
  const int32_t* dtri = tri;
  const uint8_t* dcorner = corner;
  if (!s) s = cuda_status(upload_tab(m), "mesh table");
  if (!s) s = cuda_status(upload_prefix(m, m.nv, m.ne), "mesh offsets");
  if (!s) {
    cudaMemsetAsync(m.S.tab.active, 0xFF, nmesh * sizeof(int), m.stream);
    if (host) {
      const size_t bxy = (size_t)nvt * 2 * sizeof(double), btri = (size_t)net * 3 * sizeof(int32_t);
      const size_t bc = corner ? (size_t)nvt : 0;
      e = cudaMallocAsync((void**)&tmp, bxy + btri + bc + 64, m.stream);
      if (!e) e = cudaMemcpyAsync(tmp, xy, bxy, cudaMemcpyHostToDevice, m.stream);
      if (!e) e = cudaMemcpyAsync(tmp + bxy, tri, btri, cudaMemcpyHostToDevice, m.stream);
      if (!e && corner) e = cudaMemcpyAsync(tmp + bxy + btri, corner, bc, cudaMemcpyHostToDevice,
                                            m.stream);
      dxy = (const double*)tmp;
      dtri = (const int32_t*)(tmp + bxy);
      dcorner = corner ? (const uint8_t*)(tmp + bxy + btri) : nullptr;
      s = cuda_status(e, "uploading mesh");
    }
  }
  if (!s) {
    PM_LAUNCH(k_ingest, grid_for(m, std::max(nvt, net)), BLOCK, 0, m.stream, m.S, dxy, dtri,
              dcorner, (int)nvt, (int)net);
    int err = validate_mesh(m);
    if (err) s = (pm_status)err;
    if (s == PM_ERR_INVALID_ARG) set_last_error("non-finite coordinate");
    if (s == PM_ERR_INVALID_MESH)
      set_last_error("invalid mesh: vertex id out of range, repeated in an element, or an "
                     "element that is not counter-clockwise");
    if (!s) {
      err = rebuild_adjacency(m, true, corner != nullptr);
      if (err) {
        s = (pm_status)err;
        if (s == PM_ERR_INVALID_MESH)
          set_last_error("invalid mesh: overlapping elements, non-manifold or unused vertex");
      }
    }
  }
  if (tmp) cudaFreeAsync(tmp, m.stream);
  if (s) {
    set_free(m);
    set_release(m);
    if (own_stream) cudaStreamDestroy(m.stream);
    delete h;
    return s;
  }
  cudaMemsetAsync(m.st, 0, sizeof(DevStatus), m.stream);
  *out = h;
  return PM_OK;
}

// Per-mesh parameters into the table; round counters and op counts cleared;
// every mesh active.
pm_status begin_call(MeshSet& m, const pm_params* P, int stride) {
  if (int err = ensure_quality(m)) return (pm_status)err;
  for (int i = 0; i < m.nmesh; ++i) {
    const pm_params& p = P[stride ? i : 0];
    m.seed[i] = p.seed;
    m.L_low[i] = p.L_low;
    m.L_up[i] = p.L_up;
    m.q_thresh[i] = p.q_thresh;
    m.select[i] = p.select;
  }
  pm_status s = cuda_status(upload_tab(m), "mesh table");
  if (s) return s;
  cudaMemsetAsync(m.S.tab.r, 0, m.nmesh * sizeof(uint32_t), m.stream);
  cudaMemsetAsync(m.S.tab.had, 0, 2 * m.nmesh * sizeof(int), m.stream);
  cudaMemsetAsync(m.S.tab.active, 0xFF, m.nmesh * sizeof(int), m.stream);
  cudaMemsetAsync(m.st, 0, sizeof(DevStatus), m.stream);
  zero_ops(m);
  // evaluations from earlier calls may predate a new metric or parameters
  m.lo_coarsen = m.lo_swap = m.lo_refine = m.tag;
  return PM_OK;
}

struct CallStats {
  std::vector<long long> collapses, splits, flips, moves;
  std::vector<int> converged;
  void init(int n) {
    collapses.assign(n, 0);
    splits.assign(n, 0);
    flips.assign(n, 0);
    moves.assign(n, 0);
    converged.assign(n, 0);
  }
};

// Run one operator and add its per-mesh operation counts to `acc`.
template <class F>
pm_status run_counted(MeshSet& m, F&& f, std::vector<long long>& acc,
                      std::vector<unsigned long long>* last = nullptr) {
  zero_ops(m);
  int err = f();
  if (err) return (pm_status)err;
  std::vector<unsigned long long> ops;
  pm_status s = cuda_status(fetch_ops(m, ops), "reading counters");
  if (s) return s;
  for (int i = 0; i < m.nmesh; ++i) acc[i] += (long long)ops[i];
  if (last) *last = ops;
  return PM_OK;
}

// Runs one operator and queues the read-back of its operation counts into
// pinned slot `slot` without waiting (the caller reads them after its next
// synchronisation).
template <class F>
pm_status run_counted_async(MeshSet& m, F&& f, int slot) {
  zero_ops(m);
  int err = f();
  if (err) return (pm_status)err;
  return cuda_status(cudaMemcpyAsync(m.hops + (size_t)slot * m.nmesh, m.S.tab.ops,
                                     m.nmesh * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, m.stream),
                     "reading counters");
}

pm_status fill_stats(MeshSet& m, const CallStats& cs, double t0, pm_stats* out, int n) {
  if (!out) return PM_OK;
  std::vector<uint32_t> r(m.nmesh);
  cudaError_t e = cudaMemcpyAsync(r.data(), m.S.tab.r, m.nmesh * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, m.stream);
  if (!e) e = cudaStreamSynchronize(m.stream);
  if (e) return cuda_status(e, "reading counters");
  double ms = now_ms() - t0;
  for (int i = 0; i < n; ++i) {
    out[i].rounds = r[i];
    out[i].collapses = cs.collapses[i];
    out[i].splits = cs.splits[i];
    out[i].flips = cs.flips[i];
    out[i].moves = cs.moves[i];
    out[i].converged = cs.converged[i];
    out[i].ms = ms;
  }
  return PM_OK;
}

enum OpKind { OP_COARSEN, OP_SWAP, OP_REFINE, OP_SMOOTH, OP_OPT, OP_ADAPT };

// Algorithm 1 (Sec. 2.3) over every mesh of the set: iterate coarsen, swap,
// refine (a mesh leaves the loop after an iteration that changed nothing, or
// after max_iter), renumber after each iteration; then Laplacian smoothing,
// optional optimisation-based smoothing, renumber.
pm_status adapt_set(MeshSet& m, const pm_params* P, int stride, CallStats& cs) {
  int n = m.nmesh;
  if (int err = presize(m)) return (pm_status)err;
  int max_iter = 0;
  for (int i = 0; i < n; ++i) max_iter = std::max(max_iter, P[stride ? i : 0].max_iter);
  std::vector<int> active(n, 1);
  for (int it = 0; it < max_iter; ++it) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (active[i] && it >= P[stride ? i : 0].max_iter) active[i] = 0;
      any |= active[i] != 0;
    }
    if (!any) break;
    cudaMemcpyAsync(m.S.tab.active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice,
                    m.stream);
    pm_status s;
    const int mr = P[0].max_rounds;
    if ((s = run_counted_async(m, [&] { return op_coarsen(m, mr); }, 0))) return s;
    if ((s = run_counted_async(m, [&] { return op_swap(m, mr); }, 1))) return s;
    if ((s = run_counted_async(m, [&] { return op_refine(m, mr); }, 2))) return s;
    int err = renumber(m, false);  // synchronises: the op counts have arrived
    if (err) return (pm_status)err;
    const unsigned long long* h = m.hops;
    for (int i = 0; i < n; ++i) {
      const long long c_i = (long long)h[i], sw_i = (long long)h[n + i];
      const long long rf_i = (long long)h[2 * n + i];
      if (!active[i]) continue;
      cs.collapses[i] += c_i;
      cs.flips[i] += sw_i;
      cs.splits[i] += rf_i;
      if (c_i + sw_i + rf_i == 0) {
        cs.converged[i] = 1;
        active[i] = 0;
      }
    }
  }
  std::vector<int> all(n, 1);
  cudaMemcpyAsync(m.S.tab.active, all.data(), n * sizeof(int), cudaMemcpyHostToDevice, m.stream);
  int sweeps = 0, opt = 0;
  for (int i = 0; i < n; ++i) {
    sweeps = std::max(sweeps, P[stride ? i : 0].max_smooth_sweeps);
    opt = std::max(opt, P[stride ? i : 0].opt_smooth_rounds);
  }
  pm_status s;
  const int mr = P[0].max_rounds;
  if ((s = run_counted(m, [&] { return op_smooth(m, sweeps, mr); }, cs.moves))) return s;
  if (opt > 0)
    if ((s = run_counted(m, [&] { return op_opt_smooth(m, opt, mr); }, cs.moves))) return s;
  int err = renumber(m, true);
  return (pm_status)err;
}

pm_status run_op(pm_mesh* h, const pm_params* P, pm_stats* st, OpKind kind) {
  if (!h) return fail(PM_ERR_INVALID_ARG, "mesh is null");
  pm_status s = check_params(P);
  if (s) return s;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  double t0 = now_ms();
  if ((s = begin_call(m, P, 0))) return s;
  CallStats cs;
  cs.init(1);
  switch (kind) {
    case OP_COARSEN:
      s = run_counted(m, [&] { return op_coarsen(m, P->max_rounds); }, cs.collapses);
      break;
    case OP_SWAP:
      s = run_counted(m, [&] { return op_swap(m, P->max_rounds); }, cs.flips);
      break;
    case OP_REFINE:
      s = run_counted(m, [&] { return op_refine(m, P->max_rounds); }, cs.splits);
      break;
    case OP_SMOOTH:
      s = run_counted(m, [&] { return op_smooth(m, P->max_smooth_sweeps, P->max_rounds); },
                      cs.moves);
      if (!s && P->opt_smooth_rounds > 0)
        s = run_counted(m, [&] { return op_opt_smooth(m, P->opt_smooth_rounds, P->max_rounds); },
                        cs.moves);
      break;
    case OP_OPT:
      s = run_counted(m, [&] { return op_opt_smooth(m, P->opt_smooth_rounds, P->max_rounds); },
                      cs.moves);
      break;
    case OP_ADAPT:
      s = adapt_set(m, P, 0, cs);
      break;
  }
  if (s) return s;
  int err = sync_status(m);
  if (err) return (pm_status)err;
  return fill_stats(m, cs, t0, st, 1);
}

// ---- batching ------------------------------------------------------------------

// Copy mesh `src` (a one-mesh set) into region `i` of `dst`, or back.
pm_status copy_region(MeshSet& dst, int di, MeshSet& src, int si, cudaStream_t s) {
  int nv = src.nv[si], ne = src.ne[si];
  size_t vd = dst.vbase[di], vs = src.vbase[si], ed = dst.ebase[di], es = src.ebase[si];
  auto cp = [&](void* d, const void* sp, size_t bytes) {
    return cudaMemcpyAsync(d, sp, bytes, cudaMemcpyDeviceToDevice, s);
  };
  cudaError_t e = cudaSuccess;
  if (!e) e = cp(dst.S.xy + vd, src.S.xy + vs, nv * sizeof(double2));
  if (!e) e = cp(dst.S.M + vd, src.S.M + vs, nv * sizeof(double4));
  if (!e) e = cp(dst.S.vflag + vd, src.S.vflag + vs, nv);
  if (!e) e = cp(dst.S.NNlen + vd, src.S.NNlen + vs, nv * sizeof(int));
  if (!e) e = cp(dst.S.NElen + vd, src.S.NElen + vs, nv * sizeof(int));
  if (!e) e = cp(dst.S.EN + ed, src.S.EN + es, ne * sizeof(int4));
  if (!e) e = cp(dst.S.qK + ed, src.S.qK + es, ne * sizeof(double));
  if (dst.S.W == src.S.W) {
    if (!e) e = cp(dst.S.NN + vd * dst.S.W, src.S.NN + vs * src.S.W, (size_t)nv * src.S.W * 4);
    if (!e) e = cp(dst.S.NE + vd * dst.S.W, src.S.NE + vs * src.S.W, (size_t)nv * src.S.W * 4);
  } else {
    size_t wmin = std::min(dst.S.W, src.S.W);
    if (!e)
      e = cudaMemcpy2DAsync(dst.S.NN + vd * dst.S.W, dst.S.W * 4, src.S.NN + vs * src.S.W,
                            src.S.W * 4, wmin * 4, nv, cudaMemcpyDeviceToDevice, s);
    if (!e)
      e = cudaMemcpy2DAsync(dst.S.NE + vd * dst.S.W, dst.S.W * 4, src.S.NE + vs * src.S.W,
                            src.S.W * 4, wmin * 4, nv, cudaMemcpyDeviceToDevice, s);
  }
  return cuda_status(e, "copying a mesh region");
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace pm

using namespace pm;

extern "C" {

const char* pm_status_string(pm_status s) {
  switch (s) {
    case PM_OK: return "ok";
    case PM_ERR_INVALID_ARG: return "invalid argument";
    case PM_ERR_INVALID_MESH: return "invalid mesh";
    case PM_ERR_OOM: return "out of device memory";
    case PM_ERR_CAPACITY: return "capacity exceeded";
    case PM_ERR_CUDA: return "CUDA error";
    case PM_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* pm_last_error(void) { return g_last_error.c_str(); }

pm_status pm_mesh_create(const double* xy, int32_t nv, const int32_t* tri, int32_t ne,
                         const uint8_t* corner, int32_t cap_factor, int device, pm_mesh** out) {
  if (!out) return fail(PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!xy || !tri || nv < 3 || ne < 1 || cap_factor < 1)
    return fail(PM_ERR_INVALID_ARG, "need xy, tri, nv >= 3, ne >= 1, cap_factor >= 1");
  // ids and coordinates are checked on the device after the upload
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(PM_ERR_INVALID_ARG, "no such CUDA device");
  DeviceGuard g(device);
  set_mem_pool_retain(device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(PM_ERR_CUDA, "creating a stream");
  return create_set(xy, &nv, tri, &ne, 1, corner, cap_factor, device, s, true, true, out);
}

pm_status pm_mesh_create_dev(const double* xy, int32_t nv, const int32_t* tri, int32_t ne,
                             const uint8_t* corner, int32_t cap_factor, void* stream,
                             pm_mesh** out) {
  if (!out) return fail(PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!xy || !tri || nv < 3 || ne < 1 || cap_factor < 1)
    return fail(PM_ERR_INVALID_ARG, "need xy, tri, nv >= 3, ne >= 1, cap_factor >= 1");
  int dev = 0;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, xy) != cudaSuccess || pa.type != cudaMemoryTypeDevice)
    return fail(PM_ERR_INVALID_ARG, "xy is not device memory");
  dev = pa.device;
  DeviceGuard g(dev);
  set_mem_pool_retain(dev);
  cudaStream_t s = (cudaStream_t)stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(PM_ERR_CUDA, "creating a stream");
    own = true;
  }
  return create_set(xy, &nv, tri, &ne, 1, corner, cap_factor, dev, s, own, false, out);
}

pm_status pm_mesh_destroy(pm_mesh* h) {
  if (!h) return PM_OK;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  set_free(m);
  set_release(m);
  if (m.own_stream) cudaStreamDestroy(m.stream);
  delete h;
  return PM_OK;
}

pm_status pm_set_stream(pm_mesh* h, void* stream) {
  if (!h) return fail(PM_ERR_INVALID_ARG, "mesh is null");
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  cudaStreamSynchronize(m.stream);
  if (m.own_stream) cudaStreamDestroy(m.stream);
  m.own_stream = false;
  m.stream = (cudaStream_t)stream;
  if (!m.stream) {
    cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking);
    m.own_stream = true;
  }
  return PM_OK;
}

static pm_status set_metric_impl(pm_mesh* h, const double* M, bool host) {
  if (!h || !M) return fail(PM_ERR_INVALID_ARG, "mesh or metric is null");
  MeshSet& m = h->set;
  long long nvl = 0;
  for (int i = 0; i < m.nmesh; ++i) nvl += m.nv[i];
  const int nv = (int)nvl;
  DeviceGuard g(m.device);
  const double* src = M;
  double* tmp = nullptr;
  if (host) {
    cudaError_t e = cudaMallocAsync(&tmp, (size_t)nv * 3 * sizeof(double), m.stream);
    if (!e) e = cudaMemcpyAsync(tmp, M, (size_t)nv * 3 * sizeof(double), cudaMemcpyHostToDevice,
                                m.stream);
    if (e) {
      if (tmp) cudaFreeAsync(tmp, m.stream);
      return cuda_status(e, "uploading metric");
    }
    src = tmp;
  }
  // checked on the device, from host and device arrays alike
  PM_LAUNCH(k_metric_check, grid_for(m, nv), BLOCK, 0, m.stream, src, nv, m.st);
  if (int err = sync_status(m)) {
    cudaMemsetAsync(m.st, 0, sizeof(DevStatus), m.stream);
    if (tmp) cudaFreeAsync(tmp, m.stream);
    return fail((pm_status)err, "metric must be finite and symmetric positive definite");
  }
  pm_status s = cuda_status(upload_prefix(m, m.nv, m.ne), "mesh offsets");
  if (!s) PM_LAUNCH(k_metric_set, grid_for(m, nv), BLOCK, 0, m.stream, m.S, src, nv);
  if (tmp) cudaFreeAsync(tmp, m.stream);
  if (s) return s;
  return (pm_status)refresh_quality(m);
}

pm_status pm_set_metric(pm_mesh* h, const double* M) { return set_metric_impl(h, M, true); }
pm_status pm_set_metric_dev(pm_mesh* h, const double* M) { return set_metric_impl(h, M, false); }

pm_status pm_coarsen(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_COARSEN);
}
pm_status pm_refine(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_REFINE);
}
pm_status pm_swap(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_SWAP);
}
pm_status pm_smooth(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_SMOOTH);
}
pm_status pm_opt_smooth(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_OPT);
}
pm_status pm_adapt(pm_mesh* h, const pm_params* p, pm_stats* st) {
  return run_op(h, p, st, OP_ADAPT);
}

pm_status pm_adapt_batch(pm_mesh** meshes, int32_t n, const pm_params* params, pm_stats* stats) {
  if (!meshes || n < 1 || !params) return fail(PM_ERR_INVALID_ARG, "need meshes, n >= 1, params");
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return fail(PM_ERR_INVALID_ARG, "null mesh in batch");
    if (pm_status gs = single_only(meshes[i], "pm_adapt_batch")) return gs;
    pm_status s = check_params(params + i);
    if (s) return s;
    if (meshes[i]->set.device != meshes[0]->set.device)
      return fail(PM_ERR_INVALID_ARG, "all meshes of a batch must be on one device");
  }
  double t0 = now_ms();
  MeshSet& m0 = meshes[0]->set;
  DeviceGuard g(m0.device);
  for (int i = 1; i < n; ++i) cudaStreamSynchronize(meshes[i]->set.stream);
  MeshSet b;
  b.device = m0.device;
  b.stream = m0.stream;
  b.nmesh = n;
  b.num_sms = m0.num_sms;
  int W = 16;
  std::vector<int> vcap(n), ecap(n);
  b.nv.resize(n);
  b.ne.resize(n);
  b.seed.resize(n);
  b.L_low.resize(n);
  b.L_up.resize(n);
  b.q_thresh.resize(n);
  b.select.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    MeshSet& s = meshes[i]->set;
    W = std::max(W, s.S.W);
    b.nv[i] = s.nv[0];
    b.ne[i] = s.ne[0];
    vcap[i] = std::max(s.vcap[0], 2 * s.nv[0] + 64);
    ecap[i] = std::max(s.ecap[0], 2 * s.ne[0] + 64);
  }
  pm_status st = cuda_status(set_alloc(b, vcap, ecap, W), "allocating the batch");
  if (!st) {
    for (int i = 0; i < n; ++i) {
      b.seed[i] = params[i].seed;
      b.L_low[i] = params[i].L_low;
      b.L_up[i] = params[i].L_up;
      b.q_thresh[i] = params[i].q_thresh;
      b.select[i] = params[i].select;
    }
    st = cuda_status(upload_tab(b), "batch table");
  }
  for (int i = 0; i < n && !st; ++i) {
    st = (pm_status)ensure_quality(meshes[i]->set);
    if (!st) st = copy_region(b, i, meshes[i]->set, 0, b.stream);
  }
  b.qvalid = true;  // the copied cache of every mesh is current
  CallStats cs;
  cs.init(n);
  if (!st) st = begin_call(b, params, 1);
  if (!st) st = adapt_set(b, params, 1, cs);
  // results back into each mesh (growing it where needed)
  for (int i = 0; i < n && !st; ++i) {
    MeshSet& s = meshes[i]->set;
    if (b.nv[i] > s.vcap[0] || b.ne[i] > s.ecap[0] || b.S.W != s.S.W) {
      // the mesh's old contents are replaced below: new storage, nothing copied
      std::vector<int> v1 = {std::max(s.vcap[0], b.vcap[i])}, e1 = {std::max(s.ecap[0], b.ecap[i])};
      set_free(s);
      st = cuda_status(set_alloc(s, v1, e1, b.S.W), "growing a mesh");
      s.lo_coarsen = s.lo_swap = s.lo_refine = s.tag;
    }
    if (st) break;
    s.nv[0] = b.nv[i];
    s.ne[0] = b.ne[i];
    st = cuda_status(upload_tab(s), "mesh table");
    if (!st) st = copy_region(s, 0, b, i, b.stream);
  }
  if (!st) st = (pm_status)sync_status(b);
  if (!st && stats) st = fill_stats(b, cs, t0, stats, n);
  set_free(b);
  set_release(b);
  return st;
}

pm_status pm_get_mesh(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                      double* M) {
  if (!h || !nv || !ne) return fail(PM_ERR_INVALID_ARG, "mesh, nv and ne are required");
  if (pm_status gs = single_only(h, "pm_get_mesh")) return gs;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  int n1 = 0, n2 = 0;
  if (!xy && !tri && !M) {
    int err = compact_out(m, 0, nullptr, nullptr, nullptr, &n1, &n2);
    if (err) return (pm_status)err;
    *nv = n1;
    *ne = n2;
    return PM_OK;
  }
  // one compaction into device buffers sized by the used slots (an upper
  // bound of the live counts), then the copies of the live part
  const size_t vb = std::max(m.nv[0], 1), eb = std::max(m.ne[0], 1);
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, vb * 5 * sizeof(double) + eb * 3 * sizeof(int32_t),
                                  m.stream);
  pm_status s = cuda_status(e, "output buffers");
  if (s) return s;
  double* dxy = (double*)buf;
  double* dm = dxy + 2 * vb;
  int32_t* dtri = (int32_t*)(dm + 3 * vb);
  int err = compact_out(m, 0, xy ? dxy : nullptr, tri ? dtri : nullptr, M ? dm : nullptr, &n1, &n2);
  if (err) s = (pm_status)err;
  if (!s) {
    *nv = n1;
    *ne = n2;
    if (xy) cudaMemcpyAsync(xy, dxy, n1 * 2 * sizeof(double), cudaMemcpyDeviceToHost, m.stream);
    if (M) cudaMemcpyAsync(M, dm, n1 * 3 * sizeof(double), cudaMemcpyDeviceToHost, m.stream);
    if (tri) cudaMemcpyAsync(tri, dtri, n2 * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, m.stream);
  }
  cudaFreeAsync(buf, m.stream);
  err = sync_status(m);
  return s ? s : (pm_status)err;
}

pm_status pm_get_mesh_dev(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                          double* M) {
  if (!h || !nv || !ne) return fail(PM_ERR_INVALID_ARG, "mesh, nv and ne are required");
  if (pm_status gs = single_only(h, "pm_get_mesh_dev")) return gs;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  int n1 = 0, n2 = 0;
  int err = compact_out(m, 0, xy, tri, M, &n1, &n2);
  *nv = n1;
  *ne = n2;
  return (pm_status)err;
}

pm_status pm_get_raw(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, double* M, int32_t* tri,
                     uint8_t* valive, uint8_t* talive, uint8_t* vflag) {
  if (!h || !nv || !ne) return fail(PM_ERR_INVALID_ARG, "mesh, nv and ne are required");
  if (pm_status gs = single_only(h, "pm_get_raw")) return gs;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  int n1 = m.nv[0], n2 = m.ne[0];
  *nv = n1;
  *ne = n2;
  if (!xy && !M && !tri && !valive && !talive && !vflag) return PM_OK;
  std::vector<double2> pxy(n1);
  std::vector<double4> pm4(n1);
  std::vector<uint8_t> pf(n1);
  std::vector<int4> pe(n2);
  cudaMemcpyAsync(pxy.data(), m.S.xy, n1 * sizeof(double2), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(pm4.data(), m.S.M, n1 * sizeof(double4), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(pf.data(), m.S.vflag, n1, cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(pe.data(), m.S.EN, n2 * sizeof(int4), cudaMemcpyDeviceToHost, m.stream);
  int err = sync_status(m);
  if (err) return (pm_status)err;
  for (int i = 0; i < n1; ++i) {
    if (xy) {
      xy[2 * i] = pxy[i].x;
      xy[2 * i + 1] = pxy[i].y;
    }
    if (M) {
      M[3 * i] = pm4[i].x;
      M[3 * i + 1] = pm4[i].y;
      M[3 * i + 2] = pm4[i].z;
    }
    if (valive) valive[i] = (pf[i] & VF_ALIVE) ? 1 : 0;
    if (vflag) vflag[i] = (uint8_t)(((pf[i] & VF_BND) ? 1 : 0) | ((pf[i] & VF_CORNER) ? 2 : 0));
  }
  for (int i = 0; i < n2; ++i) {
    if (tri) {
      tri[3 * i] = pe[i].x;
      tri[3 * i + 1] = pe[i].y;
      tri[3 * i + 2] = pe[i].z;
    }
    if (talive) talive[i] = pe[i].w ? 1 : 0;
  }
  return PM_OK;
}

pm_status pm_adjacency(pm_mesh* h, int32_t v, int32_t* nn, int32_t* nnlen, int32_t* ne,
                       int32_t* nelen, int32_t cap) {
  if (!h || !nnlen || !nelen || cap < 0) return fail(PM_ERR_INVALID_ARG, "bad arguments");
  if (pm_status gs = single_only(h, "pm_adjacency")) return gs;
  MeshSet& m = h->set;
  if (v < 0 || v >= m.nv[0]) return fail(PM_ERR_INVALID_ARG, "vertex slot out of range");
  DeviceGuard g(m.device);
  int W = m.S.W;
  std::vector<int> r1(W), r2(W);
  int l1 = 0, l2 = 0;
  cudaMemcpyAsync(&l1, m.S.NNlen + v, sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(&l2, m.S.NElen + v, sizeof(int), cudaMemcpyDeviceToHost, m.stream);
  cudaMemcpyAsync(r1.data(), m.S.NN + (size_t)v * W, W * sizeof(int), cudaMemcpyDeviceToHost,
                  m.stream);
  cudaMemcpyAsync(r2.data(), m.S.NE + (size_t)v * W, W * sizeof(int), cudaMemcpyDeviceToHost,
                  m.stream);
  int err = sync_status(m);
  if (err) return (pm_status)err;
  *nnlen = l1;
  *nelen = l2;
  for (int k = 0; k < l1 && k < cap; ++k) nn[k] = r1[k];
  for (int k = 0; k < l2 && k < cap; ++k) ne[k] = r2[k];
  return PM_OK;
}

pm_status pm_quality(pm_mesh* h, double* q_sum, double* dxy, double* dm) {
  if (!h || !q_sum) return fail(PM_ERR_INVALID_ARG, "mesh and q_sum are required");
  if (pm_status gs = single_only(h, "pm_quality")) return gs;
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  return (pm_status)quality_mesh(m, q_sum, dxy, dm);
}

pm_status pm_quality_arrays_dev(const double* xy, const double* M, int32_t nv, const int32_t* tri,
                                int32_t ne, double* q_sum, double* dxy, double* dm,
                                void* stream) {
  if (!xy || !M || (!tri && ne > 0) || !q_sum || nv < 1 || ne < 0)
    return fail(PM_ERR_INVALID_ARG, "need xy, m, tri, q_sum, nv >= 1, ne >= 0");
  return (pm_status)quality_arrays(xy, M, nv, tri, ne, q_sum, dxy, dm, (cudaStream_t)stream);
}

// ---- batch handles ---------------------------------------------------------------

static pm_status check_batch_sizes(const int32_t* nv, const int32_t* ne, int32_t nmesh) {
  long long vt = 0, et = 0;
  for (int i = 0; i < nmesh; ++i) {
    if (nv[i] < 3 || ne[i] < 1) return fail(PM_ERR_INVALID_ARG, "every mesh needs nv >= 3, ne >= 1");
    vt += nv[i];
    et += ne[i];
  }
  if (vt >= (1LL << 30) || et >= (1LL << 30))
    return fail(PM_ERR_CAPACITY, "batch too large for 32-bit slot ids");
  return PM_OK;
}

pm_status pm_batch_create(const double* xy, const int32_t* nv, const int32_t* tri,
                          const int32_t* ne, int32_t nmesh, const uint8_t* corner,
                          int32_t cap_factor, int device, pm_mesh** out) {
  if (!out) return fail(PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!xy || !nv || !tri || !ne || nmesh < 1 || cap_factor < 1)
    return fail(PM_ERR_INVALID_ARG, "need xy, nv, tri, ne, nmesh >= 1, cap_factor >= 1");
  if (pm_status s = check_batch_sizes(nv, ne, nmesh)) return s;
  // ids and coordinates are checked on the device after the upload (one
  // pass over 20M ids on one host core cost more than the upload itself)
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(PM_ERR_INVALID_ARG, "no such CUDA device");
  DeviceGuard g(device);
  set_mem_pool_retain(device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(PM_ERR_CUDA, "creating a stream");
  return create_set(xy, nv, tri, ne, nmesh, corner, cap_factor, device, s, true, true, out);
}

pm_status pm_batch_create_dev(const double* xy, const int32_t* nv, const int32_t* tri,
                              const int32_t* ne, int32_t nmesh, const uint8_t* corner,
                              int32_t cap_factor, void* stream, pm_mesh** out) {
  if (!out) return fail(PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!xy || !nv || !tri || !ne || nmesh < 1 || cap_factor < 1)
    return fail(PM_ERR_INVALID_ARG, "need xy, nv, tri, ne, nmesh >= 1, cap_factor >= 1");
  if (pm_status s = check_batch_sizes(nv, ne, nmesh)) return s;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, xy) != cudaSuccess || pa.type != cudaMemoryTypeDevice)
    return fail(PM_ERR_INVALID_ARG, "xy is not device memory");
  const int dev = pa.device;
  DeviceGuard g(dev);
  set_mem_pool_retain(dev);
  cudaStream_t s = (cudaStream_t)stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(PM_ERR_CUDA, "creating a stream");
    own = true;
  }
  return create_set(xy, nv, tri, ne, nmesh, corner, cap_factor, dev, s, own, false, out);
}

pm_status pm_batch_size(const pm_mesh* h, int32_t* nmesh) {
  if (!h || !nmesh) return fail(PM_ERR_INVALID_ARG, "mesh and nmesh are required");
  *nmesh = h->set.nmesh;
  return PM_OK;
}

pm_status pm_batch_adapt(pm_mesh* h, const pm_params* params, pm_stats* stats) {
  if (!h || !params) return fail(PM_ERR_INVALID_ARG, "mesh and params are required");
  MeshSet& m = h->set;
  for (int i = 0; i < m.nmesh; ++i)
    if (pm_status s = check_params(params + i)) return s;
  DeviceGuard g(m.device);
  double t0 = now_ms();
  pm_status s = begin_call(m, params, 1);
  if (s) return s;
  CallStats cs;
  cs.init(m.nmesh);
  if ((s = adapt_set(m, params, 1, cs))) return s;
  int err = sync_status(m);
  if (err) return (pm_status)err;
  return fill_stats(m, cs, t0, stats, m.nmesh);
}

static pm_status batch_get(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                           double* M, bool host) {
  if (!h || !nv || !ne) return fail(PM_ERR_INVALID_ARG, "mesh, nv and ne are required");
  MeshSet& m = h->set;
  DeviceGuard g(m.device);
  if (!xy && !tri && !M) return (pm_status)compact_out_set(m, nullptr, nullptr, nullptr, nv, ne);
  if (!host) return (pm_status)compact_out_set(m, xy, tri, M, nv, ne);
  // one compaction into device buffers sized by the used slots, then one
  // copy of each array's live part
  long long vb = 0, eb = 0;
  for (int i = 0; i < m.nmesh; ++i) {
    vb += m.nv[i];
    eb += m.ne[i];
  }
  char* buf = nullptr;
  pm_status s = cuda_status(cudaMallocAsync((void**)&buf, (size_t)std::max(vb, 1LL) * 5 * 8 +
                                                              (size_t)std::max(eb, 1LL) * 12,
                                            m.stream),
                            "output buffers");
  if (s) return s;
  double* dxy = (double*)buf;
  double* dm = dxy + 2 * std::max(vb, 1LL);
  int32_t* dtri = (int32_t*)(dm + 3 * std::max(vb, 1LL));
  int err = compact_out_set(m, xy ? dxy : nullptr, tri ? dtri : nullptr, M ? dm : nullptr, nv, ne);
  if (err) s = (pm_status)err;
  if (!s) {
    long long tv = 0, te = 0;
    for (int i = 0; i < m.nmesh; ++i) {
      tv += nv[i];
      te += ne[i];
    }
    cudaError_t e = cudaSuccess;
    if (xy) e = cudaMemcpyAsync(xy, dxy, tv * 2 * sizeof(double), cudaMemcpyDeviceToHost, m.stream);
    if (!e && M) e = cudaMemcpyAsync(M, dm, tv * 3 * sizeof(double), cudaMemcpyDeviceToHost, m.stream);
    if (!e && tri)
      e = cudaMemcpyAsync(tri, dtri, te * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, m.stream);
    s = cuda_status(e, "copying the output");
  }
  cudaFreeAsync(buf, m.stream);
  err = sync_status(m);
  return s ? s : (pm_status)err;
}

pm_status pm_batch_get_mesh(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                            double* M) {
  return batch_get(h, nv, ne, xy, tri, M, true);
}

pm_status pm_batch_get_mesh_dev(pm_mesh* h, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                                double* M) {
  return batch_get(h, nv, ne, xy, tri, M, false);
}

}  // extern "C"
