/*
 * pm.h - C interface of the GB300 library for round-based independent-set
 * 2D anisotropic mesh adaptation.
 *
 * The method is that of Rokos, Gorman, Jensen and Kelly, "Thread Parallelism
 * for Highly Irregular Computation in Anisotropic Mesh Adaptation":
 *   - Algorithm 1 (Sec. 2.3): repeat {coarsen; swap; refine} until no change
 *     or the iteration limit, then smooth;
 *   - the four kernels of Sec. 2.4 (edge collapse, edge split with refinement
 *     templates, edge flip, quality-constrained vertex smoothing), each swept
 *     until nothing changes (propagation, Sec. 2.4.5);
 *   - rounds of independent sets of the vertex graph (Sec. 3.2), worklists
 *     built by atomic fetch-and-add (Sec. 3.4) and a deferred update that
 *     commits adjacency changes after each set (Sec. 3.3).
 * Inputs follow the problem statement of Sec. 2.3: a triangulation M and a
 * node-wise metric tensor field S.
 *
 * Conventions shared by every entry point:
 *   - All floating point is IEEE binary64.  Vertex coordinates are interleaved
 *     (x0, y0, x1, y1, ...).  The metric of a vertex is the symmetric positive
 *     definite 2x2 tensor [[m00, m01], [m01, m11]], stored as (m00, m01, m11).
 *     Triangles are int32 vertex-id triples in counter-clockwise order.
 *   - Plain pointers are HOST memory and are only read or written during the
 *     call; the library keeps no pointer to them.  Entry points ending in _dev
 *     take DEVICE pointers on the mesh's device, used in stream order on the
 *     mesh's stream (the call returns after the stream has been synchronised
 *     unless stated otherwise).
 *   - The library owns all device state of a mesh (released by
 *     pm_mesh_destroy).  A handle is not thread-safe; different handles may be
 *     used from different threads.
 *   - Every call returns a pm_status.  Invalid pointers, sizes and parameters
 *     are rejected before any device work; the contents of input arrays
 *     (vertex ids, coordinates, metric) are checked on the device after their
 *     upload and before the mesh is built or adapted.  Errors detected on the
 *     device (invalid contents, capacity, timeout) come back through a status
 *     word; pm_last_error() gives a message.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_mesh pm_mesh;

typedef enum {
  PM_OK = 0,
  PM_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter */
  PM_ERR_INVALID_MESH = 2,  /* ids out of range, inverted or overlapping
                               elements, non-manifold vertex, isolated vertex */
  PM_ERR_OOM = 3,           /* device allocation failed */
  PM_ERR_CAPACITY = 4,      /* a fixed capacity was exceeded */
  PM_ERR_CUDA = 5,          /* CUDA runtime error */
  PM_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
} pm_status;

/* Adaptation parameters.
 *   L_low, L_up      metric edge-length bounds: edges shorter than L_low are
 *                    collapsed (Sec. 2.4.1), longer than L_up split (2.4.2);
 *                    0 < L_low < L_up.
 *   q_thresh         quality below which an element's edges may be flipped
 *                    (2.4.3) and its vertices smoothed (2.4.4); >= 0.
 *   max_iter         iteration limit of Algorithm 1 (>= 0).
 *   max_smooth_sweeps  limit of Laplacian smoothing sweeps (>= 0).
 *   seed             seed of the independent-set priorities.
 *   opt_smooth_rounds  rounds of optimisation-based smoothing run after the
 *                    Laplacian sweeps (0 = none).
 *   max_rounds       cap on the rounds of one operator call (0 = none).
 *   select           how a round's independent set is formed (Sec. 3.2):
 *                    PM_SELECT_HASH (0), the candidates whose hash priority
 *                    beats every candidate neighbour's; PM_SELECT_COLOUR (1),
 *                    the vertex graph coloured at the start of every
 *                    collapse, flip and smoothing pass and round r taking
 *                    the candidates of colour r mod (number of colours), with
 *                    the same priority rule among neighbours of that colour.
 *                    Optimisation smoothing always uses PM_SELECT_HASH. */
enum { PM_SELECT_HASH = 0, PM_SELECT_COLOUR = 1 };
typedef struct {
  double L_low, L_up, q_thresh;
  int32_t max_iter, max_smooth_sweeps;
  uint32_t seed;
  int32_t opt_smooth_rounds;
  int32_t max_rounds;
  int32_t select;
} pm_params;

/* Counters of one call: rounds executed (every round that formed a
 * non-empty candidate set), operations applied, whether Algorithm 1 stopped
 * because an iteration changed nothing, and wall time in milliseconds
 * (host clock around the call, device synchronised). */
typedef struct {
  int64_t rounds, collapses, splits, flips, moves;
  int32_t converged;
  double ms;
} pm_stats;

/* Create a mesh on CUDA device `device` from host arrays.
 *   xy[2*nv], tri[3*ne]; corner[nv] (nullable): 1 marks a vertex that must
 *   never move or disappear; when null, corners are the boundary vertices
 *   whose two boundary edges are not collinear.
 *   cap_factor >= 1: initial slot capacity as a multiple of nv and ne (the
 *   mesh grows beyond it by itself when refinement needs room).
 * The metric starts as the identity; set it with pm_set_metric.
 * Builds the adjacency (Sec. 3.1: NN vertex-vertex and NE vertex-element
 * lists, kept as sorted sets) and checks the mesh on the device, after the
 * upload and before any adjacency is built: PM_ERR_INVALID_ARG for a
 * non-finite coordinate; PM_ERR_INVALID_MESH when a vertex id lies outside
 * [0, nv) or repeats in a triangle, a triangle is not counter-clockwise, an
 * edge is used twice in the same direction, a vertex is not manifold, or a
 * vertex is not used. */
pm_status pm_mesh_create(const double* xy, int32_t nv, const int32_t* tri, int32_t ne,
                         const uint8_t* corner, int32_t cap_factor, int device,
                         pm_mesh** out);

/* Same as pm_mesh_create with device input arrays (read on `stream`, a
 * cudaStream_t or null for a new stream of the library's own). */
pm_status pm_mesh_create_dev(const double* xy, int32_t nv, const int32_t* tri, int32_t ne,
                             const uint8_t* corner, int32_t cap_factor, void* stream,
                             pm_mesh** out);

pm_status pm_mesh_destroy(pm_mesh* mesh);

/* Use `stream` (a cudaStream_t on the mesh's device) for all later work. */
pm_status pm_set_stream(pm_mesh* mesh, void* stream);

/* Set the node-wise metric (Sec. 2.1): m[3*nv] = (m00, m01, m11) per vertex
 * in the mesh's current vertex numbering.  PM_ERR_INVALID_ARG unless every
 * entry is finite and m00 > 0, m00*m11 - m01^2 > 0. */
pm_status pm_set_metric(pm_mesh* mesh, const double* m);
pm_status pm_set_metric_dev(pm_mesh* mesh, const double* m);

/* The operators (Sec. 2.4), each run in rounds of independent sets until no
 * candidate is left.  They do not renumber: removed vertices and elements
 * keep their slots until pm_adapt renumbers or pm_get_mesh compacts a copy.
 *   pm_coarsen  collapse every edge shorter than L_low where valid (2.4.1);
 *   pm_refine   split every edge longer than L_up, templates per element;
 *   pm_swap     flip edges whose two elements' minimum quality improves;
 *   pm_smooth   quality-constrained Laplacian smoothing, then
 *               opt_smooth_rounds rounds of optimisation-based smoothing;
 *   pm_adapt    Algorithm 1 (Sec. 2.3) followed by smoothing; renumbers
 *               after every iteration (new vertex ids, slots left in
 *               place) and compacts the slots at the end, so that on
 *               return ids and slots agree as after a full compaction.
 * `stats` may be null. */
pm_status pm_coarsen(pm_mesh* mesh, const pm_params* params, pm_stats* stats);
pm_status pm_refine(pm_mesh* mesh, const pm_params* params, pm_stats* stats);
pm_status pm_swap(pm_mesh* mesh, const pm_params* params, pm_stats* stats);
pm_status pm_smooth(pm_mesh* mesh, const pm_params* params, pm_stats* stats);
pm_status pm_adapt(pm_mesh* mesh, const pm_params* params, pm_stats* stats);

/* Optimisation-based smoothing only (Sec. 2.4.4, gradient form):
 * params->opt_smooth_rounds rounds of independent sets of interior vertices. */
pm_status pm_opt_smooth(pm_mesh* mesh, const pm_params* params, pm_stats* stats);

/* Adapt n meshes together (each with its own parameters and seed): every
 * round of every operator is one launch per kernel over all meshes'
 * worklists, and a run of small rounds one persistent launch.  Results are identical to n separate pm_adapt calls.
 * stats[n] may be null.  All meshes must live on the same device. */
pm_status pm_adapt_batch(pm_mesh** meshes, int32_t n, const pm_params* params,
                         pm_stats* stats);

/* Batch handles: many independent meshes held by one handle, in one device
 * store.  Every round of every operator runs over all of them at once: a
 * round's independent set (Sec. 3.2) is taken over the union of the meshes'
 * vertex graphs, which share no edge, so each mesh's result is the result of
 * adapting it alone (its own seed, parameters and round counter).
 *
 * pm_batch_create: nmesh meshes concatenated, mesh after mesh.
 *   nv[nmesh], ne[nmesh]: vertex and element count of each mesh (nv >= 3,
 *   ne >= 1); xy[2 * sum(nv)], tri[3 * sum(ne)] with vertex ids LOCAL to
 *   each mesh (0 .. nv[i]-1); corner[sum(nv)] nullable (as pm_mesh_create).
 *   cap_factor and device as pm_mesh_create; every mesh is checked as there
 *   (PM_ERR_INVALID_MESH names no mesh).  The handle works with
 *   pm_set_metric (m[3 * sum(nv)], mesh after mesh), the operators
 *   (pm_coarsen ... pm_adapt: the same parameters for every mesh) and
 *   pm_mesh_destroy; pm_get_mesh, pm_get_raw, pm_adjacency and pm_quality
 *   take one-mesh handles only (PM_ERR_INVALID_ARG).
 * pm_batch_create_dev: the same with device arrays xy, tri, corner (read on
 *   `stream`, a cudaStream_t or null for a new stream of the library's own);
 *   nv and ne stay host arrays. */
pm_status pm_batch_create(const double* xy, const int32_t* nv, const int32_t* tri,
                          const int32_t* ne, int32_t nmesh, const uint8_t* corner,
                          int32_t cap_factor, int device, pm_mesh** out);
pm_status pm_batch_create_dev(const double* xy, const int32_t* nv, const int32_t* tri,
                              const int32_t* ne, int32_t nmesh, const uint8_t* corner,
                              int32_t cap_factor, void* stream, pm_mesh** out);

/* Number of meshes a handle holds (1 for pm_mesh_create handles). */
pm_status pm_batch_size(const pm_mesh* mesh, int32_t* nmesh);

/* Algorithm 1 (Sec. 2.3) and smoothing on every mesh of the handle, each
 * with its own parameters params[nmesh]; stats[nmesh] (nullable) receives
 * each mesh's counters, the same as a pm_adapt call on that mesh alone
 * would report (ms: the whole call).  A mesh leaves the outer loop after an
 * iteration that changed nothing or after its max_iter; the call returns
 * when every mesh has, and max_rounds is taken from params[0]. */
pm_status pm_batch_adapt(pm_mesh* mesh, const pm_params* params, pm_stats* stats);

/* Compacted output of every mesh, mesh after mesh, as pm_get_mesh gives it
 * for one mesh: nv[nmesh], ne[nmesh] receive the live counts; xy, tri, m
 * (each nullable) receive sum(nv) vertices and sum(ne) triangles with vertex
 * ids local to each mesh.  With all three null only the counts are written.
 * pm_batch_get_mesh takes host arrays (page-locked ones are filled by direct
 * DMA), pm_batch_get_mesh_dev device arrays on the handle's stream. */
pm_status pm_batch_get_mesh(pm_mesh* mesh, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                            double* m);
pm_status pm_batch_get_mesh_dev(pm_mesh* mesh, int32_t* nv, int32_t* ne, double* xy,
                                int32_t* tri, double* m);

/* Copy out the mesh, compacted (live vertices and elements in ascending slot
 * order) with every triangle rotated so its smallest vertex id comes first.
 * Two-call protocol: with null arrays only *nv and *ne are written.
 * xy[2*nv], tri[3*ne], m[3*nv] may each be null.  Host arrays in page-locked
 * memory (cudaHostAlloc / pinned) are filled by direct DMA; pageable ones go
 * through the CUDA driver's staging copy, several times slower. */
pm_status pm_get_mesh(pm_mesh* mesh, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                      double* m);
pm_status pm_get_mesh_dev(pm_mesh* mesh, int32_t* nv, int32_t* ne, double* xy, int32_t* tri,
                          double* m);

/* Raw slot state without compaction (for round-by-round comparisons):
 * *nv, *ne = slots in use; xy[2*nv], m[3*nv], tri[3*ne], valive[nv],
 * talive[ne], vflag[nv] (bit0 boundary, bit1 corner).  Null arrays: sizes
 * only. */
pm_status pm_get_raw(pm_mesh* mesh, int32_t* nv, int32_t* ne, double* xy, double* m,
                     int32_t* tri, uint8_t* valive, uint8_t* talive, uint8_t* vflag);

/* Sorted adjacency rows of vertex slot v (Sec. 3.1): nn[cap], ne[cap];
 * *nnlen, *nelen receive the full row lengths. */
pm_status pm_adjacency(pm_mesh* mesh, int32_t v, int32_t* nn, int32_t* nnlen, int32_t* ne,
                       int32_t* nelen, int32_t cap);

/* Element quality functional (Sec. 2.2, Vasilevskii et al.) and its gradient
 * over the live elements of the mesh.  *q_sum = sum of qualities; dxy[2*nv]
 * and dm[3*nv] (nullable) receive d(q_sum)/d(x,y) and d(q_sum)/d(m00,m01,m11)
 * per vertex slot (zero for dead slots), each the sum over the vertex's
 * elements in ascending element id. */
pm_status pm_quality(pm_mesh* mesh, double* q_sum, double* dxy, double* dm);

/* The same functional on plain device arrays (no mesh handle), for use under
 * automatic differentiation: xy[2*nv], m[3*nv], tri[3*ne] on the current
 * device (ne may be 0: the sum is 0).  q_sum (1 double), dxy[2*nv], dm[3*nv]
 * are device outputs; dxy and dm may be null for the forward value only.
 * Runs on `stream` (cudaStream_t, null = legacy default stream), waits for
 * it and returns the device status: PM_ERR_INVALID_MESH when a vertex id in
 * tri lies outside [0, nv), PM_ERR_TIMEOUT when the gradient's scan gave up
 * a bounded wait; the outputs then hold NaN.  Temporary device memory (one
 * block) is allocated and released in the call (PM_ERR_OOM when that
 * fails).  Gradient rows: each vertex sums its elements in ascending id. */
pm_status pm_quality_arrays_dev(const double* xy, const double* m, int32_t nv,
                                const int32_t* tri, int32_t ne, double* q_sum, double* dxy,
                                double* dm, void* stream);

/* Measurement support (not part of the method).
 * pm_kernel_launches: number of CUDA kernels this library has launched in
 * the process so far.
 * pm_profile_enable: while `kernel_substring` is non-empty, every launch of a
 * library kernel whose name contains it is bracketed by CUDA events on the
 * stream it runs on; enabling (or disabling with null/"") clears earlier
 * records.  pm_profile_read waits for the recorded launches and returns their
 * summed device time and count, and (work, nullable) the algorithmic work the
 * profiled kernel counted: FP64 operations (+ - * / sqrt, one each) along
 * the paths its threads took, for kernels that count (k_smooth_eval), else 0. */
uint64_t pm_kernel_launches(void);
pm_status pm_profile_enable(const char* kernel_substring);
pm_status pm_profile_read(double* total_ms, int64_t* launches, double* work);

/* Measurement support: the FP64 add and multiply throughput of the current
 * device, in G operations per second, from a kernel that keeps every SM's
 * FP64 pipe busy with independent additions and multiplications (no fused
 * multiply-add).  Runs on the default stream and synchronises; about 20 ms.
 * The paper has no counterpart. */
pm_status pm_fp64_peak(double* gops);

/* Test support: the bounded wait of the persistent rounds' grid barrier.  On
 * the current device, one block per SM waits at a barrier that no arrival can
 * complete; each block gives up after limit_ms (0 < limit_ms <= 2000) and
 * records PM_ERR_TIMEOUT in the device status word.  *device_status receives
 * that word, *elapsed_ms the kernel's duration.  Returns PM_OK when the
 * kernel ran and ended (the device stays usable), PM_ERR_INVALID_ARG for a
 * null pointer or a limit out of range, PM_ERR_CUDA / PM_ERR_OOM on a runtime
 * failure.  Runs on the default stream and synchronises.  The paper has no
 * counterpart. */
pm_status pm_selftest_wait_timeout(double limit_ms, int32_t* device_status, double* elapsed_ms);

/* Test support: out[i] = x[i] / 3.0 for i < n, computed the way the quality
 * functional (Sec. 2.2) forms its means of three terms on the device (one
 * multiplication and two fused multiply-adds, equal to the IEEE quotient).
 * x[n] and out[n] are device arrays; runs on `stream` (cudaStream_t, null =
 * legacy default stream) without synchronising.  PM_ERR_INVALID_ARG for a
 * null pointer or n < 0.  The paper has no counterpart. */
pm_status pm_selftest_div3_dev(const double* x, double* out, int64_t n, void* stream);

/* Test support: out[i] = the exact orientation sign (-1, 0, +1) of the points
 * (px, py), (qx, qy), (rx, ry) = pts[6i .. 6i+5], the predicate behind every
 * validity decision of the operators (an element counter-clockwise, a point
 * in the closed element, a corner; Sec. 2.4): the sign of the determinant of
 * the doubles' exact values.  pts[6n] and out[n] are device arrays; runs on
 * `stream` without synchronising.  PM_ERR_INVALID_ARG for a null pointer or
 * n < 0. */
pm_status pm_selftest_orient_dev(const double* pts, int32_t* out, int64_t n, void* stream);

/* pm_quality_arrays_dev for callers that cannot allocate device memory
 * during the call (a framework that has already reserved the device memory
 * for its own allocator, a latency-bound loop, or a program that allows no
 * allocation after start-up).  The paper has no counterpart: this is a
 * service of this library.  Same arguments, results, stream behaviour and
 * statuses as pm_quality_arrays_dev, but every temporary lives in one fixed array
 * (about 9.6 MB) compiled into the library, which each GPU that loads the
 * library keeps until the process exits; the call allocates and frees
 * nothing.  Limits: ne <= 65536 elements and nv <= 65536 vertices, else
 * PM_ERR_CAPACITY.  The first call on a device looks up the array's device
 * address (with that device current), so make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * race, so order them on one stream or synchronise in between. */
pm_status pm_quality_arrays_noalloc_dev(const double* xy, const double* m, int32_t nv,
                                        const int32_t* tri, int32_t ne, double* q_sum,
                                        double* dxy, double* dm, void* stream);

/* Launch shapes (a service of this library; the paper's counterpart is its
 * load balancing, Sec. 3.5).  Process-wide; no choice changes any result.
 *   block[4], blocks_per_sm[4]: per operator (collapse, flip, split,
 *     smoothing), threads per block (64, 128 or 256) and the cap on blocks
 *     per SM (1..32) of the one-kernel-per-phase round kernels: together they
 *     set the worklist chunk each thread walks.
 *   rounds_limit[3]: per operator (collapse, flip, smoothing), the largest
 *     list (vertices) whose rounds run inside one persistent launch (0: never;
 *     at most 2^30).
 *   rounds_blocks_per_sm[3]: resident blocks per SM of those persistent
 *     launches (1 or 2; fewer when the kernel's registers allow fewer).
 *   fuse_limit[2]: flips, smoothing: inside the persistent launch, lists up
 *     to this size (and at most one per 8-lane tile of the grid) are scanned
 *     and evaluated in one phase.
 * Defaults: 128 threads, 16 blocks per SM, 131072, 1 block, fuse_limit
 * {0, 2^30} (on the 2M workload the one-phase flip evaluation was slower). */
typedef struct {
  int32_t block[4];
  int32_t blocks_per_sm[4];
  int32_t rounds_limit[3];
  int32_t rounds_blocks_per_sm[3];
  int32_t fuse_limit[2];
} pm_tuning;

/* Set the launch shapes (null: the defaults).  PM_ERR_INVALID_ARG for a value
 * out of range (nothing changes then).  Takes effect at the next operator
 * call; an explicit setting is never replaced by a tuning cache. */
pm_status pm_set_tuning(const pm_tuning* t);
pm_status pm_get_tuning(pm_tuning* t);

/* Load the entry of a tuning cache (JSON written by the package's autotuner)
 * for GPU model `gpu_name` (null: the current device's name) and this
 * library build (pm_build_id).  PM_OK when an entry was applied;
 * PM_ERR_INVALID_ARG when the file is missing or holds no valid entry for
 * them (the current shapes stay).  Without any call, the first mesh created
 * in the process applies the first of these caches that holds an entry for
 * its GPU and build: the file named by the environment variable
 * PM_TUNING_CACHE, tuning.json beside the library, tuning.json in the
 * directory above the library's. */
pm_status pm_tuning_load(const char* path, const char* gpu_name);

/* Where the current shapes come from: "default", "set" or "cache <path>". */
const char* pm_tuning_source(void);

/* Identity of this library build (a hash of its sources and flags), the key
 * of tuning cache entries. */
const char* pm_build_id(void);

const char* pm_status_string(pm_status s);

/* Message of the last error on the calling thread ("" if none). */
const char* pm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
