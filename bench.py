"""Benchmark: adapted elements/s of the full 2D adaptation loop on GB300,
batched against one mesh per launch.

Default workload (the metric's own): 512 independent unit-square meshes,
initial sizes log-uniform in 1k..200k triangles (19.1M in all), each with its
own seeded constant anisotropic metric (rotation U[0, pi), aspect
log-U[1, 100], size log-U[0.002, 0.05]).  One step adapts all 512:
  pm_batch_create_dev (ingest + adjacency of every mesh in one store),
  pm_set_metric_dev, pm_batch_adapt (Algorithm 1 with every operator round of
  every mesh in the same launches, smoothing, renumbering),
  pm_batch_get_mesh_dev (compacted output of every mesh).
Inputs are resident in HBM when a step's timer starts (CUDA events on the
library's stream); the L2 is flushed (256 MiB write) between steps, outside
the timed region.  value = output triangles of all steps of all ranks / max
over ranks of the summed step time.  Beside it: the same 512 meshes adapted
one mesh per launch sequence (pm_mesh_create_dev, pm_set_metric_dev,
pm_adapt, pm_get_mesh_dev per mesh), and e2e through the host-pointer calls
with pinned buffers.

Other workloads (--workload): psi2m / psi20m / paper550k (one psi-Hessian
mesh, Sec. 4's synthetic benchmark at t = 0), grad (quality forward and
backward, optimisation smoothing), psi_t (time-dependent psi).

--impl reference times the CPU oracle (sequential C++) on the same workload,
one oracle process per host core, each step a size-stratified quarter of the
meshes; see the `cpu_baseline` key.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Adapted elements/s, full 2D adapt loop, 1 GB300; batched vs one-mesh-per-launch"
WORKLOAD = "psi-Hessian anisotropic adaptation, 257x257 jittered grid (131,072 triangles) -> ~2.1M triangles"
BATCH_WORKLOAD = ("batch of 512 unit-square meshes, initial sizes log-uniform 1k-200k triangles "
                  "(19.1M), constant anisotropic metrics (theta U[0,pi), aspect log-U[1,100], "
                  "h log-U[0.002,0.05]), seed 5")
# bounded CPU sample of the same workload family (about 10-20 s of oracle work)
SAMPLE = dict(n=181, target=1.0e6, seed=2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-steps", type=int, default=2,
                    help="timed steps of the one-mesh-per-launch comparison (batch workload)")
    ap.add_argument("--roofline-kernel", default=None)
    ap.add_argument("--select", default="hash", choices=["hash", "colour"],
                    help="how a round's independent set is formed: hash-priority local maxima "
                         "(default) or colour classes (the vertex graph coloured per pass)")
    ap.add_argument("--batch-every", type=int, default=1,
                    help="batch workload: every n-th mesh by initial size (a sub-batch for "
                         "profiling captures; 1 = the 512-mesh batch)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="device-resident steps only (no e2e pass, no CPU baseline)")
    ap.add_argument("--workload", default="batch",
                    choices=["psi2m", "psi20m", "paper550k", "batch", "grad", "psi_t"],
                    help="batch (default, the headline line: 512 meshes batched vs one mesh "
                         "per launch); psi2m / psi20m / paper550k: one psi-Hessian mesh; "
                         "grad: quality forward+backward and optimisation smoothing; "
                         "psi_t: time-dependent psi, each step re-adapts the last mesh")
    return ap.parse_args()


def dist_init(n, host_only=False):
    """Rank, world size and local rank from the launcher's environment; a
    process group when several ranks run (gloo for the oracle arm, whose
    ranks hold no GPU work)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if n > 1 and not host_only else "gloo")
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
                for name, val in zip(names, s[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# The dominant kernel of a step and its roofline.  The candidates are the
# kernels that carry the evaluation arithmetic: the persistent round kernels
# (small rounds) and the one-kernel-per-phase evaluation kernels (large
# rounds).  The one with the most event time in an untimed step is reported.
# Their arithmetic is FP64 and DRAM traffic is far below the HBM roofline
# (ncu), so the ceiling is the FP64 issue rate: ncu reports 304 FP64 results
# per cycle for the whole GPU
# (sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained; 2 per SM
# on 152 SMs) at the 2070 MHz maximum SM clock.  Work = FP64 operations
# (+ - * / sqrt, one each) along the paths the kernel took, counted by the
# kernel while profiled.
ROOFLINE_CANDIDATES = ("k_swap_rounds", "k_smooth_rounds", "k_coarsen_rounds", "k_smooth_eval",
                       "k_coarsen_check", "k_swap_edge")
FP64_RESULTS_PER_CYCLE = 304


def roofline(kname, kms, klaunch, kwork, total_ms, peaks, how, fp64_meas=None, workload=None):
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = FP64_RESULTS_PER_CYCLE * mhz * 1e6 / 1e9  # G FP64 ops/s
    out = {"kernel": kname, "bound": "alu", "unit": "GFLOP/s (FP64 ops)",
           "peak": peak, "peak_source": f"derived: {FP64_RESULTS_PER_CYCLE} FP64 results/cycle x "
                                        f"{mhz:.0f} MHz (sm_max_mhz {how})",
           "achieved": None, "frac": None,
           "traffic": traffic_of(kname, workload) if workload else None,
           "kernel_ms_per_step_share": (kms / total_ms) if total_ms else None,
           "launches": klaunch, "kernel_ms": kms, "fp64_ops": kwork}
    if fp64_meas:
        out["peak_measured"] = fp64_meas
        out["peak_measured_source"] = ("pm_fp64_peak: independent FP64 multiply and add chains "
                                       "on every SM, best of 3 runs")
    if kms > 0 and kwork > 0:
        ach = kwork / (kms / 1e3) / 1e9
        out["achieved"] = ach
        out["frac"] = ach / peak
        if fp64_meas:
            out["frac_of_measured"] = ach / fp64_meas
    return out


def traffic_of(kname, workload):
    """DRAM bytes per launch of the kernel on this workload from the committed
    ncu summary (profiles/traffic.txt: "kernel workload bytes_per_launch" per
    line), or None when no capture of the current kernel exists."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split("#", 1)[0].split()
                if len(parts) >= 3 and parts[0] == kname and parts[1] == workload:
                    return float(parts[2])
    except OSError:
        pass
    return None


def timed(fn, dev):
    import torch

    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    r = fn()
    torch.cuda.synchronize(dev)
    return r, time.perf_counter() - t


# ---- CPU oracle over the batch (a pool of spawned processes, one per core) ----

_WS = None


def _oracle_batch_mesh(i):
    """Adapt batch mesh i with the oracle; (i, output triangles, seconds)."""
    global _WS
    from oracle import oracle as O
    from paper_1505_04694_gb300 import inputs

    if _WS is None:
        _WS = inputs.batch_workloads()
    w = _WS[i]
    o = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
    t = time.perf_counter()
    o.adapt(O.make_params(seed=w.params.seed))
    dt = time.perf_counter() - t
    return i, int(o.get_mesh()[1].shape[0]), dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_pool(procs):
    """A pool of spawned oracle workers, warmed (inputs built, oracle loaded)."""
    import multiprocessing as mp

    pool = mp.get_context("spawn").Pool(procs)
    pool.map(_oracle_batch_mesh, [int(i) for i in small_meshes(procs)], chunksize=1)
    return pool


def small_meshes(k):
    from paper_1505_04694_gb300 import inputs

    sizes = [w.tri.shape[0] for w in inputs.batch_workloads()]
    return sorted(range(len(sizes)), key=lambda i: sizes[i])[:k]


def oracle_batch(pool, idx):
    """Adapt meshes idx over the pool (largest first); (triangles, wall s)."""
    from paper_1505_04694_gb300 import inputs

    sizes = {i: w.tri.shape[0] for i, w in enumerate(inputs.batch_workloads())}
    order = sorted(idx, key=lambda i: -sizes[i])
    t = time.perf_counter()
    res = pool.map(_oracle_batch_mesh, order, chunksize=1)
    return sum(r[1] for r in res), time.perf_counter() - t


def stratified(k, parts, idx=None):
    """Part k (of `parts`) of the batch meshes `idx`, stratified by initial size."""
    from paper_1505_04694_gb300 import inputs

    ws = inputs.batch_workloads()
    idx = list(range(len(ws))) if idx is None else list(idx)
    order = sorted(idx, key=lambda i: ws[i].tri.shape[0])
    return [i for r, i in enumerate(order) if r % parts == k % parts]


def run_batch(args, rank, world, local):
    """The 512-mesh batch: one pm_batch_* sequence per step (every round of
    every operator over all meshes at once) against the same meshes one
    mesh per launch sequence, same GPU, same inputs.  Over N ranks the
    meshes are split by size with no collective in the data path."""
    import numpy as np
    import torch

    from paper_1505_04694_gb300 import inputs, pm, shard

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    ws = inputs.batch_workloads()
    if args.batch_every > 1:
        order = sorted(range(len(ws)), key=lambda i: ws[i].tri.shape[0])
        ws = [ws[i] for i in order[::args.batch_every]]
    batch_key = f"batch{len(ws)}"
    parts = shard.partition([w.tri.shape[0] for w in ws], world)
    mine_idx = parts[rank]
    mine = [ws[i] for i in mine_idx]
    nv = np.array([w.xy.shape[0] for w in mine], np.int32)
    ne = np.array([w.tri.shape[0] for w in mine], np.int32)
    ov = np.concatenate([[0], np.cumsum(nv)])
    oe = np.concatenate([[0], np.cumsum(ne)])
    h_xy = np.ascontiguousarray(np.concatenate([w.xy for w in mine]))
    h_tri = np.ascontiguousarray(np.concatenate([w.tri for w in mine]).astype(np.int32))
    h_m = np.ascontiguousarray(np.concatenate([w.m for w in mine]))
    xy_d = torch.tensor(h_xy, device=dev)
    tri_d = torch.tensor(h_tri, device=dev)
    m_d = torch.tensor(h_m, device=dev)
    sel = pm.SELECT_COLOUR if args.select == "colour" else pm.SELECT_HASH
    params = [pm.Params(seed=w.params.seed, select=sel) for w in mine]
    cap = 40_000_000
    oxy = torch.empty((cap, 2), dtype=torch.float64, device=dev)
    otri = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    om_ = torch.empty((cap, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.batch_every == 1:
        pool = oracle_pool(host_cores())  # spawned before any GPU work of this process

    last = {"rounds": 0}

    def step():
        b = pm.Batch.from_device(xy_d, nv, tri_d, ne, stream=sp)
        b.set_metric_dev(m_d)
        st = b.adapt(params)
        last["rounds"] = sum(x["rounds"] for x in st)
        _, c = b.get_mesh_dev(oxy, otri, om_)
        b.close()
        return int(c.sum())

    def step_single():
        n = 0
        for i in range(len(mine)):
            g = pm.Mesh.from_device(xy_d[ov[i]:ov[i + 1]], tri_d[oe[i]:oe[i + 1]], stream=sp)
            g.set_metric_dev(m_d[ov[i]:ov[i + 1]])
            g.adapt(params[i])
            n += g.get_mesh_dev(oxy, otri, om_)[1]
            g.close()
        return n

    def timed_steps(fn, k):
        ms, tris = 0.0, 0
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tris += fn()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return tris, ms

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    kname, cand_ms, fp64_meas = choose_roofline_kernel(args, step, flush, pm)
    barrier()
    pm.profile_enable(kname)
    launches0 = pm.kernel_launches()
    with ClockSampler(local) as clk:
        tris, total_ms = timed_steps(step, args.steps)
    barrier()
    launches = pm.kernel_launches() - launches0
    kms, klaunch, kwork = pm.profile_read()
    pm.profile_enable(None)
    t_local = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    n_local = torch.tensor([float(tris)], dtype=torch.float64, device=dev)
    # one mesh per launch sequence, the same meshes (fewer timed steps: each
    # takes seconds); left out of --kernel-only runs, whose launch lists hold
    # the batched steps alone
    s_local = torch.tensor([1.0, 0.0], dtype=torch.float64, device=dev)
    if not args.kernel_only:
        step_single()
        s_tris, s_ms = timed_steps(step_single, max(1, args.single_steps))
        s_local = torch.tensor([s_ms, float(s_tris)], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(n_local, op=dist.ReduceOp.SUM)
        tmax = s_local[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(s_local, op=dist.ReduceOp.SUM)
        s_local[0] = tmax[0]
    t_max = float(t_local.item())
    value = float(n_local.item()) / (t_max / 1e3)
    single_value = float(s_local[1].item()) / (float(s_local[0].item()) / 1e3)
    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "elements/s",
                              "ms_per_step": t_max / args.steps, "gpu_launches": launches,
                              "select": args.select, "rounds_per_step": last["rounds"],
                              "output_triangles_per_step": tris // max(args.steps, 1)}))
        return
    # end to end through the host-pointer calls, inputs and outputs pinned
    pin = [torch.from_numpy(a).pin_memory() for a in (h_xy, h_tri, h_m)]
    p_xy, p_tri, p_m = (t.numpy() for t in pin)
    out_h = (torch.empty((cap, 2), dtype=torch.float64).pin_memory().numpy(),
             torch.empty((cap, 3), dtype=torch.int32).pin_memory().numpy(),
             torch.empty((cap, 3), dtype=torch.float64).pin_memory().numpy())
    e2e_s, e2e_tris, d2h = 0.0, 0, 0
    for i in range(1 + args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        b = pm.Batch.from_arrays(p_xy, nv, p_tri, ne, device=local)
        b.set_metric(p_m)
        b.adapt(params)
        got = b.get_meshes(out=out_h)
        b.close()
        dt = time.perf_counter() - t
        if i >= 1:
            e2e_s += dt
            e2e_tris += sum(g[1].shape[0] for g in got)
            d2h = sum(g[0].nbytes + g[1].nbytes + g[2].nbytes for g in got)
    h2d = p_xy.nbytes + p_tri.nbytes + p_m.nbytes
    peaks, how = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD if len(ws) == 512 else
                   f"{len(ws)} of the 512 meshes (every {args.batch_every}-th by initial size) of "
                   + BATCH_WORKLOAD, "meshes": len(ws),
                   "output_triangles_per_step": tris // max(args.steps, 1),
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "independent_sets": args.select, "rounds_per_step": last["rounds"],
                   "parallelism": f"meshes split over {world} GPUs by size" if world > 1
                   else "single GPU"},
        "one_mesh_per_launch": {
            "value": single_value, "unit": "elements/s",
            "ms_per_step": float(s_local[0].item()) / max(1, args.single_steps),
            "steps": max(1, args.single_steps),
            "batched_speedup": value / single_value,
            "how": "per mesh: pm_mesh_create_dev, pm_set_metric_dev, pm_adapt, "
                   f"pm_get_mesh_dev; CUDA events around all {len(ws)}"},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_tris / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "pm_batch_create + pm_set_metric + pm_batch_adapt + pm_batch_get_mesh, "
                       "inputs and outputs in pinned host buffers, wall clock per step"},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / max(args.steps, 1),
        "tuning": dict(pm.get_tuning(), source=pm.tuning_source()),
        "roofline": dict(roofline(kname, kms, klaunch, kwork, total_ms, peaks, how, fp64_meas,
                                  batch_key),
                         chosen_from={k: round(v, 4) for k, v in cand_ms.items()},
                         chosen_by="largest event time in one untimed step (ms)"),
    }
    if pool is not None:
        ncore = host_cores()
        model = cpu_model()
        allm = list(range(len(ws)))
        ot, osec = oracle_batch(pool, allm)
        pool.close()
        one = stratified(0, 16)
        pool1 = oracle_pool(1)
        ot1, osec1 = oracle_batch(pool1, one)
        pool1.close()
        line["cpu_baseline"] = {
            "value": ot / osec, "unit": "elements/s", "cores": ncore, "kind": "oracle",
            "sample": f"all {len(allm)} meshes of the batch, one spawned oracle process per host "
                      f"core ({ncore} x {model}), largest meshes first; oracle = sequential "
                      f"C++ -O3 -ffp-contract=off; value = output triangles / wall time",
            "seconds": osec}
        line["cpu_baseline_1core"] = {
            "value": ot1 / osec1, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(one)} of the {len(allm)} meshes (every 16th by initial size) on one "
                      f"core ({model}), sequential", "seconds": osec1}
    if rank == 0:
        print(json.dumps(line), flush=True)


def choose_roofline_kernel(args, step, flush, pm):
    """The dominant evaluation kernel of a step (most event time in one untimed
    step each), and the measured FP64 peak."""
    fp64_meas = None if args.kernel_only else pm.fp64_peak()
    cand_ms = {}
    for name in ([args.roofline_kernel] if args.roofline_kernel else ROOFLINE_CANDIDATES):
        pm.profile_enable(name)
        flush.zero_()
        step()
        cand_ms[name] = pm.profile_read()[0]
    pm.profile_enable(None)
    return max(cand_ms, key=cand_ms.get), cand_ms, fp64_meas


def run_grad(args, rank, world, local):
    """The ~1M-vertex adapted mesh of the 2M workload: quality forward +
    hand-written backward through torch.autograd (elements/s), and 20 rounds
    of optimisation-based smoothing on independent sets."""
    import torch

    from paper_1505_04694_gb300 import inputs, pm
    from paper_1505_04694_gb300.autograd import quality

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.anisotropic_2m()
    g = pm.Mesh.from_host(w.xy, w.tri, device=local)
    g.set_metric(w.m)
    g.adapt(pm.Params(seed=w.params.seed))
    xy0, tri0, m0 = g.get_mesh()
    g.close()
    xy = torch.tensor(xy0, device=dev, requires_grad=True)
    m = torch.tensor(m0, device=dev, requires_grad=True)
    tri = torch.tensor(tri0, dtype=torch.int32, device=dev)

    def fwd_bwd():
        xy.grad = None
        m.grad = None
        q = quality(xy, m, tri)
        q.backward()
        return q

    for _ in range(max(args.warmup, 1)):
        fwd_bwd()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        fwd_bwd()
    e1.record(stream)
    e1.synchronize()
    ms_fb = e0.elapsed_time(e1) / args.steps
    opt_ms = []
    for _ in range(args.steps):
        h = pm.Mesh.from_host(xy0, tri0, device=local)
        h.set_metric(m0)
        st, dt = timed(lambda: h.opt_smooth(pm.Params(seed=4, opt_smooth_rounds=20)), dev)
        opt_ms.append(1e3 * dt)
        h.close()
    if rank == 0:
        print(json.dumps({
            "metric": "quality functional forward+backward elements/s", "value":
            tri0.shape[0] / (ms_fb / 1e3), "unit": "elements/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_fb, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"adapted psi mesh, {xy0.shape[0]} vertices, "
                                   f"{tri0.shape[0]} triangles"},
            "opt_smooth_20_rounds_ms": sorted(opt_ms)[len(opt_ms) // 2],
            "opt_smooth_moves": st["moves"],
        }), flush=True)


def run_time_series(args, rank, world, local):
    """Sec. 4's time-dependent benchmark at the paper's size: after an
    untimed adaptation at t = 0, every step re-adapts the previous step's
    mesh to the metric of psi(x, y, t_k), t_k = k T / 50, evaluated on the
    host at that mesh's vertices (input generation, untimed).  The timed step
    is the metric upload from device memory, Algorithm 1 with smoothing, and
    the compacted output."""
    import numpy as np
    import torch

    from paper_1505_04694_gb300 import inputs, pm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = inputs.paper_550k()
    target = 5.5e5
    params = pm.Params(seed=w.params.seed)
    g = pm.Mesh.from_host(w.xy, w.tri, cap_factor=2, device=local)
    g.set_stream(stream.cuda_stream)  # the events below are recorded on this stream
    g.set_metric(w.m)
    g.adapt(params)
    cap_out = 4_000_000
    oxy = torch.empty((cap_out, 2), dtype=torch.float64, device=dev)
    otri = torch.empty((cap_out, 3), dtype=torch.int32, device=dev)
    om_ = torch.empty((cap_out, 3), dtype=torch.float64, device=dev)
    k = 0

    def next_metric():
        nonlocal k
        k += 1
        xy, tri, _ = g.get_mesh()
        return inputs.psi_metric(xy, tri, target, phase=inputs.psi_phase(k))

    for _ in range(args.warmup):
        g.set_metric(next_metric())
        g.adapt(params)
    launches = 0
    total_ms = 0.0
    tris = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            m_d = torch.tensor(next_metric(), dtype=torch.float64, device=dev)
            torch.cuda.synchronize(dev)
            l0 = pm.kernel_launches()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.set_metric_dev(m_d)
            g.adapt(params)
            nv, ne = g.get_mesh_dev(oxy, otri, om_)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            launches += pm.kernel_launches() - l0
            tris += ne
    # end to end: host metric in pinned memory, output into pinned arrays
    out_h = (torch.empty((cap_out, 2), dtype=torch.float64).pin_memory().numpy(),
             torch.empty((cap_out, 3), dtype=torch.int32).pin_memory().numpy(),
             torch.empty((cap_out, 3), dtype=torch.float64).pin_memory().numpy())
    e2e_s, e2e_tris, h2d, d2h = 0.0, 0, 0, 0
    for _ in range(args.steps):
        m_h = torch.from_numpy(next_metric()).pin_memory().numpy()
        t = time.perf_counter()
        g.set_metric(m_h)
        g.adapt(params)
        oxyh, otrih, omh = g.get_mesh(out=out_h)
        e2e_s += time.perf_counter() - t
        e2e_tris += otrih.shape[0]
        h2d += m_h.nbytes
        d2h += oxyh.nbytes + otrih.nbytes + omh.nbytes
    g.close()
    if rank == 0:
        print(json.dumps({
            "metric": "adapted elements/s, time-dependent psi (each step re-adapts the last mesh)",
            "value": tris / (total_ms / 1e3), "unit": "elements/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"time-dependent psi (Sec. 4), {w.name}, time steps "
                                   f"{args.warmup + 1}..{args.warmup + args.steps} of 50 per "
                                   f"period", "output_triangles_per_step": tris // args.steps},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_tris / e2e_s, "unit": "elements/s",
                    "h2d_bytes_per_step": h2d // args.steps,
                    "d2h_bytes_per_step": d2h // args.steps,
                    "how": "pm_set_metric + pm_adapt + pm_get_mesh on the previous step's "
                           "mesh, metric and output in pinned host buffers, wall clock"},
            "gpu_launches": launches, "roofline": None,
        }), flush=True)


def cpu_baseline_run(samples=1):
    """Oracle (sequential C++) on the bounded sample; returns elements/s etc."""
    from oracle import oracle as O
    from paper_1505_04694_gb300 import inputs

    w = inputs.psi_workload(SAMPLE["n"], SAMPLE["target"], True, SAMPLE["seed"])
    vals = []
    for _ in range(samples):
        om = O.OracleMesh(w.xy, w.tri).set_metric(w.m)
        t = time.perf_counter()
        om.adapt(O.make_params(seed=SAMPLE["seed"]))
        _, tri, _ = om.get_mesh()
        dt = time.perf_counter() - t
        vals.append((tri.shape[0], dt))
    return vals


def sample_desc():
    return (f"oracle (sequential C++, -O3 -ffp-contract=off) full adapt loop on the same workload "
            f"family at {SAMPLE['n']}x{SAMPLE['n']} jittered grid, target {SAMPLE['target']:.0e} "
            f"triangles; value = output triangles / wall time")


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload != "batch":
        return run_reference_single(args)
    ncore = host_cores()
    model = cpu_model()
    pool = oracle_pool(ncore)
    for _ in range(args.warmup):
        oracle_batch(pool, small_meshes(ncore))
    tri, secs = 0, 0.0
    for k in range(args.steps):
        t, dt = oracle_batch(pool, stratified(k, 4))
        tri += t
        secs += dt
    pool.close()
    v = tri / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "meshes": 512,
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "parallelism": "single GPU"},
        "cpu_baseline": {"value": v, "unit": "elements/s", "cores": ncore, "kind": "oracle",
                         "sample": f"step k adapts a size-stratified quarter of the 512 meshes "
                                   f"(rank by initial size = k mod 4), one spawned oracle process "
                                   f"per host core ({ncore} x {model}); warm-up steps adapt the "
                                   f"{ncore} smallest meshes; oracle = sequential C++ -O3 "
                                   f"-ffp-contract=off"},
        "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_single(args):
    for _ in range(args.warmup):
        cpu_baseline_run(1)
    res = cpu_baseline_run(args.steps)
    tri = sum(r[0] for r in res)
    secs = sum(r[1] for r in res)
    v = tri / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{SAMPLE}"},
        "cpu_baseline": {"value": v, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": sample_desc()},
        "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args.gpus, host_only=args.impl == "reference")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    if args.workload == "grad":
        run_grad(args, rank, world, local)
        return
    if args.workload == "psi_t":
        run_time_series(args, rank, world, local)
        return
    import numpy as np
    import torch

    from paper_1505_04694_gb300 import inputs, pm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    w = {"psi2m": inputs.anisotropic_2m, "psi20m": inputs.anisotropic_20m,
         "paper550k": inputs.paper_550k}[args.workload]()
    workload_name = WORKLOAD if args.workload == "psi2m" else w.name
    params = pm.Params(seed=w.params.seed)
    xy_d = torch.tensor(w.xy, dtype=torch.float64, device=dev)
    tri_d = torch.tensor(w.tri, dtype=torch.int32, device=dev)
    m_d = torch.tensor(w.m, dtype=torch.float64, device=dev)
    cap_out = 40_000_000 if args.workload == "psi20m" else 4_000_000
    oxy = torch.empty((cap_out, 2), dtype=torch.float64, device=dev)
    otri = torch.empty((cap_out, 3), dtype=torch.int32, device=dev)
    om_ = torch.empty((cap_out, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        g = pm.Mesh.from_device(xy_d, tri_d, cap_factor=2, stream=sp)
        g.set_metric_dev(m_d)
        g.adapt(params)
        nv, ne = g.get_mesh_dev(oxy, otri, om_)
        g.close()
        return ne

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    # untimed, before the warm-up steps; left out of --kernel-only runs so that
    # their launch lists hold the step's kernels alone
    fp64_meas = None if args.kernel_only else pm.fp64_peak()
    cand_ms = {}
    for name in ([args.roofline_kernel] if args.roofline_kernel else ROOFLINE_CANDIDATES):
        pm.profile_enable(name)
        flush.zero_()
        step()
        cand_ms[name] = pm.profile_read()[0]
    pm.profile_enable(None)
    barrier()
    kname = max(cand_ms, key=cand_ms.get)
    pm.profile_enable(kname)
    launches0 = pm.kernel_launches()
    total_ms = 0.0
    tris = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tris += step()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
    barrier()
    launches = pm.kernel_launches() - launches0
    kms, klaunch, kwork = pm.profile_read()
    pm.profile_enable(None)
    t_local = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    n_local = torch.tensor([float(tris)], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(n_local, op=dist.ReduceOp.SUM)
    t_max = float(t_local.item())
    value = float(n_local.item()) / (t_max / 1e3)

    # end to end through the public C interface with host buffers
    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "elements/s",
                              "ms_per_step": t_max / args.steps, "gpu_launches": launches}))
        return
    pin_xy = torch.from_numpy(w.xy.copy()).pin_memory()
    pin_tri = torch.from_numpy(w.tri.astype(np.int32)).pin_memory()
    pin_m = torch.from_numpy(w.m.copy()).pin_memory()
    h_xy, h_tri, h_m = pin_xy.numpy(), pin_tri.numpy(), pin_m.numpy()
    # page-locked output arrays, allocated once (the capacity bounds the output)
    out_h = (torch.empty((cap_out, 2), dtype=torch.float64).pin_memory().numpy(),
             torch.empty((cap_out, 3), dtype=torch.int32).pin_memory().numpy(),
             torch.empty((cap_out, 3), dtype=torch.float64).pin_memory().numpy())
    e2e_s = 0.0
    d2h = 0
    e2e_tris = 0
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        g = pm.Mesh.from_host(h_xy, h_tri, cap_factor=2, device=local)
        g.set_metric(h_m)
        g.adapt(params)
        oxyh, otrih, omh = g.get_mesh(out=out_h)
        g.close()
        dt = time.perf_counter() - t
        if i >= args.warmup:
            e2e_s += dt
            e2e_tris += otrih.shape[0]
            d2h = oxyh.nbytes + otrih.nbytes + omh.nbytes
    h2d = h_xy.nbytes + h_tri.nbytes + h_m.nbytes

    peaks, how = measured_peaks()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "elements/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name, "output_triangles_per_step": tris // max(args.steps, 1),
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_tris / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "pm_mesh_create + pm_set_metric + pm_adapt + pm_get_mesh, inputs and "
                       "outputs in pinned host buffers, wall clock per step"},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / max(args.steps, 1),
        "roofline": dict(roofline(kname, kms, klaunch, kwork, total_ms, peaks, how, fp64_meas,
                                  args.workload),
                         chosen_from={k: round(v, 4) for k, v in cand_ms.items()},
                         chosen_by="largest event time in one untimed step (ms)"),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = cpu_baseline_run(1)
        tri_c, secs = res[0]
        line["cpu_baseline"] = {"value": tri_c / secs, "unit": "elements/s", "cores": 1,
                                "kind": "oracle", "sample": sample_desc(),
                                "seconds": secs}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
