"""Autotuner of the library's launch shapes (pm_tuning, include/pm.h).

Per operator the library has knobs that decide which thread takes which
worklist item and in which launch, never a result: threads per block and
blocks per SM of the one-kernel-per-phase round kernels (the worklist chunk
each thread walks), the list size below which rounds run inside one
persistent launch, that launch's blocks per SM, and (flips, smoothing) the
list size up to which its rounds evaluate in one phase.  This is the GPU side of the paper's load balancing
(Sec. 3.5): instead of work-stealing between threads, the tuner measures
which shapes keep the SMs busiest on a workload.

The sweep is a coordinate descent over the knobs, operator by operator
(each knob's candidate values timed with CUDA events, best of `reps`
adaptations, kept when at least 1% faster).  The winner must reproduce the
default shapes' meshes bit for bit before it is written to the cache, a
JSON file keyed by "<GPU name>|<library build id>": an entry applies only
to the GPU model and the build it was measured with.  The library loads the
cache by itself (PM_TUNING_CACHE, else tuning.json beside libpm.so).

    python -m paper_1505_04694_gb300.autotune [--out PATH] [--fraction 4]
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import time

CANDIDATES = {
    "block": [64, 128, 256],
    "blocks_per_sm": [4, 8, 16, 32],
    "rounds_limit": [0, 16384, 65536, 131072, 524288],
    "rounds_blocks_per_sm": [1, 2],
    "fuse_limit": [0, 1024, 4096, 1 << 30],
}
OPERATORS = ("collapse", "flip", "split", "smoothing")


def default_cache_path() -> str:
    from . import pm

    return os.path.join(os.path.dirname(pm.LIB_PATH), "tuning.json")


def cache_key(gpu_name: str, build_id: str) -> str:
    return f"{gpu_name}|{build_id}"


def read_cache(path: str) -> dict:
    """The cache's entries ({} when the file is missing or unreadable)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict) or data.get("format") != 1:
        return {}
    entries = data.get("entries", {})
    return entries if isinstance(entries, dict) else {}


def write_entry(path: str, key: str, entry: dict) -> None:
    """Add or replace one entry, keeping the others (atomic replace)."""
    entries = read_cache(path)
    entries[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump({"format": 1, "entries": entries}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def knobs():
    """(field, index) of every knob in sweep order: operator by operator."""
    out = []
    for op in range(4):
        out.append(("block", op))
        out.append(("blocks_per_sm", op))
        if op != 2:  # refinement has no persistent rounds
            r = {0: 0, 1: 1, 3: 2}[op]
            out.append(("rounds_limit", r))
            out.append(("rounds_blocks_per_sm", r))
            if op in (1, 3):  # flips and smoothing have a one-phase evaluation
                out.append(("fuse_limit", 0 if op == 1 else 1))
    return out


def with_knob(t: dict, field: str, idx: int, value: int) -> dict:
    n = {k: list(v) for k, v in t.items()}
    n[field][idx] = value
    return n


class BatchWorkload:
    """A size-stratified part of the 512-mesh batch recipe (every `fraction`-th
    mesh by initial size), resident on the device."""

    def __init__(self, fraction: int = 4, device: int = 0):
        import numpy as np
        import torch

        from . import inputs, pm

        self.torch, self.np, self.pm = torch, np, pm
        allw = inputs.batch_workloads()
        order = sorted(range(len(allw)), key=lambda i: allw[i].tri.shape[0])
        ws = [allw[i] for i in order[::fraction]]
        self.name = (f"{len(ws)} of the {len(allw)} batch-recipe meshes (every {fraction}-th "
                     f"by initial size), {sum(w.tri.shape[0] for w in ws)} triangles")
        self.dev = torch.device("cuda", device)
        self.nv = np.array([w.xy.shape[0] for w in ws], np.int32)
        self.ne = np.array([w.tri.shape[0] for w in ws], np.int32)
        self.xy = torch.tensor(np.concatenate([w.xy for w in ws]), device=self.dev)
        self.tri = torch.tensor(np.concatenate([w.tri for w in ws]), dtype=torch.int32,
                                device=self.dev)
        self.m = torch.tensor(np.concatenate([w.m for w in ws]), device=self.dev)
        self.params = [pm.Params(seed=w.params.seed) for w in ws]

    def run(self):
        """One adaptation: (device ms of pm_batch_adapt, fingerprint of the meshes)."""
        torch, pm = self.torch, self.pm
        stream = torch.cuda.current_stream(self.dev)
        b = pm.Batch.from_device(self.xy, self.nv, self.tri, self.ne, stream=stream.cuda_stream)
        b.set_metric_dev(self.m)
        torch.cuda.synchronize(self.dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = b.adapt(self.params)
        e1.record(stream)
        e1.synchronize()
        meshes = b.get_meshes()
        b.close()
        h = hashlib.sha256()
        for xy, tri, m in meshes:
            h.update(xy.tobytes())
            h.update(tri.tobytes())
            h.update(m.tobytes())
        keys = ("rounds", "collapses", "splits", "flips", "moves", "converged")
        h.update(json.dumps([[x[k] for k in keys] for x in st]).encode())
        return e0.elapsed_time(e1), h.hexdigest()


def measure(work, tuning: dict, reps: int):
    from . import pm

    pm.set_tuning(tuning)
    best, fp = float("inf"), None
    for _ in range(reps):
        ms, f = work.run()
        best = min(best, ms)
        if fp is None:
            fp = f
        elif f != fp:
            raise RuntimeError("two adaptations with the same shapes differ")
    return best, fp


def tune(work=None, reps: int = 2, out: str | None = None, log=print) -> dict:
    """Sweep, verify and write the cache entry; returns the entry."""
    import torch

    from . import pm

    work = work or BatchWorkload()
    work.run()  # warm-up: pools, module loading
    pm.set_tuning(None)
    base = pm.get_tuning()
    t_base, fp_base = measure(work, base, reps)
    best, t_best, tried = base, t_base, 1
    log(f"default {t_base:.2f} ms")
    for field, idx in knobs():
        for value in CANDIDATES[field]:
            if value == best[field][idx]:
                continue
            cfg = with_knob(best, field, idx, value)
            t, fp = measure(work, cfg, reps)
            tried += 1
            if fp != fp_base:
                raise RuntimeError(f"shapes {cfg} changed the result")
            if t < 0.99 * t_best:
                best, t_best = cfg, t
                log(f"{field}[{idx}] = {value}: {t:.2f} ms (kept)")
    t_final, fp = measure(work, best, reps)
    if fp != fp_base:
        raise RuntimeError("the tuned shapes changed the result")
    pm.set_tuning(None)
    gpu = torch.cuda.get_device_name(work.dev)
    entry = dict(best, ms=t_final, default_ms=t_base, workload=work.name, configurations=tried,
                 reps=reps, operators=list(OPERATORS),
                 when=datetime.datetime.now(datetime.timezone.utc).isoformat(timespec="seconds"))
    out = out or default_cache_path()
    write_entry(out, cache_key(gpu, pm.build_id()), entry)
    log(f"tuned {t_final:.2f} ms (default {t_base:.2f} ms) -> {out}")
    return entry


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=None, help="cache file (default: tuning.json beside libpm.so)")
    ap.add_argument("--fraction", type=int, default=4, help="every n-th batch mesh by size")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    t0 = time.time()
    tune(BatchWorkload(a.fraction), reps=a.reps, out=a.out)
    print(f"swept in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
