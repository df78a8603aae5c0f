"""Host logic of bench.py, no GPU: the roofline arithmetic, the traffic table
lookup, and the oracle arm's JSON line (run for one short step)."""
import importlib.util
import json
import math
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_arithmetic():
    b = load_bench()
    # 5e10 FP64 operations in 100 ms at a 2070 MHz maximum clock
    r = b.roofline("k_swap_edge", 100.0, 10, 5e10, 500.0, {"sm_max_mhz": 2070.0}, "measured",
                   fp64_meas=529.0, workload="batch512")
    peak = 304 * 2070e6 / 1e9
    assert r["bound"] == "alu"
    assert math.isclose(r["peak"], peak)
    assert math.isclose(r["achieved"], 500.0)
    assert math.isclose(r["frac"], 500.0 / peak)
    assert math.isclose(r["frac_of_measured"], 500.0 / 529.0)
    assert math.isclose(r["kernel_ms_per_step_share"], 0.2)
    assert r["launches"] == 10
    # no counted work: no achieved figure, no fraction
    r0 = b.roofline("k_other", 10.0, 1, 0, 50.0, {}, "fallback")
    assert r0["achieved"] is None and r0["frac"] is None and r0["traffic"] is None


def test_traffic_table_lookup():
    b = load_bench()
    entries = {}
    with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) >= 3:
                entries[(parts[0], parts[1])] = float(parts[2])
    assert entries, "the committed traffic table has entries"
    for (k, w), v in entries.items():
        assert b.traffic_of(k, w) == v
    assert b.traffic_of("k_no_such_kernel", "batch512") is None


def test_oracle_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    b = load_bench()
    assert d["impl"] == "reference"
    assert d["metric"] == b.METRIC
    assert d["unit"] == "elements/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["config"]["workload"] == b.BATCH_WORKLOAD and d["config"]["meshes"] == 512
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "elements/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_oracle_arm_under_two_ranks_prints_once(tmp_path):
    """Launched with two ranks, rank 0 alone runs the oracle arm and prints
    its line; the other rank exits 0 without work."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, TMPDIR=str(tmp_path)))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
