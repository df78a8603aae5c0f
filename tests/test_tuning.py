"""Launch-shape tuning: the cache format and its loading by the library (no
GPU here), and (GPU) that no shape changes a result."""
import json
import os

import numpy as np
import pytest

from paper_1505_04694_gb300 import autotune


@pytest.fixture(scope="module")
def pm():
    from paper_1505_04694_gb300 import build

    build.build()
    from paper_1505_04694_gb300 import pm as binding

    yield binding
    binding.set_tuning(None)


def test_cache_entries_merge_and_survive_rewrites(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert autotune.read_cache(path) == {}
    autotune.write_entry(path, "A|1", {"block": [64] * 4})
    autotune.write_entry(path, "B|2", {"block": [256] * 4})
    autotune.write_entry(path, "A|1", {"block": [128] * 4})
    e = autotune.read_cache(path)
    assert set(e) == {"A|1", "B|2"} and e["A|1"]["block"] == [128] * 4
    with open(path) as f:
        assert json.load(f)["format"] == 1
    with open(path, "w") as f:
        f.write("not json")
    assert autotune.read_cache(path) == {}


def test_sweep_covers_every_operator_knob():
    ks = autotune.knobs()
    assert {("block", i) for i in range(4)} <= set(ks)
    assert {("blocks_per_sm", i) for i in range(4)} <= set(ks)
    assert {("rounds_limit", i) for i in range(3)} <= set(ks)
    assert {("rounds_blocks_per_sm", i) for i in range(3)} <= set(ks)
    assert {("fuse_limit", i) for i in range(2)} <= set(ks)
    t = {"block": [128] * 4, "blocks_per_sm": [16] * 4, "rounds_limit": [131072] * 3}
    n = autotune.with_knob(t, "block", 2, 64)
    assert n["block"] == [128, 128, 64, 128] and t["block"] == [128] * 4


def _entry(block, bps, lim, rbps=(1, 1, 1), fuse=(0, 0)):
    return {"block": block, "blocks_per_sm": bps, "rounds_limit": lim,
            "rounds_blocks_per_sm": list(rbps), "fuse_limit": list(fuse), "ms": 1.0}


def test_library_loads_only_its_own_entry(pm, tmp_path):
    path = str(tmp_path / "tuning.json")
    bid = pm.build_id()
    assert len(bid) == 16
    good = _entry([64, 256, 128, 64], [8, 32, 4, 16], [0, 65536, 524288], (2, 1, 2), (4096, 0))
    autotune.write_entry(path, autotune.cache_key("Fake GPU", bid), good)
    autotune.write_entry(path, autotune.cache_key("Fake GPU", "0" * 16),
                         _entry([256] * 4, [1] * 4, [1] * 3))
    autotune.write_entry(path, autotune.cache_key("Bad GPU", bid),
                         _entry([96, 128, 128, 128], [16] * 4, [1] * 3))
    pm.set_tuning(None)
    assert pm.load_tuning(path, "Fake GPU")
    got = pm.get_tuning()
    assert got == {k: good[k] for k in ("block", "blocks_per_sm", "rounds_limit",
                                        "rounds_blocks_per_sm", "fuse_limit")}
    assert pm.tuning_source().startswith("cache ")
    # another GPU model, an invalid entry, a missing file: nothing changes
    assert not pm.load_tuning(path, "Other GPU")
    assert not pm.load_tuning(path, "Bad GPU")
    assert not pm.load_tuning(str(tmp_path / "missing.json"), "Fake GPU")
    assert pm.get_tuning() == got
    pm.set_tuning(None)
    assert pm.get_tuning()["block"] == [128] * 4 and pm.tuning_source() == "default"
    with pytest.raises(pm.PmError) as e:
        pm.set_tuning({"block": [128] * 4, "blocks_per_sm": [0] * 4, "rounds_limit": [1] * 3})
    assert e.value.status == 1
    assert pm.get_tuning()["blocks_per_sm"] == [16] * 4


@pytest.mark.gpu
def test_no_launch_shape_changes_a_result(pm):
    """The same meshes (a psi-Hessian mesh and a small batch) under the
    defaults, under small blocks with every round one kernel per phase,
    with every round persistent and one-phase evaluations, and under large
    blocks with every round persistent on two blocks per SM and no one-phase
    evaluation: bit for bit the same."""
    from paper_1505_04694_gb300 import inputs

    ws = [inputs.psi_workload(25, 8000, True, 22)]
    ws += inputs.batch_workloads(count=6, seed=11, tmin=500, tmax=6000)
    shapes = [None,
              {"block": [64] * 4, "blocks_per_sm": [2] * 4, "rounds_limit": [0] * 3,
               "fuse_limit": [1 << 30] * 2},
              {"block": [128] * 4, "blocks_per_sm": [8] * 4, "rounds_limit": [1 << 30] * 3,
               "fuse_limit": [1 << 30] * 2},
              {"block": [256] * 4, "blocks_per_sm": [32] * 4, "rounds_limit": [1 << 30] * 3,
               "rounds_blocks_per_sm": [2] * 3, "fuse_limit": [0, 0]}]
    results = []
    for t in shapes:
        pm.set_tuning(t)
        b = pm.Batch.from_host([(w.xy, w.tri) for w in ws])
        b.set_metric(np.concatenate([w.m for w in ws]))
        st = b.adapt([pm.Params(seed=w.params.seed) for w in ws])
        results.append((b.get_meshes(), [{k: s[k] for k in ("rounds", "collapses", "splits",
                                                              "flips", "moves")} for s in st]))
        b.close()
    pm.set_tuning(None)
    (m0, s0) = results[0]
    for mi, si in results[1:]:
        assert si == s0
        for a, b in zip(m0, mi):
            for x, y in zip(a, b):
                assert x.shape == y.shape and np.array_equal(
                    np.ascontiguousarray(x).view(np.uint8), np.ascontiguousarray(y).view(np.uint8))
