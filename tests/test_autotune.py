"""The autotuner's plan cache (host logic, no GPU): JSON load/save round trip
and lookup by problem class; and, on the GPU, tuning a problem and computing
with the tuned plan (exact whatever the plan)."""
import json

import numpy as np
import pytest

import paper_cs_0601133_gb300 as ff


def key(path, m, n, k, p):
    pl = ff.fgemm_plan(m, n, k, p)
    b = lambda x: (x + 255) // 256 * 256
    return "%d:%d:%d:%d:%d:%d" % (path, b(m), b(n), b(k), pl["mode"], pl["channels"])


def test_cache_round_trip_and_lookup(tmp_path):
    ff.autotune_clear()
    plans = [
        {"key": key(0, 1000, 1000, 1000, 2147483647), "kernel": 1, "winograd_levels": 0, "chunk_steps": 16, "ms": 1.5},
        {"key": key(1, 512, 512, 512, 65521), "kernel": 0, "winograd_levels": 2, "chunk_steps": 0, "ms": 20.25},
    ]
    src = tmp_path / "in.json"
    src.write_text(json.dumps({"version": 1, "plans": plans}, indent=None).replace("}, {", "},\n{"))
    ff.autotune_load(str(src))
    got = ff.autotune_lookup(1000, 1000, 1000, 2147483647)
    assert got == dict(kernel="pair", winograd_levels=0, chunk_steps=16, ms=1.5)
    # same bucket (multiples of 256) and channel count -> same plan
    assert ff.autotune_lookup(1024, 1001, 777, 2147483647) == got
    assert ff.autotune_lookup(512, 512, 512, 65521, path="fp64")["winograd_levels"] == 2
    assert ff.autotune_lookup(4096, 4096, 4096, 2147483647) is None
    out = tmp_path / "out.json"
    ff.autotune_save(str(out))
    saved = json.loads(out.read_text())
    assert sorted(saved["plans"], key=lambda d: d["key"]) == sorted(plans, key=lambda d: d["key"])
    ff.autotune_clear()
    assert ff.autotune_lookup(1000, 1000, 1000, 2147483647) is None


def test_load_rejects_malformed(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"plans": [ {"key": "0:1:2", "kernel": "x"} ]}\n')
    with pytest.raises(ff.FFGPUError):
        ff.autotune_load(str(bad))


@pytest.mark.gpu
def test_tune_then_compute_exactly():
    import torch
    import oracle
    from paper_cs_0601133_gb300 import workloads as W
    from tests.gpu_util import from_dev, to_dev
    ff.autotune_clear()
    p = 2147483647
    m, k, n = 1024, 1536, 768
    t = ff.autotune(m, n, k, p)
    assert t["kernel"] in ("single", "pair") and t["ms"] > 0
    assert ff.autotune_lookup(m, n, k, p) == t
    rng = W.rng_for("precision", 77)
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    dC = to_dev(C)
    ff.fgemm_auto(to_dev(A), to_dev(B), p, 3, 4, dC)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p, 3, 4, C))
    # a comparison path is tuned over its Winograd levels
    t64 = ff.autotune(512, 512, 512, 65521, path="fp64")
    assert t64["winograd_levels"] in (0, 1)
