"""The autotuner's plan cache (host logic, no GPU): JSON load/save round trip
and lookup by (path, shape bucket, modulus); and, on the GPU: tuning a
problem, then every plan the tuner can choose applied by the shipped entry
points (ffgpu_fgemm, the batched launch per instance, the request server)
giving the oracle's result bit for bit."""
import json
import itertools

import numpy as np
import pytest

import paper_cs_0601133_gb300 as ff


def key(path, m, n, k, p):
    b = lambda x: (x + 255) // 256 * 256
    return "%d:%d:%d:%d:%d" % (path, b(m), b(n), b(k), p)


def plan(k_, kernel=1, levels=0, chunk=16, route=0, raster=16, ms=1.0):
    return {"key": k_, "kernel": kernel, "winograd_levels": levels, "chunk_steps": chunk, "route": route,
            "raster_rows": raster, "ms": ms}


def write_plans(path, plans, batched=None):
    head = {"version": 2, "plans": plans}
    if batched is not None:
        head["batched_small_macs"] = batched
    # one plan object per line, the layout ffgpu_autotune_save writes
    txt = json.dumps(head).replace("}, {", "},\n{").replace('"plans": [{', '"plans": [\n{')
    path.write_text(txt + "\n")


def test_cache_round_trip_and_lookup(tmp_path):
    ff.autotune_clear()
    plans = [plan(key(0, 1000, 1000, 1000, 2147483647), kernel=1, chunk=16, ms=1.5),
             plan(key(1, 512, 512, 512, 65521), kernel=-1, levels=2, chunk=0, route=-1, raster=0, ms=20.25),
             plan(key(0, 300, 300, 300, 65521), kernel=-1, chunk=0, route=1, raster=0, ms=0.5)]
    src = tmp_path / "in.json"
    write_plans(src, plans)
    ff.autotune_load(str(src))
    got = ff.autotune_lookup(1000, 1000, 1000, 2147483647)
    assert got == dict(kernel="pair", winograd_levels=0, chunk_steps=16, route="tensor", raster_rows=16, ms=1.5)
    # same bucket (multiples of 256) and modulus -> same plan; another modulus -> none
    assert ff.autotune_lookup(1024, 1001, 777, 2147483647) == got
    assert ff.autotune_lookup(1000, 1000, 1000, 2147483629) is None
    assert ff.autotune_lookup(512, 512, 512, 65521, path="fp64")["winograd_levels"] == 2
    assert ff.autotune_lookup(300, 300, 300, 65521)["route"] == "cuda_cores"
    assert ff.autotune_lookup(4096, 4096, 4096, 2147483647) is None
    out = tmp_path / "out.json"
    ff.autotune_save(str(out))
    saved = json.loads(out.read_text())
    assert saved["version"] == 2 and saved["batched_small_macs"] == 2**23
    assert sorted(saved["plans"], key=lambda d: d["key"]) == sorted(plans, key=lambda d: d["key"])
    ff.autotune_clear()
    assert ff.autotune_lookup(1000, 1000, 1000, 2147483647) is None


def test_load_rejects_malformed(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"plans": [ {"key": "0:1:2", "kernel": "x"} ]}\n')
    with pytest.raises(ff.FFGPUError):
        ff.autotune_load(str(bad))
    bad.write_text('{"plans": [\n' + json.dumps(plan("0:256:256:256:65521", route=3)) + "\n]}\n")
    with pytest.raises(ff.FFGPUError):
        ff.autotune_load(str(bad))


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

def _dev():
    from tests.gpu_util import from_dev, to_dev
    return from_dev, to_dev


@pytest.mark.gpu
def test_tune_then_compute_exactly():
    import torch
    import oracle
    from paper_cs_0601133_gb300 import workloads as W
    from_dev, to_dev = _dev()
    ff.autotune_clear()
    p = 2147483647
    m, k, n = 1024, 1536, 768
    t = ff.autotune(m, n, k, p)
    assert t["route"] in ("tensor", "cuda_cores", "default") and t["ms"] > 0
    assert ff.autotune_lookup(m, n, k, p) == t
    rng = W.rng_for("precision", 77)
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    dC = to_dev(C)
    ff.fgemm_auto(to_dev(A), to_dev(B), p, 3, 4, dC)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p, 3, 4, C))
    # ffgpu_fgemm itself now runs this bucket with the tuned plan
    dC = to_dev(C)
    ff.fgemm(to_dev(A), to_dev(B), p, 3, 4, dC)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p, 3, 4, C))
    # a comparison path is tuned over its Winograd levels
    t64 = ff.autotune(512, 512, 512, 65521, path="fp64")
    assert t64["winograd_levels"] in (0, 1)
    ff.autotune_clear()


PLANS = ([dict(kernel=-1, levels=0, chunk=0, route=1, raster=0)] +
         [dict(kernel=kn, levels=0, chunk=ch, route=0, raster=rs)
          for kn, ch, rs in itertools.product((0, 1), (16, 7), (4, 16, 64))] +
         [dict(kernel=-1, levels=lv, chunk=0, route=-1, raster=0) for lv in (1, 2)])


@pytest.mark.gpu
@pytest.mark.parametrize("p", [65521, 2147483647])
def test_every_plan_gives_the_oracle_result(p, tmp_path):
    """Each plan the tuner can choose (CUDA cores; one-CTA or CTA-pair tiles
    with full or shortened chunks and three tile orders; one or two Winograd
    levels), loaded into the cache and applied by ffgpu_fgemm and
    ffgpu_fgemm_ws, gives the oracle's result on a ragged problem."""
    import torch
    import oracle
    from paper_cs_0601133_gb300 import workloads as W
    from_dev, to_dev = _dev()
    m, k, n = 1100, 1030, 1300
    rng = W.rng_for("precision", 78, p)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    expect = oracle.fgemm(A, B, p, alpha, beta, C)
    dA, dB = to_dev(A), to_dev(B)
    ws = torch.empty(ff.fgemm_workspace_size(m, n, k, p), dtype=torch.uint8, device="cuda")
    try:
        for pl in PLANS:
            ff.autotune_clear()
            src = tmp_path / "plan.json"
            write_plans(src, [plan(key(0, m, n, k, p), pl["kernel"], pl["levels"], pl["chunk"], pl["route"],
                                   pl["raster"])])
            ff.autotune_load(str(src))
            assert ff.autotune_lookup(m, n, k, p) is not None
            dC = to_dev(C)
            ff.fgemm(dA, dB, p, alpha, beta, dC)
            torch.cuda.synchronize()
            assert ff.last_device_error() == 0
            assert np.array_equal(from_dev(dC), expect), pl
            if pl["levels"] == 0:
                dC = to_dev(C)
                ff.fgemm_ws(dA, dB, p, alpha, beta, dC, ws)
                torch.cuda.synchronize()
                assert np.array_equal(from_dev(dC), expect), ("ws", pl)
    finally:
        ff.autotune_clear()


@pytest.mark.gpu
def test_batched_routes_follow_the_cache(tmp_path):
    """A batch whose instances' routes come from cached plans (a CUDA-core
    route for a bucket the size rule sends to the tensor cores, a tensor-core
    route for one it sends to the CUDA cores), then the batched threshold
    tuned on the same batch: every result equals the oracle's."""
    import torch
    import oracle
    from paper_cs_0601133_gb300 import workloads as W
    from_dev, to_dev = _dev()
    p = 2147483629
    shapes = [(600, 500, 700), (100, 90, 80), (40, 300, 50), (600, 500, 700), (257, 129, 300)]
    rng = W.rng_for("multimodular", 90)
    host, probs = [], []
    for m, k, n in shapes:
        A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
        host.append((A, B, C))
        probs.append((to_dev(A), to_dev(B), to_dev(C), p, 5, 6))
    try:
        ff.autotune_clear()
        src = tmp_path / "plans.json"
        write_plans(src, [plan(key(0, 600, 700, 500, p), kernel=-1, chunk=0, route=1, raster=0),
                          plan(key(0, 100, 80, 90, p), kernel=0, chunk=16, route=0, raster=16)])
        ff.autotune_load(str(src))
        descs, nd = ff.batched_descs(probs)
        ff.fgemm_batched_descs(descs, nd)
        torch.cuda.synchronize()
        for (A, B, C), pr in zip(host, probs):
            assert np.array_equal(from_dev(pr[2]), oracle.fgemm(A, B, p, 5, 6, C))
        old = ff.autotune_batched(descs, nd)
        assert 2**20 <= old <= 2**26
        torch.cuda.synchronize()
        for (A, B, C), pr in zip(host, probs):   # the tuner wrote alpha*A*B (beta taken as 0)
            assert np.array_equal(from_dev(pr[2]), oracle.fgemm(A, B, p, 5, 0, C))
    finally:
        ff.autotune_clear()
        reset = tmp_path / "reset.json"          # the default batched threshold for later tests
        write_plans(reset, [], batched=2**23)
        ff.autotune_load(str(reset))
