"""The request server: continuous batching against an HBM budget.

Every result of a mixed fgemm / ftrsm workload served with overlapping
requests must equal the oracle's and the result of the same request served
alone; admission must respect the budget; a request that can never fit is
rejected at submission; a singular solve is reported in its completion."""
import numpy as np
import pytest

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import serving
from paper_cs_0601133_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    return serving.HostPool(n_max=512, ring=12, seed=1)


def expected(req, pool):
    A, B = pool.operands(req)
    if req["kind"] == "fgemm":
        return oracle.fgemm(np.ascontiguousarray(A), np.ascontiguousarray(B), req["p"])
    return oracle.ftrsm(np.ascontiguousarray(A), np.ascontiguousarray(B), req["p"], 1, "L", "L", "U")


def test_mix_equals_alone_and_oracle(pool):
    reqs = W.serving_requests(40, rate_per_s=1.0, lo=64, hi=512, seed_extra=5)
    arr = serving.poisson_arrivals(40, 2000.0, seed=5)
    keep = set(range(40))
    mixed = serving.replay(reqs, arr, streams=4, budget_bytes=4 << 30, pool=pool, keep_outputs=keep)
    assert mixed["failed"] == 0
    assert mixed["peak_inflight"] >= 2          # requests really overlapped
    for i, r in enumerate(reqs):
        alone = serving.replay([r], np.zeros(1), streams=1, budget_bytes=1 << 30, pool=pool, keep_outputs={0})
        assert np.array_equal(mixed["outputs"][i], alone["outputs"][0])
        assert np.array_equal(mixed["outputs"][i], expected(r, pool))


def test_budget_limits_admission(pool):
    reqs = [dict(kind="fgemm", n=512, nrhs=512, p=2147483647, t_arrival=0.0, seed=i) for i in range(6)]
    one = 3 * 512 * 512 * 4 + ff.fgemm_workspace_size(512, 512, 512, 2147483647)
    budget = int(2.5 * one) + (1 << 20)
    res = serving.replay(reqs, np.zeros(6), streams=4, budget_bytes=budget, pool=pool, keep_outputs={0, 5})
    assert res["failed"] == 0
    assert res["peak_bytes"] <= budget
    assert res["peak_inflight"] <= 2
    exp = expected(reqs[0], pool)
    assert np.array_equal(res["outputs"][0], exp) and np.array_equal(res["outputs"][5], exp)


def test_request_beyond_budget_rejected(pool):
    with ff.Server(streams=2, budget_bytes=8 << 20) as sv:
        A, B = pool.operands(dict(kind="fgemm", n=512, nrhs=512))
        out = pool.outs[0]
        with pytest.raises(ff.FFGPUError) as e:
            sv.submit_fgemm(A, B, out[:512, :512], 65521)
        assert e.value.status == -6   # FFGPU_ERR_BUDGET


def test_singular_solve_reported_in_completion(pool):
    p = 65521
    rng = W.rng_for("serving", 77)
    T = W.triangular(rng, 100, p, "L", False)
    T[10, 10] = 0
    B = W.uniform_residues(rng, (100, 8), p)
    out = np.zeros((100, 8), np.uint32)
    with ff.Server(streams=1, budget_bytes=64 << 20) as sv:
        sv.submit_ftrsm(T, B, out, p, 1, "L", "L", "N", tag=42)
        comps = []
        while not comps:
            comps = sv.poll(wait_ms=100)
        assert comps[0][0] == 42 and comps[0][1] == -1   # FFGPU_ERR_INVALID


def test_requests_run_with_cached_plans(tmp_path):
    """With plans in the cache for the requests' shape buckets (the CUDA-core
    route for a product the size rule sends to the tensor cores, one-CTA tiles
    with bands of 4 tile rows for another), the server applies them and every
    result still equals the oracle's."""
    import json
    p = 2147483647
    rng = W.rng_for("serving", 78)
    shapes = [(600, 520, 700), (300, 280, 260)]       # (m, k, n)
    b = lambda x: (x + 255) // 256 * 256
    plans = [{"key": "0:%d:%d:%d:%d" % (b(600), b(700), b(520), p), "kernel": -1, "winograd_levels": 0,
              "chunk_steps": 0, "route": 1, "raster_rows": 0, "ms": 1.0},
             {"key": "0:%d:%d:%d:%d" % (b(300), b(260), b(280), p), "kernel": 0, "winograd_levels": 0,
              "chunk_steps": 16, "route": 0, "raster_rows": 4, "ms": 1.0}]
    src = tmp_path / "plans.json"
    src.write_text('{"version": 2, "plans": [\n' + ",\n".join(json.dumps(x) for x in plans) + "\n]}\n")
    ff.autotune_clear()
    ff.autotune_load(str(src))
    try:
        probs = []
        for m, k, n in shapes:
            A, B = W.uniform_residues(rng, (m, k), p), W.uniform_residues(rng, (k, n), p)
            probs.append((A, B, np.zeros((m, n), np.uint32)))
        with ff.Server(streams=2, budget_bytes=2 << 30) as sv:
            for i, (A, B, out) in enumerate(probs):
                sv.submit_fgemm(A, B, out, p, 3, 0, tag=i)
            done = []
            while len(done) < len(probs):
                done += sv.poll(wait_ms=100)
        assert all(c[1] == 0 for c in done)
        for A, B, out in probs:
            assert np.array_equal(out, oracle.fgemm(A, B, p, 3, 0))
    finally:
        ff.autotune_clear()
