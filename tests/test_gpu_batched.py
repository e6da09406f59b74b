"""GPU parity of ffgpu_fgemm_batched (small products in one grouped CUDA-core
launch; the others in one grouped conversion per operand and one persistent
grouped tensor-core launch per wave) against the CPU oracle, and against
ffgpu_fgemm on the same descriptors.

Workloads follow the multi-modular configuration: uneven shapes drawn
log-uniform in [16, 1024], integer matrices with entries in [-2^20, 2^20]
reduced modulo several of the 32 primes just below 2^31, plus mixed moduli of
every size class in one batch."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=["mixed", "tensor_only"])
def routing(request):
    """Each test twice: with the default routing (products of at most 2^23
    multiply-adds in the grouped CUDA-core launch, the rest on the tensor
    cores) and with every product on the tensor-core waves."""
    old = ff.get_small_threshold()
    if request.param == "tensor_only":
        ff.set_small_threshold(0)
    yield request.param
    ff.set_small_threshold(old)


def run_batch(problems):
    dev = [(to_dev(A), to_dev(B), to_dev(C), p, al, be) for (A, B, C, p, al, be) in problems]
    ff.fgemm_batched(dev)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    return [from_dev(d[2]) for d in dev]


def test_mixed_shapes_and_moduli():
    rng = W.rng_for("multimodular", 100)
    primes = [2, 3, 251, 256, 257, 65521, 1000003, 8388593, 2147483647]
    problems = []
    for i in range(40):
        m, n, k = (int(v) for v in W.log_uniform_int(rng, 16, 600, 3))
        p = primes[i % len(primes)]
        A = W.uniform_words(rng, (m, k))
        B = W.uniform_words(rng, (k, n))
        C = W.uniform_words(rng, (m, n))
        problems.append((A, B, C, p, int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))))
    outs = run_batch(problems)
    for (A, B, C, p, al, be), got in zip(problems, outs):
        assert np.array_equal(got, oracle.fgemm(A, B, p, al, be, C)), (A.shape, B.shape, p)


def test_tile_classes_and_ragged_inner_dimensions():
    """Small products on both tile sizes of the grouped CUDA-core launch (32 x
    32 tiles for a dimension of at most 32 or where they pad less, e.g. 90 x
    90 or 129 x 65; 64 x 64 tiles for 64 x 64 or 100 x 64) with inner
    dimensions that end inside a 32-long chunk (1, 5, 31, 33, 63, 100), words
    not reduced mod p: every entry against the oracle."""
    rng = W.rng_for("multimodular", 101)
    shapes = [(33, 33), (40, 700), (90, 90), (65, 130), (96, 96), (100, 64), (31, 500), (64, 64), (129, 65)]
    ks = [1, 5, 31, 33, 63, 100]
    primes = [251, 65521, 2147483647]
    problems = []
    for i, (m, n) in enumerate(shapes):
        for j, k in enumerate(ks):
            p = primes[(i + j) % len(primes)]
            A = W.uniform_words(rng, (m, k))
            B = W.uniform_words(rng, (k, n))
            C = W.uniform_words(rng, (m, n))
            problems.append((A, B, C, p, int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))))
    outs = run_batch(problems)
    for (A, B, C, p, al, be), got in zip(problems, outs):
        assert np.array_equal(got, oracle.fgemm(A, B, p, al, be, C)), (A.shape, B.shape, p)


def test_multimodular_instances_subset():
    shapes, primes = W.multimodular_instances(count=24, nprimes=32)
    use = primes[::8]  # 4 of the 32 primes
    problems = []
    for i, (m, n, k) in enumerate(shapes):
        Ai, Bi = W.multimodular_integers(i, int(m), int(n), int(k))
        for p in use:
            A = W.reduce_signed(Ai, p)
            B = W.reduce_signed(Bi, p)
            C = np.zeros((int(m), int(n)), np.uint32)
            problems.append((A, B, C, p, 1, 0))
    outs = run_batch(problems)
    for (A, B, C, p, al, be), got in zip(problems, outs):
        assert np.array_equal(got, oracle.fgemm(A, B, p, al, be, C))


def test_batched_equals_single_calls():
    rng = W.rng_for("multimodular", 101)
    problems = []
    for i in range(12):
        m, n, k = (int(v) for v in W.log_uniform_int(rng, 16, 1024, 3))
        p = W.primes_below(2**31, 32)[i]
        problems.append((W.uniform_residues(rng, (m, k), p), W.uniform_residues(rng, (k, n), p),
                         W.uniform_residues(rng, (m, n), p), p, 3, 4))
    outs = run_batch(problems)
    for (A, B, C, p, al, be), got in zip(problems, outs):
        dC = to_dev(C)
        ff.fgemm(to_dev(A), to_dev(B), p, al, be, dC)
        torch.cuda.synchronize()
        assert np.array_equal(got, from_dev(dC))


def test_degenerate_members():
    p = 65521
    rng = W.rng_for("multimodular", 102)
    C0 = W.uniform_words(rng, (20, 30))
    A1 = W.uniform_residues(rng, (40, 50), p)
    B1 = W.uniform_residues(rng, (50, 60), p)
    C1 = W.uniform_residues(rng, (40, 60), p)
    problems = [
        (np.zeros((20, 0), np.uint32), np.zeros((0, 30), np.uint32), C0, p, 5, 7),   # k = 0: beta*C
        (A1, B1, C1, p, 2, 3),
    ]
    outs = run_batch(problems)
    assert np.array_equal(outs[0], (7 * C0.astype(np.uint64) % p).astype(np.uint32))
    assert np.array_equal(outs[1], oracle.fgemm(A1, B1, p, 2, 3, C1))
    assert ff.fgemm_batched([]) == []


def test_many_instances_several_waves_sampled():
    """2048 fgemms (256 integer instances x 8 primes): more channel planes than
    one wave holds.  32 products checked entirely, every other one on 16
    sampled entries."""
    shapes, primes = W.multimodular_instances(count=256, nprimes=32)
    use = primes[::4]
    problems = []
    for i, (m, n, k) in enumerate(shapes):
        Ai, Bi = W.multimodular_integers(i, int(m), int(n), int(k))
        for p in use:
            problems.append((W.reduce_signed(Ai, p), W.reduce_signed(Bi, p),
                             np.zeros((int(m), int(n)), np.uint32), p, 1, 0))
    outs = run_batch(problems)
    rng = np.random.default_rng(0)
    for idx, ((A, B, C, p, al, be), got) in enumerate(zip(problems, outs)):
        if idx % 64 == 0:
            assert np.array_equal(got, oracle.fgemm(A, B, p, al, be, C))
        else:
            r = rng.integers(0, A.shape[0], 16)
            c = rng.integers(0, B.shape[1], 16)
            assert np.array_equal(got[r, c], oracle.fgemm_entries(A, B, p, al, be, C, r, c))


def test_batched_plan_graph_runs_track_inputs():
    """A captured plan (CUDA graph) gives the oracle's result, and a second run
    after the inputs change in place gives the new result: the graph reads the
    buffers, not a snapshot.  The batch mixes moduli of every size class and a
    k = 0 member (run outside the grouped launch)."""
    rng = W.rng_for("multimodular", 103)
    primes = [3, 251, 65521, 8388593, 2147483647]
    host, dev = [], []
    for i in range(25):
        m, n, k = (int(v) for v in W.log_uniform_int(rng, 16, 500, 3))
        if i == 7:
            k = 0
        p = primes[i % len(primes)]
        A = W.uniform_words(rng, (m, k))
        B = W.uniform_words(rng, (k, n))
        C = W.uniform_words(rng, (m, n))
        al, be = int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))
        host.append((A, B, C, p, al, be))
        dev.append((to_dev(A), to_dev(B), to_dev(C), p, al, be))
    with ff.BatchedPlan(dev) as plan:
        info = plan.info()
        assert info["waves"] >= 1 and info["singles"] == 1 and info["graph_nodes"] >= 3
        plan.run()
        assert plan.error() == 0
        for (A, B, C, p, al, be), d in zip(host, dev):
            assert np.array_equal(from_dev(d[2]), oracle.fgemm(A, B, p, al, be, C)), (A.shape, B.shape, p)
        # new contents, same buffers: C holds the first result, A and B are redrawn
        expect = []
        for i, ((A, B, C, p, al, be), d) in enumerate(zip(host, dev)):
            A2 = W.uniform_words(rng, A.shape)
            B2 = W.uniform_words(rng, B.shape)
            d[0].copy_(to_dev(A2))
            d[1].copy_(to_dev(B2))
            C1 = from_dev(d[2])
            expect.append(oracle.fgemm(A2, B2, p, al, be, C1))
        plan.run()
        assert plan.error() == 0
        for e, d in zip(expect, dev):
            assert np.array_equal(from_dev(d[2]), e)


def test_batched_plan_equals_immediate_on_multimodular_batch():
    shapes, primes = W.multimodular_instances(count=64, nprimes=32)
    use = primes[::8]
    dev_a, dev_b = [], []
    for i, (m, n, k) in enumerate(shapes):
        Ai, Bi = W.multimodular_integers(i, int(m), int(n), int(k))
        for p in use:
            A = to_dev(W.reduce_signed(Ai, p))
            B = to_dev(W.reduce_signed(Bi, p))
            dev_a.append((A, B, torch.zeros((int(m), int(n)), dtype=torch.int32, device="cuda"), p, 1, 0))
            dev_b.append((A, B, torch.zeros((int(m), int(n)), dtype=torch.int32, device="cuda"), p, 1, 0))
    ff.fgemm_batched(dev_a)
    plan = ff.BatchedPlan(dev_b)
    plan.run()
    plan.run()  # idempotent with beta = 0
    assert plan.error() == 0
    plan.close()
    torch.cuda.synchronize()
    for x, y in zip(dev_a, dev_b):
        assert torch.equal(x[2], y[2])


def test_config4_full_batch_sampled():
    """The batched configuration at its full size, in the launch the bench
    times: 4096 integer instances (m, n, k log-uniform in [16, 1024], entries
    in [-2^20, 2^20]) reduced modulo each of the 32 primes below 2^31 on the
    device, 131072 fgemms in one ffgpu_fgemm_batched call.  256 products drawn
    at random are checked on 8 sampled entries each (a corner among them), and
    every product's first entry."""
    shapes, primes = W.multimodular_instances(count=4096, nprimes=32)
    problems, ints = [], []
    for i, (m, n, k) in enumerate(shapes):
        Ai, Bi = W.multimodular_integers(i, int(m), int(n), int(k))
        ints.append((Ai, Bi))
        dAi, dBi = torch.from_numpy(Ai).cuda(), torch.from_numpy(Bi).cuda()
        for p in primes:
            problems.append((torch.remainder(dAi, p).to(torch.int32), torch.remainder(dBi, p).to(torch.int32),
                             torch.zeros((int(m), int(n)), dtype=torch.int32, device="cuda"), int(p), 1, 0))
    descs, nd = ff.batched_descs(problems)
    ff.fgemm_batched_descs(descs, nd)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    rng = np.random.default_rng(4096)
    picks = set(rng.integers(0, len(problems), 256).tolist())
    firsts = torch.stack([pr[2][0, 0] for pr in problems]).cpu().numpy().view(np.uint32)
    for idx, (dA, dB, dC, p, al, be) in enumerate(problems):
        Ai, Bi = ints[idx // len(primes)]
        if idx not in picks and idx % 97 != 0:
            continue
        A, B = W.reduce_signed(Ai, p), W.reduce_signed(Bi, p)
        C = np.zeros((A.shape[0], B.shape[1]), np.uint32)
        r = np.concatenate([rng.integers(0, A.shape[0], 7), [A.shape[0] - 1]])
        c = np.concatenate([rng.integers(0, B.shape[1], 7), [B.shape[1] - 1]])
        got = from_dev(dC)
        assert np.array_equal(got[r, c], oracle.fgemm_entries(A, B, p, al, be, C, r, c)), idx
    # the first entry of every product: one dot product each, against exact integers
    for i, (Ai, Bi) in enumerate(ints):
        v = int(np.dot(Ai[0].astype(object), Bi[:, 0].astype(object)))
        for j, p in enumerate(primes):
            assert firsts[i * len(primes) + j] == v % p, (i, p)
