"""GPU parity of ffgpu_fgemm_multimod (one exact integer product, reduced mod
many primes) against the CPU oracle: for each prime p, the oracle's fgemm of
the inputs reduced mod p.  Shapes ragged in every dimension, several tiles,
entries at the stated bound (both signs), the integer-magnitude limit and the
int64 bound on k, and the degenerate k = 0."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(Ai, Bi, primes, bits):
    dA = torch.from_numpy(Ai.astype(np.int32)).cuda()
    dB = torch.from_numpy(Bi.astype(np.int32)).cuda()
    Cs = ff.fgemm_multimod(dA, dB, primes, bits)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    return [C.cpu().numpy().view(np.uint32) for C in Cs]


def expect(Ai, Bi, p):
    return oracle.fgemm(W.reduce_signed(Ai, p), W.reduce_signed(Bi, p), p, 1, 0,
                        np.zeros((Ai.shape[0], Bi.shape[1]), np.uint32))


@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 300, 129), (300, 520, 1100), (130, 70, 257), (513, 1, 64)])
def test_config4_entries_against_oracle(shape):
    m, k, n = shape
    rng = W.rng_for("multimodular", 200, m, k, n)
    Ai = rng.integers(-(2**20), 2**20 + 1, size=(m, k), dtype=np.int64)
    Bi = rng.integers(-(2**20), 2**20 + 1, size=(k, n), dtype=np.int64)
    primes = W.primes_below(2**31, 32)[::5] + [2, 3, 251, 65521]
    outs = run(Ai, Bi, primes, 20)
    for p, got in zip(primes, outs):
        assert np.array_equal(got, expect(Ai, Bi, p)), p


def test_extreme_entries_and_exact_integer():
    """All entries at +-2^20 (the largest product magnitude), checked against
    numpy's exact int64 product as well."""
    m, k, n = 200, 1024, 300
    rng = W.rng_for("multimodular", 201)
    Ai = np.where(rng.integers(0, 2, size=(m, k)) == 1, 2**20, -(2**20)).astype(np.int64)
    Bi = np.where(rng.integers(0, 2, size=(k, n)) == 1, 2**20, -(2**20)).astype(np.int64)
    Ai[0, :] = 2**20
    Bi[:, 0] = 2**20  # entry (0, 0) = k 2^40, the bound
    X = Ai @ Bi  # exact in int64 (|X| <= 2^50)
    primes = [2147483647, 2147483629, 65521, 7]
    outs = run(Ai, Bi, primes, 20)
    for p, got in zip(primes, outs):
        assert np.array_equal(got, np.mod(X, p).astype(np.uint32)), p


@pytest.mark.parametrize("bits,k", [(8, 3000), (25, 2048), (30, 3)])
def test_other_bounds(bits, k):
    m, n = 150, 270
    rng = W.rng_for("multimodular", 202, bits)
    Ai = rng.integers(-(2**bits), 2**bits + 1, size=(m, k), dtype=np.int64)
    Bi = rng.integers(-(2**bits), 2**bits + 1, size=(k, n), dtype=np.int64)
    primes = [2147483647, 1000003]
    outs = run(Ai, Bi, primes, bits)
    for p, got in zip(primes, outs):
        assert np.array_equal(got, expect(Ai, Bi, p)), p


def test_rejects_int64_overflow_and_k_zero():
    A = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    B = torch.zeros((8, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(ff.FFGPUError):
        ff.fgemm_multimod(A, B, [65521], 31)
    A0 = torch.zeros((4, 0), dtype=torch.int32, device="cuda")
    B0 = torch.zeros((0, 5), dtype=torch.int32, device="cuda")
    Cs = ff.fgemm_multimod(A0, B0, [65521, 7], 20)
    torch.cuda.synchronize()
    assert all(int(C.abs().sum()) == 0 for C in Cs)


def test_batched_multimodular_instances():
    """The batched form on uneven instances of the multi-modular workload
    (plus a k = 0 instance), 8 primes each: every output against the oracle
    (all of the first instances, sampled entries of the rest)."""
    shapes, primes = W.multimodular_instances(count=40, nprimes=32)
    use = primes[::4]
    probs, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        m, n, k = int(m), int(n), int(k)
        if i == 5:
            k = 0
        Ai, Bi = W.multimodular_integers(i, m, n, k)
        dA = torch.from_numpy(Ai.astype(np.int32)).cuda()
        dB = torch.from_numpy(Bi.astype(np.int32)).cuda()
        Cs = [torch.full((m, n), -1, dtype=torch.int32, device="cuda") for _ in use]
        probs.append((dA, dB, Cs))
        host.append((Ai, Bi))
    ff.fgemm_multimod_batched(probs, use, 20)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    rng = np.random.default_rng(3)
    for i, ((Ai, Bi), (_, _, Cs)) in enumerate(zip(host, probs)):
        for p, C in zip(use, Cs):
            got = C.cpu().numpy().view(np.uint32)
            if i < 8:
                assert np.array_equal(got, expect(Ai, Bi, p)), (i, p)
            else:
                r = rng.integers(0, Ai.shape[0], 12)
                c = rng.integers(0, Bi.shape[1], 12)
                X = (Ai[r, :] * Bi[:, c].T).sum(axis=1)  # exact in int64
                assert np.array_equal(got[r, c], np.mod(X, p).astype(np.uint32)), (i, p)
