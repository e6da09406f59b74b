"""GPU parity of the CUDA-core kernel that ffgpu_fgemm uses for small
products (exact 96-bit integer dot products, one reduction per output).

Against the oracle: ragged shapes across the 64 x 64 output tiles and the
32-long k chunks (k split into 2 to 16 parts, and unsplit over several
chunks), raw 32-bit words (products up to 2^64, sums up to 2^64 k),
padded leading dimensions, alpha and beta, the all-(p-1) closed form with a
long inner dimension.  The dispatch itself: below the threshold the kernel
runs and no tensor-core product does, at threshold 0 the reverse."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 251, 65521, 8388593, 2147483647]


def run(A, B, C, p, alpha, beta, pad=0):
    dA, dB, dC = to_dev(A, pad), to_dev(B, pad), to_dev(C, pad)
    ff.fgemm(dA, dB, p, alpha, beta, dC)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    return from_dev(dC)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 64), (65, 63, 33), (130, 200, 97), (7, 300, 1000),
                                   (300, 5, 31), (33, 65, 2049), (600, 1100, 77)])
def test_against_oracle(p, m, n, k):
    rng = W.rng_for("square", p % 99991, m, n, k)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    assert np.array_equal(run(A, B, C, p, alpha, beta), oracle.fgemm(A, B, p, alpha, beta, C))
    assert np.array_equal(run(A, B, C, p, alpha, beta, pad=5), oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_largest_words_long_k(p):
    # every word 2^32 - 1: each product is just below 2^64, the sum of k of
    # them needs the third accumulator word
    m, n, k = 8, 9, 100000
    A = np.full((m, k), 0xFFFFFFFF, np.uint32)
    B = np.full((k, n), 0xFFFFFFFF, np.uint32)
    C = np.zeros((m, n), np.uint32)
    want = (k * pow(0xFFFFFFFF % p, 2, p)) % p
    got = run(A, B, C, p, 1, 0)
    assert (got == want).all()
    Am = np.full((m, k), p - 1, np.uint32)
    Bm = np.full((k, n), p - 1, np.uint32)
    Cm = np.full((m, n), p - 1, np.uint32)
    got = run(Am, Bm, Cm, p, 3, 5)  # (p-1)^2 = 1: result 3k + 5(p-1) mod p
    assert (got == (3 * k + 5 * (p - 1)) % p).all()


def kernels_of(call):
    ff.profile_enable(True)
    call()
    torch.cuda.synchronize()
    prof = ff.profile_read()
    ff.profile_enable(False)
    return set(prof)


def test_dispatch_by_threshold():
    p = 65521
    rng = W.rng_for("square", 5)
    A, B = to_dev(W.uniform_residues(rng, (96, 80), p)), to_dev(W.uniform_residues(rng, (80, 70), p))
    C = torch.zeros((96, 70), dtype=torch.int32, device="cuda")
    names = kernels_of(lambda: ff.fgemm(A, B, p, 1, 0, C))
    assert "small_gemm" in names and not any(n.startswith("rns_gemm") for n in names)
    small = from_dev(C).copy()
    old = ff.get_small_threshold()
    try:
        ff.set_small_threshold(0)
        names = kernels_of(lambda: ff.fgemm(A, B, p, 1, 0, C))
        assert "small_gemm" not in names and any(n.startswith("rns_gemm") for n in names)
    finally:
        ff.set_small_threshold(old)
    assert np.array_equal(from_dev(C), small)
    with pytest.raises(ff.FFGPUError):
        ff.set_small_threshold(-1)
