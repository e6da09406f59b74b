"""Winograd's levels over Z with one reduction at the end (section 3.2,
Theorem 3.1, Corollaries 3.3-3.4).

CPU: the library's admission limit (the largest k that l unreduced levels
admit for p) equals the oracle's own reading of Theorem 3.1 with a 62-bit
exact range and balanced residues, wherever the operands fit int32
(4^l (p-1)/2 < 2^31), and is 0 where they do not.
GPU: results equal the oracle's, odd shapes (dynamic peeling), alpha and
beta, 1-3 levels; a k just above the limit is refused, the limit itself runs."""
import numpy as np
import pytest

import oracle
from oracle import bounds
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W


@pytest.mark.parametrize("p", [2, 3, 251, 65521, 1048573, 8388593, 2147483647])
@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
def test_admission_limit_matches_theorem_3_1(p, levels):
    got = ff.winograd_unreduced_kmax(p, levels)
    half = 1 if p == 2 else (p - 1) // 2   # balanced residues of Z/2Z are 0 and -1
    if 4 ** levels * half >= 2 ** 31:
        assert got == 0
    elif p == 2:
        # Theorem 3.1 with entries in [-1, 1]: the largest k with the bound below 2^62
        lo, hi = 1, 2 ** 63
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if bounds.winograd_bound(levels, mid, -1, 1, -1, 1) < 2 ** 62:
                lo = mid
            else:
                hi = mid - 1
        assert got == min(lo, 2 ** 63 - 1)
    else:
        assert got == bounds.k_max_winograd(p, 62, levels, balanced=True)


def test_admission_limit_rejects_bad_arguments():
    for p, levels in [(1, 1), (2 ** 31, 1), (65521, 0), (65521, 9)]:
        with pytest.raises(ff.FFGPUError):
            ff.winograd_unreduced_kmax(p, levels)


def run(A, B, C, p, alpha, beta, levels):
    import torch
    from tests.gpu_util import from_dev, to_dev
    dC = to_dev(C)
    ff.fgemm_ex(to_dev(A), to_dev(B), p, alpha, beta, dC, winograd_levels=levels, unreduced=True)
    torch.cuda.synchronize()
    return from_dev(dC)


@pytest.mark.gpu
@pytest.mark.parametrize("p", [2, 3, 251, 65521, 8388593])
@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (131, 97, 259), (2, 2, 2), (7, 300, 45)])
def test_against_oracle(p, levels, m, n, k):
    if k > ff.winograd_unreduced_kmax(p, levels):
        pytest.skip("outside the admitted range")
    rng = W.rng_for("precision", p % 99991, levels, m, n, k)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    assert np.array_equal(run(A, B, C, p, alpha, beta, levels), oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.gpu
def test_limit_boundary():
    p, levels = 8388593, 3
    kmax = ff.winograd_unreduced_kmax(p, levels)
    rng = W.rng_for("precision", 17)
    # all entries at the balanced extreme (p-1)/2: the worst magnitudes
    m, n = 9, 11
    A = np.full((m, kmax), (p - 1) // 2, np.uint32)
    B = np.full((kmax, n), (p - 1) // 2, np.uint32)
    C = W.uniform_residues(rng, (m, n), p)
    assert np.array_equal(run(A, B, C, p, 1, 1, levels), oracle.fgemm(A, B, p, 1, 1, C))
    A2 = np.zeros((m, kmax + 1), np.uint32)
    B2 = np.zeros((kmax + 1, n), np.uint32)
    with pytest.raises(ff.FFGPUError) as e:
        run(A2, B2, C, p, 1, 0, levels)
    assert e.value.status == -2


@pytest.mark.gpu
def test_large_prime_refused():
    A = np.ones((4, 4), np.uint32)
    with pytest.raises(ff.FFGPUError):
        run(A, A, A, 2147483647, 1, 0, 1)
