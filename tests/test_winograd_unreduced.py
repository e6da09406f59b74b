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
@pytest.mark.parametrize("p,levels", [(8388593, 3), (8388593, 2), (8388593, 1), (1048573, 2)])
def test_limit_boundary(p, levels):
    """The appendix's A_l, B_l for balanced residues (entries -(p-1)/2 and
    (p-1)/2), every entry widened to a block so that the inner dimension is
    the largest multiple of 2^l the admission limit allows: the unreduced
    levels then reach Theorem 3.1's bound itself (the oracle's CPU model of
    the schedule confirms the largest intermediate on a narrower copy), and
    the result must still be exact.  One k past the limit is refused."""
    from oracle.winograd import optimal_matrices, winograd_fgemm_z
    kmax = ff.winograd_unreduced_kmax(p, levels)
    h = (p - 1) // 2
    d = kmax // 2**levels
    assert d >= 1
    A_l, B_l = optimal_matrices(levels, -h, h, -h, h)
    widen = lambda X, r, c: np.kron(X, np.ones((r, c), dtype=object))
    # the bound with d inner blocks, checked against the CPU model at d = 1, 2
    for dd in (1, 2):
        _, zmax = winograd_fgemm_z(widen(A_l, 1, dd), widen(B_l, dd, 1), None, 1, 0, levels)
        assert zmax == bounds.winograd_bound(levels, 2**levels * dd, -h, h, -h, h)
    thm = bounds.winograd_bound(levels, 2**levels * d, -h, h, -h, h)
    assert thm < 2**62 <= bounds.winograd_bound(levels, 2**levels * (d + 1), -h, h, -h, h)
    r, s = 9, 11
    A_w = np.kron(A_l.astype(np.int64), np.ones((r, d), np.int64))    # m = 2^l r, k = 2^l d
    B_w = np.kron(B_l.astype(np.int64), np.ones((d, s), np.int64))    # n = 2^l s
    A, B = (A_w % p).astype(np.uint32), (B_w % p).astype(np.uint32)
    m, k, n = A.shape[0], A.shape[1], B.shape[1]
    assert k == 2**levels * d <= kmax
    rng = W.rng_for("precision", 17, p, levels)
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


@pytest.mark.gpu
@pytest.mark.parametrize("p,levels", [(65521, 1), (65521, 2), (8388593, 2), (251, 3)])
def test_tensor_core_leaves(p, levels):
    """Leaves of at least 2^24 multiply-adds run on the tensor cores as exact
    integer products (int64 results added into the level's sums, negated
    first where the schedule subtracts); odd dimensions peel at every level."""
    m, n, k = 1031, 1029, 2051
    assert k <= ff.winograd_unreduced_kmax(p, levels)
    rng = W.rng_for("precision", 90, p, levels)
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    assert np.array_equal(run(A, B, C, p, alpha, beta, levels), oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.gpu
def test_tensor_core_leaves_at_the_limit():
    """The widened A_l, B_l of the appendix at the admission limit with
    leaves large enough for the tensor cores (p = 65521, one level)."""
    from oracle.winograd import optimal_matrices
    p, levels = 65521, 1
    h = (p - 1) // 2
    A_l, B_l = optimal_matrices(levels, -h, h, -h, h)
    r, d, s = 300, 2048, 260                 # m = 600, k = 4096, n = 520
    A = (np.kron(A_l.astype(np.int64), np.ones((r, d), np.int64)) % p).astype(np.uint32)
    B = (np.kron(B_l.astype(np.int64), np.ones((d, s), np.int64)) % p).astype(np.uint32)
    rng = W.rng_for("precision", 91)
    C = W.uniform_residues(rng, (A.shape[0], B.shape[1]), p)
    assert np.array_equal(run(A, B, C, p, 1, 1, levels), oracle.fgemm(A, B, p, 1, 1, C))
