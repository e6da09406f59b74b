"""GPU parity of the comparison paths (FP64 DMMA, FP32 SIMT) and of Winograd's
levels (Table 2 schedule, dynamic peeling) on every path, against the oracle.

This is the precision comparison: the same exact result must come out of the
residue-number-system tensor-core path, the double-precision path and the
single-precision path, each with 0, 1 or 2 levels of Winograd's algorithm."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

@pytest.fixture(autouse=True, scope="module")
def tensor_cores_only():
    """Every product of this module on the tensor-core route, small ones
    included (ffgpu_fgemm would send those to the CUDA-core kernel)."""
    old = ff.get_small_threshold()
    ff.set_small_threshold(0)
    yield
    ff.set_small_threshold(old)


CASES = [("rns", 65521), ("rns", 2147483647), ("rns", 251), ("fp64", 251), ("fp64", 65521),
         ("fp64", 1048573), ("fp64", 8388593), ("fp32", 251), ("fp32", 2)]


def run(A, B, C, p, alpha, beta, path, levels):
    dC = to_dev(C)
    ff.fgemm_ex(to_dev(A), to_dev(B), p, alpha, beta, dC, path=path, winograd_levels=levels)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    return from_dev(dC)


@pytest.mark.parametrize("path,p", CASES)
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_paths_and_levels(path, p, levels):
    rng = W.rng_for("precision", ord(path[2]), p, levels)
    m, k, n = 301, 515, 263      # odd in every dimension: peeling at each level
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta, path, levels)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("path,p", [("fp64", 8388593), ("fp32", 251), ("rns", 2147483647)])
def test_adversarial_long_k(path, p):
    # all entries p - 1: the delayed-reduction bound is reached on every path
    m, n, k = 128, 192, 4096
    A, B, C = W.adversarial_problem(m, n, k, p)
    got = run(A, B, C, p, 1, 1, path, 1)
    assert np.all(got == (k + (p - 1)) % p)


def test_three_levels_even_sizes():
    p = 65521
    rng = W.rng_for("precision", 3)
    A = W.uniform_residues(rng, (1024, 1024), p)
    B = W.uniform_residues(rng, (1024, 1024), p)
    C = W.uniform_residues(rng, (1024, 1024), p)
    got = run(A, B, C, p, 7, 9, "rns", 3)
    assert np.array_equal(got, oracle.fgemm(A, B, p, 7, 9, C))


def test_unsupported_modulus_for_a_path():
    A = to_dev(np.zeros((4, 4), np.uint32))
    with pytest.raises(ff.FFGPUError):
        ff.fgemm_ex(A, A, 257, path="fp32")
    with pytest.raises(ff.FFGPUError):
        ff.fgemm_ex(A, A, 2**25 + 1, path="fp64")


@pytest.mark.parametrize("p", [2, 251, 65521, 2147483647])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_simt_path_with_levels(p, levels):
    rng = W.rng_for("precision", p, levels, 7)
    m, n, k = 131, 97, 259
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta, "simt", levels)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("path,p,k", [("rns", 2147483647, 65536), ("rns", 65521, 65536), ("fp64", 8388593, 8192),
                                      ("fp64", 65521, 8192), ("fp32", 251, 65536)])
def test_precision_config_full_size_sampled(path, p, k):
    """The precision comparison at its own sizes (m = n = 8192, the longest
    inner dimension each path is timed at), every Winograd depth it is timed
    with: sampled entries recomputed by the oracle and Freivalds' test on the
    whole result; alpha and beta are non-trivial here (the bench times 1, 0)."""
    n = 8192
    rng = W.rng_for("precision", 51, p, k)
    A = W.uniform_residues(rng, (n, k), p)
    B = W.uniform_residues(rng, (k, n), p)
    C = W.uniform_residues(rng, (n, n), p)
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    dA, dB = to_dev(A), to_dev(B)
    srng = np.random.default_rng(k + p)
    rows = np.concatenate([srng.integers(0, n, 512), [0, n - 1, n - 1]])
    cols = np.concatenate([srng.integers(0, n, 512), [n - 1, 0, n - 1]])
    expect = oracle.fgemm_entries(A, B, p, alpha, beta, C, rows, cols)
    for levels in (0, 1, 2):
        dC = to_dev(C)
        ff.fgemm_ex(dA, dB, p, alpha, beta, dC, path=path, winograd_levels=levels)
        torch.cuda.synchronize()
        assert ff.last_device_error() == 0
        got = from_dev(dC)
        assert np.array_equal(got[rows, cols], expect), (path, p, k, levels)
        assert oracle.freivalds(A, B, C, got, p, alpha, beta, trials=1), (path, p, k, levels)
        del dC


# Worst cases of each comparison path's delayed-reduction bound (eqs. 1-2):
# entries +-floor(p/2) (the largest centred magnitude) in the sign pattern of
# workloads.sign_pattern_problem, so every partial sum between two reductions
# is a sum of equal-signed products floor(p/2)^2 -- the largest value the
# blocking admits.  (All entries p - 1 are centred to -1 and stress nothing.)

def closed_form(s, t, k, a, p, alpha, beta, C):
    v = [(alpha * k * a * a) % p, (-alpha * k * a * a) % p]
    X = np.where(np.outer(s, t) > 0, v[0], v[1]).astype(np.uint64)
    return ((X + (beta % p) * C.astype(np.uint64)) % p).astype(np.uint32)


def test_fp32_path_at_its_block_bound():
    """FP32: p = 251, entries +-125, reduced every R products with
    R 125^2 + 2p <= 2^24 (R = 1072): each block sums 1072 * 15625 = 99.8 % of
    2^24; three blocks and a ragged one."""
    p, h = 251, 125
    R = ((1 << 24) - 2 * p) // (h * h) // 16 * 16     # the path's block: whole k-tiles of 16
    assert R == 1072 and R * h * h + p < 2**24 and R * h * h >= 0.99 * 2**24
    m, n, k = 200, 136, 3 * R + 50
    rng = W.rng_for("worstcase", 10, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, h, h)
    got = run(A, B, C, p, 3, 5, "fp32", 0)
    assert np.array_equal(got, oracle.fgemm(A, B, p, 3, 5, C))
    assert np.array_equal(got, closed_form(s, t, k, h, p, 3, 5, C))


@pytest.mark.parametrize("p", [8388593, 33554393])
def test_fp64_path_at_its_block_bound(p):
    """FP64 DMMA: entries +-floor(p/2), 16-long k-tiles between reductions.
    For p = 33554393 (the largest prime below 2^25, the path's limit) a tile
    sums 16 floor(p/2)^2 = 50 % of 2^53; the accumulator keeps at most 1.5p
    after a reduction."""
    h = p // 2
    assert 16 * h * h + 3 * p // 2 < 2**53
    if p > 2**24:
        assert 16 * h * h >= 0.49 * 2**53
    m, n, k = 200, 136, 4096 + 13
    rng = W.rng_for("worstcase", 11, p)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, h, h)
    alpha, beta = int(rng.integers(1, p)), int(rng.integers(0, p))
    got = run(A, B, C, p, alpha, beta, "fp64", 0)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))
    assert np.array_equal(got, closed_form(s, t, k, h, p, alpha, beta, C))


@pytest.mark.parametrize("path,p", [("rns", 2147483647), ("fp64", 8388593), ("fp32", 251)])
@pytest.mark.parametrize("levels", [1, 2])
def test_winograd_levels_on_worst_case_inputs(path, p, levels):
    """The same inputs through Winograd's levels: the pre-additions are
    reduced mod p, so each base product sees residues anywhere in [0, p);
    the result must still be exact."""
    h = p // 2
    m, n, k = 260, 264, 2200
    rng = W.rng_for("worstcase", 12, p, levels)
    A, B, C, s, t = W.sign_pattern_problem(rng, m, n, k, p, h, h)
    got = run(A, B, C, p, 1, 1, path, levels)
    assert np.array_equal(got, closed_form(s, t, k, h, p, 1, 1, C))


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("threshold", [0, 2**30])
def test_fused_pre_additions_on_both_routes(levels, threshold):
    """The residue path's Winograd levels pass S1..S4 and T1..T4 down as sums
    of quadrants, summed inside the conversions; sub-products small enough
    for the CUDA cores have their sums written out first.  Threshold 0: every
    sub-product on the tensor cores; 2^30: every one on the CUDA cores.  Odd
    dimensions at both levels (peeling with summed operands)."""
    p = 2147483647
    rng = W.rng_for("precision", 60, levels, threshold % 1000)
    m, k, n = 523, 611, 457
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    old = ff.get_small_threshold()
    ff.set_small_threshold(threshold)
    try:
        got = run(A, B, C, p, alpha, beta, "rns", levels)
    finally:
        ff.set_small_threshold(old)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))
