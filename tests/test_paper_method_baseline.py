"""The paper-method CPU baseline of bench.py (float64 BLAS products with the
delayed reduction of eq. (1), gamma = 53): its block length is eq. (1)'s
lambda, it is exact (equal to the oracle) wherever eq. (1) admits a block,
including inner dimensions that span several blocks, and it declines the
moduli for which no product fits a double."""
import numpy as np
import pytest

import bench
import oracle
from paper_cs_0601133_gb300 import workloads as W


@pytest.mark.parametrize("p", [2, 3, 251, 65521, 1048573, 8388593, 67108859, 94906249, 2147483647])
def test_block_length_is_eq1_lambda(p):
    lam = bench.paper_method_kblk(p)
    if p == 2:
        assert lam == 2 ** 53 - 1
        return
    assert lam * (p - 1) ** 2 < 2 ** 53 <= (lam + 1) * (p - 1) ** 2


@pytest.mark.parametrize("p,k", [(2, 70), (251, 300), (65521, 257), (8388593, 300), (8388593, 127), (67108859, 9)])
def test_equals_oracle(p, k):
    rng = W.rng_for("square", p % 9973, k)
    m, n = 37, 45
    A, B, C = W.uniform_words(rng, (m, k)), W.uniform_words(rng, (k, n)), W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    got = bench.paper_method_fgemm(A, B, C, p, alpha, beta)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


def test_block_boundary_worst_case():
    # every entry p - 1: each block sums exactly lambda products of (p-1)^2
    p = 8388593
    lam = bench.paper_method_kblk(p)
    k = 3 * lam + 5
    A, B, C = W.adversarial_problem(4, 3, k, p)
    got = bench.paper_method_fgemm(A, B, C, p, 1, 1)
    assert np.array_equal(got, oracle.fgemm(A, B, p, 1, 1, C))


def test_declines_when_no_product_fits():
    A = np.ones((2, 2), np.uint32)
    assert bench.paper_method_fgemm(A, A, A, 2147483647, 1, 0) is None
