"""Pins of the Winograd schedule oracle (Table 2 with the A22 reading of row 16)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import bounds
from oracle.winograd import optimal_matrices, winograd_fgemm_z


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 12, 20), (9, 7, 11), (5, 6, 7), (12, 13, 8)])
@pytest.mark.parametrize("levels", [1, 2])
def test_schedule_computes_the_product(shape, levels):
    m, k, n = shape
    rng = np.random.default_rng(m * 100 + k * 10 + n + levels)
    A = rng.integers(-50, 51, (m, k))
    B = rng.integers(-50, 51, (k, n))
    C = rng.integers(-50, 51, (m, n))
    alpha, beta = 3, -2
    got, _ = winograd_fgemm_z(A, B, C, alpha, beta, levels)
    expect = alpha * (A.astype(object) @ B.astype(object)) + beta * C.astype(object)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("ranges", [(0, 10, 0, 10), (-3, 5, -2, 7), (-4, 4, -4, 4), (0, 250, 0, 250)])
def test_theorem_3_1_bound_is_reached(l, ranges):
    mA, MA, mB, MB = ranges
    A, B = optimal_matrices(l, mA, MA, mB, MB)
    assert A.shape == (2**l, 2**l)
    _, zmax = winograd_fgemm_z(A, B, None, 1, 0, l)
    assert zmax == bounds.winograd_bound(l, 2**l, mA, MA, mB, MB)


@pytest.mark.parametrize("l", [1, 2, 3])
def test_theorem_3_1_bound_holds_on_random_inputs(l):
    rng = np.random.default_rng(l)
    p = 251
    for _ in range(3):
        k = 2**l * int(rng.integers(1, 4))
        A = rng.integers(0, p, (2**l * 2, k))
        B = rng.integers(0, p, (k, 2**l * 2))
        _, zmax = winograd_fgemm_z(A, B, None, 1, 0, l)
        assert zmax <= bounds.winograd_bound_positive(l, k, p)


def _kron_blocks(A_l, B_l, r: int, d: int, s: int):
    """A_l with every entry widened to an r x d block of itself, B_l to d x s:
    the recursion's splits of m, k and n then fall on block edges, so every
    operand sum is one of the d = 1 case's and every leaf product is d times
    its value there -- the same matrices for an inner dimension 2^l d."""
    one = lambda a, b: np.ones((a, b), dtype=object)
    return np.kron(A_l, one(r, d)), np.kron(B_l, one(d, s))


@pytest.mark.parametrize("p", [3, 5, 7, 11, 251])
@pytest.mark.parametrize("l", [1, 2, 3])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_corollary_3_3_balanced_bound_is_reached(p, l, d):
    """Corollary 3.3 (balanced residues, entries in [-(p-1)/2, (p-1)/2]) is
    Theorem 3.1 with mA = mB = -(p-1)/2 and MA = MB = (p-1)/2, and the
    appendix's A_l, B_l for those ranges, widened to an inner dimension
    k = 2^l d, reach it exactly: (3^l/2)^2 d (p-1)^2."""
    h = (p - 1) // 2
    k = 2**l * d
    thm = bounds.winograd_bound(l, k, -h, h, -h, h)
    assert bounds.winograd_bound_balanced(l, k, p) == thm
    A_l, B_l = optimal_matrices(l, -h, h, -h, h)
    A, B = _kron_blocks(A_l, B_l, 1, d, 1)
    assert A.shape == (2**l, k) and B.shape == (k, 2**l)
    got, zmax = winograd_fgemm_z(A, B, None, 1, 0, l)
    assert np.array_equal(got, A @ B)
    assert zmax == thm
    # a slip in the leading factor ((1 + 3^l)/2 in place of 3^l/2) is caught
    assert zmax != (Fraction(1 + 3**l, 2) ** 2 * d * (p - 1) ** 2)


@pytest.mark.parametrize("l", [1, 2])
def test_theorem_3_1_reached_with_row_and_column_blocks(l):
    """Widening rows and columns as well (m = 2^l r, n = 2^l s) leaves the
    largest intermediate unchanged."""
    A_l, B_l = optimal_matrices(l, -5, 5, -5, 5)
    A, B = _kron_blocks(A_l, B_l, 3, 2, 2)
    _, zmax = winograd_fgemm_z(A, B, None, 1, 0, l)
    assert zmax == bounds.winograd_bound(l, 2**l * 2, -5, 5, -5, 5)
