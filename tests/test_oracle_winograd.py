"""Pins of the Winograd schedule oracle (Table 2 with the A22 reading of row 16)."""
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
