"""Pins of the double-cascade oracle (Algorithms 2-3, section 4.3) and of the
thresholds the library derives for it (CPU only).

  * the cascade's result mod p equals plain substitution (oracle.ftrsm, itself
    pinned by its residual and by sympy), for any t_del / t_split;
  * the thresholds: t_del equals the oracle's eq. (trsmboundcen) reading with
    gamma = 63, t_update satisfies its defining inequalities, t_split =
    floor(t_update / t_del) t_del;
  * with those thresholds the largest value the paper's algorithm holds stays
    below 2^63, and on the sign-chasing system of the optimality argument
    (Corollary 4.3) a leaf of exactly t_del rows reaches the growth bound
    h (h+1)^(t_del - 1) of Corollary 4.5.
"""
import numpy as np
import pytest

import oracle
from oracle import bounds
from oracle.trsm_cascade import trsm_rec_blas_delayed
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W


def unit_upper(rng, n, p):
    return W.triangular(rng, n, p, "U", True)


@pytest.mark.parametrize("p", [3, 5, 251, 65521, 1048573])
@pytest.mark.parametrize("t_del,t_split", [(1, 1), (2, 6), (3, 7), (5, 40)])
def test_cascade_equals_substitution(p, t_del, t_split):
    rng = W.rng_for("ftrsm", 70, p, t_del, t_split)
    n, nrhs = 23, 5
    T = unit_upper(rng, n, p)
    B = W.uniform_residues(rng, (n, nrhs), p)
    X, _ = trsm_rec_blas_delayed(T.astype(object), B.astype(object), p, t_del, t_split)
    assert np.array_equal(X.astype(np.uint32), oracle.ftrsm(T, B, p, 1, "L", "U", "U"))


@pytest.mark.parametrize("p", [3, 5, 7, 251, 1001, 65521, 1048573, 8388593, 268435399, 2147483647])
def test_library_thresholds(p):
    c = ff.ftrsm_cascade_params(p)
    h = p // 2
    # eq. (trsmboundcen) with exponent n (the oracle's reading), 63-bit carrier, capped at 128
    assert c["t_del"] == min(bounds.t_del(p, 63, balanced=True), 128)
    # t_update: the largest t with t h^2 + h < 2^62 (capped at 2^31 - 1)
    t = c["t_update"]
    assert t * h * h + h < 2**62
    assert t == 2**31 - 1 or (t + 1) * h * h + h >= 2**62
    # eq. (2) with gamma = 63: lambda ((p-1)/2)^2 < 2^62, one term reserved
    lam = bounds.lambda_centered(p, 63)
    assert t == min(2**31 - 1, lam - 1) or t == min(2**31 - 1, lam)
    assert c["t_split"] == max(1, t // c["t_del"] * c["t_del"])


@pytest.mark.parametrize("p", [5, 251, 65521, 8388593])
def test_intermediates_stay_in_63_bits(p):
    c = ff.ftrsm_cascade_params(p)
    rng = W.rng_for("ftrsm", 71, p)
    n = min(40, 3 * c["t_split"] + 2)
    T = unit_upper(rng, n, p)
    B = W.uniform_residues(rng, (n, 4), p)
    X, zmax = trsm_rec_blas_delayed(T.astype(object), B.astype(object), p, c["t_del"], c["t_split"])
    assert np.array_equal(X.astype(np.uint32), oracle.ftrsm(T, B, p, 1, "L", "U", "U"))
    assert zmax < 2**63


def sign_chasing(n, p):
    """The system of the optimality argument after Theorem 4.2 for the
    balanced range [-h, h]: unit upper T with h at odd distance from the
    diagonal and -h at even distance, b ending in h and alternating upwards;
    the unknowns alternate in sign and |x_{n-k}| = h (h+1)^k."""
    h = p // 2
    T = [[1 if j == i else (h if (j - i) % 2 else -h) if j > i else 0 for j in range(n)] for i in range(n)]
    b = [h if (n - 1 - i) % 2 == 0 else -h for i in range(n)]
    return np.array(T, dtype=object), np.array(b, dtype=object).reshape(n, 1)


@pytest.mark.parametrize("p", [5, 251, 65521])
def test_leaf_of_t_del_rows_reaches_the_growth_bound(p):
    c = ff.ftrsm_cascade_params(p)
    n = c["t_del"]
    h = p // 2
    T, b = sign_chasing(n, p)
    X, zmax = trsm_rec_blas_delayed(T, b, p, n, c["t_split"])
    assert zmax == h * (h + 1) ** (n - 1) == bounds.trsm_growth_balanced(p, n, exponent_n=False)
    assert zmax < 2**63
    Tw = (T % p).astype(np.uint32)
    assert np.array_equal(X.astype(np.uint32), oracle.ftrsm(Tw, (b % p).astype(np.uint32), p, 1, "L", "U", "U"))
