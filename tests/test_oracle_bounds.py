"""Pins of the bound calculators and operation counts against values the paper prints."""
import os

import pytest

from oracle import bounds

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def test_table1_operation_counts():
    rows = list(_rows("table1_winograd_ops.txt"))
    assert len(rows) == 25
    for n, l, ops in rows:
        assert bounds.winograd_ops(int(n), int(l)) == int(ops)


def test_trsm_threshold_table():
    for r in _rows("trsm_thresholds.txt"):
        if r[0] == "text":
            _, p, rep, nmax = r
            assert bounds.t_del(int(p), 53, balanced=(rep == "balanced")) == int(nmax)
            continue
        p, lg, td, tu = (int(v) for v in r)
        # the printed log2 column is not used: it reads ceil for p = 5 and floor
        # for the two larger primes
        assert lg in ((p - 1).bit_length(), p.bit_length() - 1)
        assert bounds.t_del(p, 53) == td
        assert bounds.t_split(p, 53) == tu


def test_balanced_trsm_reading_for_1001():
    # The text also claims n <= 6 for p = 1001 with balanced residues; neither
    # exponent (n in eq. trsmboundcen, n-1 in Corollary 4.5) gives 6.
    assert bounds.t_del(1001, 53, balanced=True, exponent_n=True) == 4
    assert bounds.t_del(1001, 53, balanced=True, exponent_n=False) == 5


def test_lambda_eq1_eq2():
    # eq. (1): lambda (p-1)^2 < 2^gamma <= (lambda+1)(p-1)^2
    for p in (3, 251, 65521, 1048583, 8388593, 2147483647):
        for g in (24, 31, 53, 64):
            lam = bounds.lambda_positive(p, g)
            assert lam * (p - 1) ** 2 < 2**g <= (lam + 1) * (p - 1) ** 2
            lc = bounds.lambda_centered(p, g)
            assert 4 * lc * ((p - 1) // 2) ** 2 <= lc * (p - 1) ** 2 < 2 ** (g + 1)
    assert bounds.lambda_positive(65521, 53) == 2098176
    assert bounds.lambda_positive(251, 24) == 268        # FP32 path at p = 251
    assert bounds.lambda_centered(251, 24) == 536        # twice as many (eq. 2, signed 24-bit)
    assert bounds.lambda_positive(8388593, 53) == 128


def test_k_winograd_consistent_with_corollary_bounds():
    for p in (251, 65521, 1048583):
        for l in (1, 2, 3):
            for bal in (False, True):
                kmax = bounds.k_max_winograd(p, 53, l, bal)
                f = bounds.winograd_bound_balanced if bal else bounds.winograd_bound_positive
                assert f(l, kmax, p) < 2**53
                assert not f(l, kmax + 1, p) < 2**53 or (kmax + 1) // 2**l == kmax // 2**l
                # Corollary 3.4's closed form agrees up to the floor
                kw = bounds.k_winograd(p, 53, l, bal)
                assert abs(kw - (kmax + 1)) <= 2**l


def test_winograd_levels_formula():
    assert bounds.winograd_levels(1000, 1000) == 1
    assert bounds.winograd_levels(999, 1000) == 0
    assert bounds.winograd_levels(4000, 1000) == 3
    assert bounds.winograd_levels(3999, 1000) == 2
