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


def _back_substitute(T, b):
    """x with T x = b over Z for unit upper triangular T (exact integers)."""
    n = len(b)
    x = [0] * n
    for i in range(n - 1, -1, -1):
        x[i] = b[i] - sum(T[i][j] * x[j] for j in range(i + 1, n))
    return x


def _sign_chasing_system(n, m, M):
    """The system of the optimality argument after Theorem 4.2: every entry at
    the end of [m, M] that pushes the next unknown further from zero, the
    unknowns alternating in sign (entries M at odd distance from the diagonal,
    m at even distance; b ends in M and alternates upwards)."""
    T = [[1 if j == i else (M if (j - i) % 2 else m) if j > i else 0 for j in range(n)] for i in range(n)]
    b = [M if (n - 1 - i) % 2 == 0 else m for i in range(n)]
    return T, b


def _v(k, m, M):
    from fractions import Fraction
    return Fraction(M - m, 2) * (M + 1) ** k + Fraction(M + m, 2) * (M - 1) ** k


@pytest.mark.parametrize("p", [3, 5, 7, 251, 1001, 65521])
def test_trsm_growth_reached_with_balanced_residues(p):
    # Corollary 4.3's bound is reached exactly for a range symmetric about
    # zero: |x_{n-k}| = v_k for every k, so Corollary 4.5 (exponent n - 1) is
    # the maximum for balanced residues
    M = (p - 1) // 2
    for n in range(1, 9):
        x = _back_substitute(*_sign_chasing_system(n, -M, M))
        assert [abs(x[n - 1 - k]) for k in range(n)] == [_v(k, -M, M) for k in range(n)]
        assert max(abs(t) for t in x) == bounds.trsm_growth_balanced(p, n, exponent_n=False)


@pytest.mark.parametrize("n,p", [(1, 11), (2, 11), (3, 11), (4, 11), (4, 7), (5, 5)])
def test_trsm_growth_positive_residues(n, p):
    # x is multilinear in the entries, so its extremes lie at the vertices
    # {0, p - 1}.  The exhaustive maximum never exceeds Theorem 4.2's v_{n-1}
    # for [m, M] = [0, p - 1], equals it up to n = 3 and stays strictly below
    # from n = 4 on (the optimality stated after the theorem holds for ranges
    # symmetric about zero); Corollary 4.4 as printed, with (p - 1)^(n-1)
    # where the theorem gives (M - 1)^(n-1) = (p - 2)^(n-1), is looser still
    # from n = 2 on.  Both stay upper bounds, which is all t_del needs.
    import itertools
    M = p - 1
    pos = [(i, j) for i in range(n) for j in range(i + 1, n)]
    best = 0
    for te in itertools.product((0, M), repeat=len(pos)):
        T = [[1 if i == j else 0 for j in range(n)] for i in range(n)]
        for (i, j), val in zip(pos, te):
            T[i][j] = val
        for b in itertools.product((0, M), repeat=n):
            best = max(best, max(abs(t) for t in _back_substitute(T, list(b))))
    theorem = _v(n - 1, 0, M)
    printed = bounds.trsm_growth_positive(p, n)
    assert best <= theorem <= printed
    assert (best == theorem) == (n <= 3)
    assert (theorem == printed) == (n == 1)
    # the sign-chasing system attains the exhaustive maximum
    x = _back_substitute(*_sign_chasing_system(n, 0, M))
    assert max(abs(t) for t in x) == best


@pytest.mark.parametrize("p", [3, 5, 251, 65521, 1048573, 8388593])
@pytest.mark.parametrize("l", [1, 2, 3])
@pytest.mark.parametrize("gamma", [53, 62])
def test_k_max_winograd_balanced_by_search(p, l, gamma):
    """k_max_winograd(balanced=True) against a search on Theorem 3.1 itself
    with balanced ranges [-(p-1)/2, (p-1)/2] (the theorem is pinned by the
    appendix's matrices in test_oracle_winograd.py): the largest k whose bound
    stays below 2^gamma."""
    h = (p - 1) // 2
    ok = lambda k: bounds.winograd_bound(l, k, -h, h, -h, h) < 2**gamma
    assert bounds.k_max_winograd(p, gamma, l, balanced=True) == _largest_k(ok, l)
    # and the positive range [0, p-1] (Corollary 3.2) the same way
    okp = lambda k: bounds.winograd_bound(l, k, 0, p - 1, 0, p - 1) < 2**gamma
    assert bounds.k_max_winograd(p, gamma, l, balanced=False) == _largest_k(okp, l)


def _largest_k(ok, l):
    """Largest k with ok(k), for a predicate that holds below 2^l (the bound
    depends on floor(k / 2^l)) and is monotone."""
    if not ok(2**l):
        return 2**l - 1
    lo, hi = 2**l, 2**(l + 1)
    while ok(hi):
        lo, hi = hi, 2 * hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo
