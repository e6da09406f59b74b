"""Delayed-reduction bounds and operation counts of the paper -- TEST INFRASTRUCTURE.

Each function restates one formula of the paper in exact integer (or Fraction)
arithmetic, with no floating point.  Pins: tests/test_oracle_bounds.py (values
the paper prints: Table 1, the t_del / t_update table of section 4.4, the
dimensions quoted after eq. trsmboundcen).
"""
from __future__ import annotations

from fractions import Fraction

INT_MAX = 2**31 - 1


def lambda_positive(p: int, gamma: int) -> int:
    """Eq. (1), section 2.1.2: the largest lambda with lambda*(p-1)^2 < 2^gamma
    (number of products of residues in [0, p-1] that can be summed exactly)."""
    q = (p - 1) ** 2
    return (2**gamma - 1) // q


def lambda_centered(p: int, gamma: int) -> int:
    """Eq. (2): the largest lambda with lambda*((p-1)/2)^2 < 2^(gamma-1)
    (balanced residues in [-(p-1)/2, (p-1)/2], odd p)."""
    # lambda*(p-1)^2/4 < 2^(gamma-1)  <=>  lambda*(p-1)^2 < 2^(gamma+1)
    q = (p - 1) ** 2
    return (2 ** (gamma + 1) - 1) // q


def winograd_bound(l: int, k: int, mA: int, MA: int, mB: int, MB: int) -> int:
    """Theorem 3.1: bound on every intermediate value of A*B + beta*C computed
    with l >= 1 recursive levels of Winograd's algorithm, entries of A in
    [mA, MA] and of B in [mB, MB]."""
    if l < 1:
        raise ValueError("Theorem 3.1 is stated for l >= 1")
    ta = Fraction(1 + 3**l, 2) * MA + Fraction(1 - 3**l, 2) * mA
    tb = Fraction(1 + 3**l, 2) * MB + Fraction(1 - 3**l, 2) * mB
    v = ta * tb * (k // 2**l)
    assert v.denominator == 1
    return int(v)


def winograd_bound_positive(l: int, k: int, p: int) -> int:
    """Corollary 3.2 (residues in [0, p-1])."""
    v = Fraction(1 + 3**l, 2) ** 2 * (k // 2**l) * (p - 1) ** 2
    return int(v) if v.denominator == 1 else v


def winograd_bound_balanced(l: int, k: int, p: int) -> Fraction:
    """Corollary 3.3 (balanced residues)."""
    return Fraction(3**l, 2) ** 2 * (k // 2**l) * (p - 1) ** 2


def k_winograd(p: int, gamma: int, l: int, balanced: bool = False) -> Fraction:
    """Corollary 3.4 as printed: l levels of Winograd need no reduction over
    gamma-bit integers as long as k < k_Winograd."""
    lead = 3**l if balanced else 1 + 3**l
    return (Fraction(2 ** (gamma + 2), (lead * (p - 1)) ** 2) + 1) * 2**l


def k_max_winograd(p: int, gamma: int, l: int, balanced: bool = False) -> int:
    """Largest k for which the bound of Corollary 3.2/3.3 stays below 2^gamma
    (the exact inequality behind Corollary 3.4)."""
    per = Fraction(3**l, 2) ** 2 if balanced else Fraction(1 + 3**l, 2) ** 2
    per = per * (p - 1) ** 2
    # largest d = floor(k/2^l) with per*d < 2^gamma, then the largest k with that floor
    d = (Fraction(2**gamma) / per)
    d = int(d) - (1 if d.denominator == 1 else 0)
    return (d + 1) * 2**l - 1


def trsm_growth_positive(p: int, n: int) -> int:
    """Corollary 4.4 / eq. (trsmboundpos) as printed:
    |x| <= (p-1)/2 * (p^(n-1) + (p-1)^(n-1)).  Theorem 4.2 with entries in
    [0, p-1] gives (p-2)^(n-1) in the second term, a tighter bound; the printed
    form is kept because the paper's t_del values follow from it."""
    v = Fraction(p - 1, 2) * (p ** (n - 1) + (p - 1) ** (n - 1))
    return int(v) if v.denominator == 1 else v


def trsm_growth_balanced(p: int, n: int, exponent_n: bool = True):
    """Eq. (trsmboundcen) with exponent n (the reading used here; Corollary 4.5
    prints exponent n-1)."""
    e = n if exponent_n else n - 1
    return Fraction(p - 1, 2) * Fraction(p + 1, 2) ** e


def t_del(p: int, gamma: int, balanced: bool = False, exponent_n: bool = True) -> int:
    """Largest dimension n of a unit-diagonal triangular system that can be
    solved over gamma-bit integers with no reduction (section 4.2)."""
    n = 1
    while True:
        g = trsm_growth_balanced(p, n + 1, exponent_n) if balanced else trsm_growth_positive(p, n + 1)
        if not g < 2**gamma:
            return n
        n += 1


def t_split(p: int, gamma: int) -> int:
    """Algorithm 2's coarse block size t_split = floor(t_W / t_del) * t_del, with
    t_W the classic delayed-reduction length of eq. (1) held in a C int
    (min(lambda, 2^31-1)) and t_del from eq. (trsmboundpos).  This reproduces
    the t_update column of the table in section 4.4."""
    tw = min(lambda_positive(p, gamma), INT_MAX)
    td = t_del(p, gamma)
    return (tw // td) * td


def winograd_ops(n: int, levels: int) -> int:
    """Table 1: arithmetic operations of an n x n product with `levels`
    recursive levels of Winograd's variant: T_0(n) = 2n^3 - n^2 (classic) and
    T_l(n) = 7 T_{l-1}(n/2) + 15 (n/2)^2 (7 products, 15 additions)."""
    if levels == 0:
        return 2 * n**3 - n**2
    h = n // 2
    return 7 * winograd_ops(h, levels - 1) + 15 * h * h


def winograd_levels(n: int, w: int) -> int:
    """Section 3.2.1: l = floor(log2(n/w)) + 1 levels for threshold w (0 if n < w)."""
    if n < w:
        return 0
    l = 0
    while (n >> (l + 1)) >= w:
        l += 1
    return l + 1
