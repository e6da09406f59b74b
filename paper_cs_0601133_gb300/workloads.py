"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws random numbers
and picks primes.  Every workload is derived from ``numpy.random.SeedSequence(601133)``
with one child stream per workload family, so any run can be reproduced.

Workload families (sizes follow the fgemm/ftrsm experiments: square products
with uniform residues modulo a word-size prime, sections 3.3 and 4.4):
  * ``square``: m = n = k, entries i.i.d. uniform in [0, p).
  * ``adversarial``: every entry equal to p - 1 (the largest residue), the case
    that reaches the delayed-reduction bound of eq. (1).
  * ``multimodular``: uneven instances (m, n, k log-uniform in [16, 1024]) of
    one integer matrix pair with entries in [-2^20, 2^20], reduced modulo each of
    32 primes just below 2^31 (the use of fgemm inside Chinese remaindering).
  * ``serving``: Poisson arrivals of mixed fgemm / ftrsm requests.
  * ``lqup``: matrices to factor (section 5): uniform residues (full rank with
    high probability), rank-deficient ones built by copying rows and columns,
    ones whose leading columns are zero, and sparse ones.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 601133
FAMILIES = ("square", "adversarial", "precision", "multimodular", "serving", "ftrsm", "smoke", "lqup",
            "worstcase")


def rng_for(family: str, *extra: int) -> np.random.Generator:
    """Independent generator for a workload family (and optional sub-indices)."""
    idx = FAMILIES.index(family)
    ss = np.random.SeedSequence(SEED, spawn_key=(idx,) + tuple(int(e) for e in extra))
    return np.random.default_rng(ss)


_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (the first twelve prime bases)."""
    if n < 2:
        return False
    for b in _MR_BASES:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_below(bound: int, count: int = 1) -> list[int]:
    """The `count` largest primes strictly below `bound`, in decreasing order."""
    out, c = [], bound - 1
    while len(out) < count and c >= 2:
        if is_prime(c):
            out.append(c)
        c -= 1
    return out


def largest_prime_below_pow2(bits: int) -> int:
    return primes_below(1 << bits, 1)[0]


# The primes of the fgemm sweep: the largest below 2^8, 2^16, 2^23, 2^31.
SWEEP_BITS = (8, 16, 23, 31)


def sweep_primes() -> list[int]:
    return [largest_prime_below_pow2(b) for b in SWEEP_BITS]


def uniform_residues(rng: np.random.Generator, shape, p: int) -> np.ndarray:
    return rng.integers(0, p, size=shape, dtype=np.uint64).astype(np.uint32)


def uniform_words(rng: np.random.Generator, shape) -> np.ndarray:
    """Arbitrary uint32 words (inputs >= p are legal and are taken mod p)."""
    return rng.integers(0, 2**32, size=shape, dtype=np.uint64).astype(np.uint32)


def square_problem(n: int, p: int, with_alpha_beta: bool = True, family: str = "square"):
    """A, B, C uniform in [0, p) of order n, alpha and beta uniform in [0, p)."""
    rng = rng_for(family, n, p)
    A = uniform_residues(rng, (n, n), p)
    B = uniform_residues(rng, (n, n), p)
    C = uniform_residues(rng, (n, n), p)
    if with_alpha_beta:
        alpha, beta = (int(v) for v in rng.integers(0, p, size=2))
    else:
        alpha, beta = 1, 0
    return A, B, C, alpha, beta


def adversarial_problem(m: int, n: int, k: int, p: int):
    """Every entry of A, B and C equal to p - 1."""
    A = np.full((m, k), p - 1, np.uint32)
    B = np.full((k, n), p - 1, np.uint32)
    C = np.full((m, n), p - 1, np.uint32)
    return A, B, C


def signed_word(v: int, p: int) -> int:
    """The word in [0, p) that stands for the signed value v (|v| < p)."""
    return v % p


def sign_pattern_problem(rng: np.random.Generator, m: int, n: int, k: int, p: int, a: int, b: int):
    """A[i][t] = s_i sigma_t a and B[t][j] = sigma_t t_j b as words mod p, with
    random signs s (rows of A), t (columns of B) and sigma (the inner index).

    Every product A[i][t] B[t][j] then equals s_i t_j a b: along each inner
    index the terms of one output entry all carry the same sign, so every
    partial sum of that entry grows monotonically to s_i t_j k a b, the largest
    magnitude a sum of k such terms can reach, while the entries of A, B and
    the result still vary in sign.  C is uniform in [0, p).  Returns
    (A, B, C, s, t) with s and t as int64 arrays of +-1."""
    s = rng.choice(np.array([-1, 1], np.int64), size=m)
    t = rng.choice(np.array([-1, 1], np.int64), size=n)
    sig = rng.choice(np.array([-1, 1], np.int64), size=k)
    wa = np.array([signed_word(a, p), signed_word(-a, p)], np.uint32)
    wb = np.array([signed_word(b, p), signed_word(-b, p)], np.uint32)
    A = wa[((s[:, None] * sig[None, :]) < 0).astype(np.int64)]
    B = wb[((sig[:, None] * t[None, :]) < 0).astype(np.int64)]
    C = uniform_residues(rng, (m, n), p)
    return A, B, C, s, t


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, size) -> np.ndarray:
    v = np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def multimodular_instances(count: int = 4096, nprimes: int = 32, lo: int = 16, hi: int = 1024):
    """Shapes and primes of the batched multi-modular workload.

    Returns (shapes [count, 3] as (m, n, k), primes list).  The integer entries of
    instance i are drawn by ``multimodular_integers(i, shape)``."""
    rng = rng_for("multimodular")
    shapes = log_uniform_int(rng, lo, hi, (count, 3))
    return shapes, primes_below(2**31, nprimes)


def multimodular_integers(i: int, m: int, n: int, k: int):
    """Integer matrices (int64) of instance i, entries uniform in [-2^20, 2^20]."""
    rng = rng_for("multimodular", 1, i)
    A = rng.integers(-(2**20), 2**20 + 1, size=(m, k), dtype=np.int64)
    B = rng.integers(-(2**20), 2**20 + 1, size=(k, n), dtype=np.int64)
    return A, B


def reduce_signed(X: np.ndarray, p: int) -> np.ndarray:
    """Canonical residue in [0, p) of signed integers (input preparation only)."""
    return np.mod(X, p).astype(np.uint32)


def unit_lower_triangular(rng: np.random.Generator, n: int, p: int) -> np.ndarray:
    """Lower triangular, unit diagonal, uniform residues below the diagonal."""
    T = uniform_residues(rng, (n, n), p)
    T = np.tril(T, -1)
    np.fill_diagonal(T, 1)
    return T.astype(np.uint32)


def triangular(rng: np.random.Generator, n: int, p: int, uplo: str, unit: bool) -> np.ndarray:
    """Triangular matrix with uniform residues; a nonzero (hence invertible for
    prime p) diagonal when not unit, an all-ones diagonal when unit."""
    T = uniform_residues(rng, (n, n), p)
    T = np.tril(T, -1) if uplo == "L" else np.triu(T, 1)
    if unit:
        np.fill_diagonal(T, 1)
    else:
        np.fill_diagonal(T, rng.integers(1, p, size=n, dtype=np.uint64).astype(np.uint32))
    return T.astype(np.uint32)


def serving_requests(n_requests: int = 2000, rate_per_s: float = 100.0, lo: int = 64, hi: int = 4096,
                     seed_extra: int = 0):
    """Poisson arrivals of a 50/50 fgemm / ftrsm mix.

    Each request: dict(kind, n, nrhs, p, t_arrival).  fgemm: square n x n;
    ftrsm: unit lower triangular n x n with nrhs uniform in [1, 2n]."""
    rng = rng_for("serving", seed_extra)
    primes = sweep_primes()
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    kinds = rng.integers(0, 2, size=n_requests)
    ns = log_uniform_int(rng, lo, hi, n_requests)
    out = []
    for i in range(n_requests):
        n = int(ns[i])
        kind = "fgemm" if kinds[i] == 0 else "ftrsm"
        nrhs = n if kind == "fgemm" else int(rng.integers(1, 2 * n + 1))
        p = int(primes[int(rng.integers(0, len(primes)))])
        out.append(dict(kind=kind, n=n, nrhs=nrhs, p=p, t_arrival=float(t[i]), seed=i))
    return out


def lqup_matrix(rng: np.random.Generator, m: int, n: int, p: int, kind: str = "uniform",
                r: int | None = None, z: int = 0, density: float = 0.1) -> np.ndarray:
    """An m x n matrix of residues mod p for the factorization tests and bench.

    kind "uniform": i.i.d. uniform residues.
    kind "copies": r uniform base rows, every row a copy of a random base row,
      then every column beyond the first r replaced, with probability 1/2, by a
      copy of a random earlier column (rank at most r; built by copying only).
    kind "zerolead": uniform, with the first z columns zero and every other
      column zero with probability 1/8 (pivots far from the diagonal).
    kind "sparse": each entry non-zero with probability `density`.
    """
    if kind == "uniform":
        return uniform_residues(rng, (m, n), p)
    if kind == "copies":
        r = max(1, min(r if r is not None else min(m, n) // 2, m, n))
        base = uniform_residues(rng, (r, n), p)
        A = base[rng.integers(0, r, size=m)].copy()
        for j in range(r, n):
            if rng.integers(0, 2):
                A[:, j] = A[:, int(rng.integers(0, j))]
        return A
    if kind == "zerolead":
        A = uniform_residues(rng, (m, n), p)
        A[:, : min(z, n)] = 0
        A[:, rng.random(n) < 0.125] = 0
        return A
    if kind == "sparse":
        A = uniform_residues(rng, (m, n), p)
        A[rng.random((m, n)) >= density] = 0
        return A
    raise ValueError("unknown kind %r" % kind)
