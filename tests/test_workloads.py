"""The seeded input generators (CPU): the primes they pick, the ranges and
shapes of every family, and that each draw is reproducible.  They hold no
arithmetic of the method; these checks pin the workload recipe itself."""
import numpy as np
import pytest

import oracle
from paper_cs_0601133_gb300 import workloads as W


def test_is_prime_against_sympy():
    sympy = pytest.importorskip("sympy")
    # small numbers, Carmichael numbers, squares of primes, strong pseudoprimes to base 2
    special = [561, 1105, 1729, 2465, 2821, 6601, 8911, 2047, 3277, 4033, 4681, 8321, 25326001,
               3215031751, 2152302898747, 65521 ** 2, 2147483647 * 3]
    for n in list(range(0, 3000)) + special + list(range(2147483000, 2147483648)):
        assert W.is_prime(n) == sympy.isprime(n), n


def test_sweep_and_multimodular_primes():
    sympy = pytest.importorskip("sympy")
    assert W.sweep_primes() == [251, 65521, 8388593, 2147483647]
    for bits, p in zip(W.SWEEP_BITS, W.sweep_primes()):
        assert p == sympy.prevprime(2 ** bits)
    _, primes = W.multimodular_instances(count=4, nprimes=32)
    want, q = [], 2 ** 31
    for _ in range(32):
        q = sympy.prevprime(q)
        want.append(q)
    assert list(primes) == want
    assert primes[0] == 2147483647 and primes[-1] == 2147482921


def test_multimodular_instances_recipe():
    shapes, primes = W.multimodular_instances(count=4096, nprimes=32)
    s = np.asarray(shapes)
    assert s.shape == (4096, 3)
    assert s.min() >= 16 and s.max() <= 1024
    # log-uniform: the median dimension is near sqrt(16 * 1024) = 128
    assert 100 <= np.median(s) <= 160
    again, _ = W.multimodular_instances(count=4096, nprimes=32)
    assert np.array_equal(s, np.asarray(again))
    A, B = W.multimodular_integers(7, 5, 6, 9)
    assert A.shape == (5, 9) and B.shape == (9, 6)
    assert A.min() >= -(2 ** 20) and A.max() <= 2 ** 20
    assert np.array_equal(A, W.multimodular_integers(7, 5, 6, 9)[0])
    p = 2147483629
    assert np.array_equal(W.reduce_signed(np.array([-1, 0, p, -p - 3]), p), np.array([p - 1, 0, 0, p - 3]))


def test_square_and_adversarial_problems():
    A, B, C, alpha, beta = W.square_problem(64, 65521)
    for X in (A, B, C):
        assert X.dtype == np.uint32 and X.shape == (64, 64) and X.max() < 65521
    assert 0 <= alpha < 65521 and 0 <= beta < 65521
    A2, _, _, a2, b2 = W.square_problem(64, 65521)
    assert np.array_equal(A, A2) and (alpha, beta) == (a2, b2)
    A, B, C = W.adversarial_problem(3, 4, 5, 251)
    assert (A == 250).all() and (B == 250).all() and (C == 250).all() and B.shape == (5, 4)


def test_serving_mix_recipe():
    reqs = W.serving_requests(2000, rate_per_s=1.0)
    assert len(reqs) == 2000
    kinds = [r["kind"] for r in reqs]
    assert 900 <= kinds.count("fgemm") <= 1100 and set(kinds) == {"fgemm", "ftrsm"}
    t = [r["t_arrival"] for r in reqs]
    assert t[0] == 0.0 and all(b >= a for a, b in zip(t, t[1:]))
    assert {r["p"] for r in reqs} == set(W.sweep_primes())
    for r in reqs:
        assert 64 <= r["n"] <= 4096
        if r["kind"] == "fgemm":
            assert r["nrhs"] == r["n"]
        else:
            assert 1 <= r["nrhs"] <= 2 * r["n"]
    # Poisson arrivals at rate 1/s: mean gap near 1 s
    assert 0.9 <= t[-1] / 1999 <= 1.1


def test_triangular_shapes():
    rng = W.rng_for("ftrsm", 1)
    for uplo in ("L", "U"):
        for unit in (True, False):
            T = W.triangular(rng, 50, 65521, uplo, unit)
            off = np.triu(T, 1) if uplo == "L" else np.tril(T, -1)
            assert not off.any()
            d = np.diag(T)
            assert (d == 1).all() if unit else (d >= 1).all()


def test_lqup_matrix_kinds():
    p = 65521
    rng = W.rng_for("lqup", 99)
    A = W.lqup_matrix(rng, 120, 150, p, "copies", r=30)
    assert oracle.rank(A, p) <= 30
    Z = W.lqup_matrix(rng, 40, 90, p, "zerolead", z=25)
    assert not Z[:, :25].any()
    S = W.lqup_matrix(rng, 200, 200, 3, "sparse", density=0.05)
    assert 0.02 < np.count_nonzero(S) / S.size < 0.05
    with pytest.raises(ValueError):
        W.lqup_matrix(rng, 2, 2, p, "other")
