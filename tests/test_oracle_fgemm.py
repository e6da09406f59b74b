"""Pins of the fgemm oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped alpha or
beta term, an index or operand transposed, a lost leading dimension, a 64-bit
overflow of the sum of products) fails at least one of them:
  * brute force over every tiny input, and random inputs, against numpy's exact
    object-dtype product (a library routine, not the oracle's loop);
  * the closed form for all-(p-1) matrices: (p-1)^2 = 1 mod p, so the product
    is k*J; with k = 64 and p = 2^31-1 the unreduced sum exceeds 2^64;
  * identities: identity and permutation matrices, associativity and
    distributivity, A*A^{-1} = I and det(AB) = det(A)det(B) with sympy's
    modular inverse and determinant.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_cs_0601133_gb300 import workloads as W

PRIMES = [2, 3, 5, 251, 65521, 8388593, 2147483647]


def ref(A, B, p, alpha=1, beta=0, C=None):
    """numpy exact product with Python ints (object dtype)."""
    prod = A.astype(object) @ B.astype(object)
    out = alpha * prod
    if C is not None:
        out = out + beta * C.astype(object)
    return (out % p).astype(np.uint64).astype(np.uint32)


def test_brute_force_all_tiny_inputs_p2():
    # every A (2x2), B (2x2), alpha, beta and C over Z/2Z
    p = 2
    vals = list(itertools.product(range(p), repeat=4))
    C = np.array([[1, 0], [1, 1]], np.uint32)
    for a in vals:
        A = np.array(a, np.uint32).reshape(2, 2)
        for b in vals:
            B = np.array(b, np.uint32).reshape(2, 2)
            for alpha, beta in ((1, 0), (1, 1), (0, 1)):
                got = oracle.fgemm(A, B, p, alpha, beta, C)
                assert np.array_equal(got, ref(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("p", [3, 5])
def test_brute_force_all_tiny_inputs_rect(p):
    # every A (1x2) and B (2x2) over Z/pZ, and every (alpha, beta)
    vals2 = list(itertools.product(range(p), repeat=2))
    vals4 = list(itertools.product(range(p), repeat=4))
    C = np.array([[p - 1, 1]], np.uint32)
    for a in vals2:
        A = np.array(a, np.uint32).reshape(1, 2)
        for b in vals4:
            B = np.array(b, np.uint32).reshape(2, 2)
            alpha, beta = (a[0] + 1) % p, (b[3] + 2) % p
            got = oracle.fgemm(A, B, p, alpha, beta, C)
            assert np.array_equal(got, ref(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("p", PRIMES)
def test_random_against_numpy(p):
    rng = np.random.default_rng(p)
    m, k, n = 37, 53, 29
    # arbitrary 32-bit words (inputs >= p are taken mod p) and padded leading dims
    Abuf = W.uniform_words(rng, (m, k + 5))
    Bbuf = W.uniform_words(rng, (k, n + 3))
    Cbuf = W.uniform_words(rng, (m, n + 7))
    A, B, C = Abuf[:, :k], Bbuf[:, :n], Cbuf[:, :n]
    alpha, beta = int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))
    got = oracle.fgemm(A, B, p, alpha, beta, C)
    assert np.array_equal(got, ref(A, B, p, alpha % p, beta % p, C))


@pytest.mark.parametrize("p", [251, 65521, 2147483647])
def test_closed_form_all_p_minus_1(p):
    m, k, n = 5, 64, 7
    A, B, C = W.adversarial_problem(m, n, k, p)
    rng = np.random.default_rng(1)
    C = W.uniform_residues(rng, (m, n), p)
    alpha, beta = 12345 % p, 678 % p
    got = oracle.fgemm(A, B, p, alpha, beta, C)
    expect = ((alpha * k + beta * C.astype(object)) % p).astype(np.uint32)
    assert np.array_equal(got, expect)


def test_degenerate_shapes():
    p = 65521
    rng = np.random.default_rng(2)
    C = W.uniform_residues(rng, (4, 3), p)
    A = np.zeros((4, 0), np.uint32)
    B = np.zeros((0, 3), np.uint32)
    got = oracle.fgemm(A, B, p, 7, 5, C)
    assert np.array_equal(got, (5 * C.astype(object) % p).astype(np.uint32))
    assert oracle.fgemm(np.zeros((0, 3), np.uint32), np.zeros((3, 4), np.uint32), p).shape == (0, 4)


@pytest.mark.parametrize("p", [5, 65521, 2147483647])
def test_identity_and_permutation(p):
    rng = np.random.default_rng(3)
    n = 19
    A = W.uniform_residues(rng, (n, n), p)
    I = np.eye(n, dtype=np.uint32)
    assert np.array_equal(oracle.fgemm(A, I, p), A)
    assert np.array_equal(oracle.fgemm(I, A, p), A)
    perm = rng.permutation(n)
    P = np.zeros((n, n), np.uint32)
    P[np.arange(n), perm] = 1
    assert np.array_equal(oracle.fgemm(P, A, p), A[perm, :])      # rows permuted
    assert np.array_equal(oracle.fgemm(A, P.T.copy(), p), A[:, perm])  # columns permuted


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
def test_associativity_distributivity(p):
    rng = np.random.default_rng(4)
    A = W.uniform_residues(rng, (11, 13), p)
    B = W.uniform_residues(rng, (13, 17), p)
    B2 = W.uniform_residues(rng, (13, 17), p)
    C = W.uniform_residues(rng, (17, 5), p)
    left = oracle.fgemm(oracle.fgemm(A, B, p), C, p)
    right = oracle.fgemm(A, oracle.fgemm(B, C, p), p)
    assert np.array_equal(left, right)
    BpB2 = ((B.astype(np.uint64) + B2) % p).astype(np.uint32)
    lhs = oracle.fgemm(A, BpB2, p)
    rhs = oracle.fgemm(A, B2, p, 1, 1, oracle.fgemm(A, B, p))
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("p", [3, 7, 251])
def test_inverse_and_determinant_small_primes(p):
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(5 + p)
    n = 6
    for _ in range(4):
        while True:
            A = W.uniform_residues(rng, (n, n), p)
            MA = sympy.Matrix(A.astype(int).tolist())
            if MA.det() % p != 0:
                break
        Ainv = np.array(MA.inv_mod(p).tolist(), dtype=np.int64).astype(np.uint32)
        assert np.array_equal(oracle.fgemm(A, Ainv, p), np.eye(n, dtype=np.uint32))
        assert np.array_equal(oracle.fgemm(Ainv, A, p), np.eye(n, dtype=np.uint32))
        B = W.uniform_residues(rng, (n, n), p)
        AB = oracle.fgemm(A, B, p)
        dAB = sympy.Matrix(AB.astype(int).tolist()).det() % p
        dA = MA.det() % p
        dB = sympy.Matrix(B.astype(int).tolist()).det() % p
        assert dAB == (dA * dB) % p


def test_entries_and_matvec_match_full():
    p = 2147483647
    rng = np.random.default_rng(6)
    A = W.uniform_words(rng, (40, 70))
    B = W.uniform_words(rng, (70, 50))
    C = W.uniform_words(rng, (40, 50))
    full = oracle.fgemm(A, B, p, 3, 4, C)
    rows = rng.integers(0, 40, 100)
    cols = rng.integers(0, 50, 100)
    got = oracle.fgemm_entries(A, B, p, 3, 4, C, rows, cols)
    assert np.array_equal(got, full[rows, cols])
    x = W.uniform_residues(rng, (70,), p)
    assert np.array_equal(oracle.matvec(A, x, p), ref(A, x.reshape(-1, 1), p).ravel())


def test_freivalds_accepts_correct_and_rejects_planted_error():
    p = 65521
    rng = np.random.default_rng(7)
    A = W.uniform_residues(rng, (30, 40), p)
    B = W.uniform_residues(rng, (40, 20), p)
    C = W.uniform_residues(rng, (30, 20), p)
    good = oracle.fgemm(A, B, p, 5, 6, C)
    assert oracle.freivalds(A, B, C, good, p, 5, 6)
    bad = good.copy()
    bad[3, 7] = (bad[3, 7] + 1) % p          # mistake planted on the CPU side
    assert not oracle.freivalds(A, B, C, bad, p, 5, 6)
