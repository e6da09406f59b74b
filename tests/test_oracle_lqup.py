"""Pins of the LQUP / rank / determinant / inverse oracle (CPU only).

  * reconstruction over exact integers: A[rowperm][:, colperm] = L U mod p,
    L unit lower trapezoidal, U upper trapezoidal with a non-zero diagonal,
    rows past the rank zero beyond column r;
  * uniqueness of the pivots (the rule of the oracle's header): the pivot rows
    are exactly the rows that raise the rank of the leading rows, and pivot k's
    column is the first column that raises the rank of the leading rows
    restricted to the earlier pivot columns -- ranks from sympy over GF(p);
  * rank against sympy's GF(p) rank and, for p = 2 and 3, a brute-force count
    of the solutions of A x = 0 (p^(n - r) of them);
  * determinant against the Leibniz formula (n <= 6) and sympy;
    det(AB) = det(A) det(B); zero for rank-deficient matrices;
  * inverse: A X = I over exact integers, sympy's inverse, None when singular.
"""
import itertools

import numpy as np
import pytest
from sympy import GF
from sympy.polys.matrices import DomainMatrix

import oracle
from paper_cs_0601133_gb300 import workloads as W

PRIMES = [2, 3, 5, 251, 65521, 2147483647]


def gf(A, p):
    K = GF(p)
    m, n = A.shape
    return DomainMatrix([[K(int(x)) for x in row] for row in A], (m, n), K)


def sym_rank(A, p):
    if A.shape[0] == 0 or A.shape[1] == 0:
        return 0
    return gf(A, p).rank()


def unpack(M, r):
    m, n = M.shape
    L = np.zeros((m, r), object)
    U = np.zeros((r, n), object)
    for a in range(m):
        for b in range(min(a, r)):
            L[a, b] = int(M[a, b])
        if a < r:
            L[a, a] = 1
    for a in range(r):
        for b in range(a, n):
            U[a, b] = int(M[a, b])
    return L, U


def cases():
    out = []
    for p in PRIMES:
        for (m, n) in [(1, 1), (4, 4), (7, 5), (5, 9), (13, 13)]:
            out.append((p, m, n, "uniform"))
        out.append((p, 10, 12, "copies"))
        out.append((p, 12, 9, "zerolead"))
        out.append((p, 11, 11, "sparse"))
    return out


def make(p, m, n, kind, seed=0):
    rng = W.rng_for("lqup", p % 1000003, m, n, seed, ["uniform", "copies", "zerolead", "sparse"].index(kind))
    return W.lqup_matrix(rng, m, n, p, kind, r=max(1, min(m, n) // 3), z=3, density=0.3)


@pytest.mark.parametrize("p,m,n,kind", cases())
def test_reconstruction_and_structure(p, m, n, kind):
    A = make(p, m, n, kind)
    M, r, rp, cp = oracle.lqup(A, p)
    assert sorted(rp.tolist()) == list(range(m)) and sorted(cp.tolist()) == list(range(n))
    L, U = unpack(M, r)
    assert np.array_equal((L.dot(U)) % p, A[rp][:, cp].astype(object) % p)
    for k in range(r):
        assert M[k, k] != 0
    assert not M[r:, r:].any()
    # stable orders: pivot rows ascending, the rest ascending; non-pivot columns ascending
    assert list(rp[:r]) == sorted(rp[:r]) and list(rp[r:]) == sorted(rp[r:])
    assert list(cp[r:]) == sorted(cp[r:])
    assert r == sym_rank(A, p)


@pytest.mark.parametrize("p,m,n,kind", [c for c in cases() if c[1] * c[2] <= 130])
def test_pivots_are_the_rank_profile(p, m, n, kind):
    A = make(p, m, n, kind, seed=1)
    _, r, rp, cp = oracle.lqup(A, p)
    piv_rows = set(int(x) for x in rp[:r])
    prev = 0
    for i in range(m):
        ri = sym_rank(A[: i + 1], p)
        assert (ri > prev) == (i in piv_rows)
        prev = ri
    for k in range(r):
        t = int(rp[k])
        earlier = [int(x) for x in cp[:k]]
        rows = A[: t + 1]
        for j in range(n):
            if j in earlier:
                continue
            grows = sym_rank(rows[:, earlier + [j]], p) == k + 1
            if j < cp[k]:
                assert not grows, "a smaller column would have been a pivot"
            elif j == cp[k]:
                assert grows
                break


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", ["uniform", "copies", "sparse"])
def test_rank_brute_force_kernel(p, kind):
    for seed in range(6):
        A = make(p, 4, 5, kind, seed=seed)
        n = A.shape[1]
        X = np.array(list(itertools.product(range(p), repeat=n)), dtype=np.int64)
        zero = ((A.astype(np.int64) @ X.T) % p == 0).all(axis=0).sum()
        r = oracle.rank(A, p)
        assert p ** (n - r) == zero
        assert oracle.lqup(A, p)[1] == r


def leibniz(A, p):
    n = A.shape[0]
    tot = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        term = 1
        for i in range(n):
            term *= int(A[i, perm[i]])
        tot += -term if inv % 2 else term
    return tot % p


@pytest.mark.parametrize("p", PRIMES)
def test_det_leibniz_and_sympy(p):
    for n in range(0, 7):
        for kind in ("uniform", "copies", "sparse"):
            A = make(p, n, n, kind, seed=2) if n else np.zeros((0, 0), np.uint32)
            d = oracle.det(A, p)
            if n:
                assert d == leibniz(A, p)
            else:
                assert d == 1 % p
    A = make(p, 25, 25, "uniform", seed=3)
    assert oracle.det(A, p) == int(gf(A, p).det()) % p


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
def test_det_multiplicative_and_singular(p):
    A = make(p, 20, 20, "uniform", seed=4)
    B = make(p, 20, 20, "uniform", seed=5)
    AB = oracle.fgemm(A, B, p)
    assert oracle.det(AB, p) == (oracle.det(A, p) * oracle.det(B, p)) % p
    S = make(p, 20, 20, "copies", seed=6)
    assert oracle.rank(S, p) < 20 and oracle.det(S, p) == 0


@pytest.mark.parametrize("p", PRIMES)
def test_inverse(p):
    for seed in range(3):
        A = make(p, 15, 15, "uniform", seed=10 + seed)
        X = oracle.inverse(A, p)
        if oracle.rank(A, p) < 15:
            assert X is None
            continue
        assert np.array_equal(A.astype(object).dot(X.astype(object)) % p, np.eye(15, dtype=object))
        K = gf(A, p).inv()
        assert [[int(v) % p for v in row] for row in K.to_Matrix().tolist()] == X.tolist()
    S = make(p, 9, 9, "copies", seed=20)
    assert oracle.inverse(S, p) is None


def test_zero_and_empty():
    M, r, rp, cp = oracle.lqup(np.zeros((4, 6), np.uint32), 7)
    assert r == 0 and list(rp) == list(range(4)) and list(cp) == list(range(6)) and not M.any()
    M, r, rp, cp = oracle.lqup(np.zeros((0, 5), np.uint32), 7)
    assert r == 0 and len(rp) == 0 and list(cp) == list(range(5))
    assert oracle.rank(np.zeros((3, 0), np.uint32), 5) == 0


def test_inputs_reduced_mod_p():
    rng = W.rng_for("lqup", 99)
    A = W.uniform_words(rng, (8, 8))
    p = 65521
    Ar = (A % p).astype(np.uint32)
    a = oracle.lqup(A, p)
    b = oracle.lqup(Ar, p)
    assert a[1] == b[1] and np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    assert oracle.det(A, p) == oracle.det(Ar, p)
