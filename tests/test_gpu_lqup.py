"""GPU parity of ffgpu_lqup / ffgpu_rank / ffgpu_det / ffgpu_inverse
(sections 5-6) against the CPU oracle.

With the pivot rule both sides follow (rows top to bottom, first non-zero
column in original order) the factorization is unique, so the packed matrix,
the rank and both permutations are compared exactly.  Shapes cross the
64-row leaf and the column window several times, with ragged ends, both
orientations of rectangles, padded leading dimensions and inputs above p.
Structured inputs reach the slow paths: rank-deficient matrices (row
rotations after the bottom half), leading zero columns (pivots beyond the
window: the leaf is split down to single rows whose pivot is found by the
whole-row check) and sparse matrices over small fields (skipped columns,
window permutations).  Full-size runs are checked by properties: the
factorization against the matrix with Freivalds' test (exact matrix-vector
products on the CPU), A A^{-1} x = x, det(AB) = det(A) det(B)."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


def gpu_lqup(A, p, pad=0):
    dA = to_dev(A, pad)
    r, rp, cp = ff.lqup(dA, p)
    torch.cuda.synchronize()
    return from_dev(dA), r, rp.cpu().numpy(), cp.cpu().numpy()


def check_same(A, p, pad=0):
    M, r, rp, cp = gpu_lqup(A, p, pad)
    M0, r0, rp0, cp0 = oracle.lqup(A, p)
    assert r == r0
    assert np.array_equal(rp, rp0)
    assert np.array_equal(cp, cp0)
    assert np.array_equal(M, M0)
    return r


def make(p, m, n, kind, seed=0, **kw):
    rng = W.rng_for("lqup", p % 1000003, m, n, seed, ["uniform", "copies", "zerolead", "sparse"].index(kind))
    return W.lqup_matrix(rng, m, n, p, kind, **kw)


SHAPES = [(1, 1), (1, 300), (300, 1), (64, 64), (65, 65), (63, 200), (200, 63), (129, 129), (300, 300),
          (257, 700), (700, 257)]


@pytest.mark.parametrize("p", [2, 3, 251, 65521, 2147483647])
@pytest.mark.parametrize("m,n", SHAPES)
def test_uniform(p, m, n):
    check_same(make(p, m, n, "uniform"), p)


@pytest.mark.parametrize("p", [2, 65521, 2147483647])
@pytest.mark.parametrize("m,n,r", [(200, 200, 37), (300, 180, 100), (180, 300, 150), (256, 256, 1), (130, 500, 70)])
def test_rank_deficient(p, m, n, r):
    rk = check_same(make(p, m, n, "copies", r=r), p)
    assert rk <= r


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
@pytest.mark.parametrize("m,n,z", [(150, 400, 150), (70, 600, 300), (130, 130, 5), (1, 500, 400)])
def test_pivots_beyond_the_window(p, m, n, z):
    check_same(make(p, m, n, "zerolead", z=z), p)


@pytest.mark.parametrize("p", [2, 3, 5, 251])
@pytest.mark.parametrize("density", [0.01, 0.05, 0.3])
def test_sparse_small_fields(p, density):
    check_same(make(p, 260, 333, "sparse", density=density), p)


def test_zero_matrix_and_padding():
    p = 65521
    for m, n in [(70, 90), (5, 5), (128, 3)]:
        M, r, rp, cp = gpu_lqup(np.zeros((m, n), np.uint32), p)
        assert r == 0 and not M.any()
        assert np.array_equal(rp, np.arange(m)) and np.array_equal(cp, np.arange(n))
    A = make(p, 150, 170, "uniform")
    check_same(A, p, pad=13)


def test_inputs_above_p():
    p = 65521
    rng = W.rng_for("lqup", 7)
    A = W.uniform_words(rng, (140, 150))
    check_same(A, p)


@pytest.mark.parametrize("p", [2, 3, 65521, 2147483647])
def test_rank_det_inverse_against_oracle(p):
    for kind, n in [("uniform", 1), ("uniform", 97), ("uniform", 300), ("copies", 120), ("sparse", 150)]:
        A = make(p, n, n, kind, seed=3, r=max(1, n // 2), density=0.05)
        dA = to_dev(A)
        assert ff.rank(dA, p) == oracle.rank(A, p)
        assert ff.det(dA, p) == oracle.det(A, p)
        X0 = oracle.inverse(A, p)
        if X0 is None:
            with pytest.raises(ff.FFGPUError) as e:
                ff.inverse(dA, p)
            assert e.value.status == -7
        else:
            X = ff.inverse(dA, p)
            torch.cuda.synchronize()
            assert np.array_equal(from_dev(X), X0)
        assert np.array_equal(from_dev(dA), A)  # input untouched
    B = make(p, 40, 65, "uniform", seed=4)
    assert ff.rank(to_dev(B), p) == oracle.rank(B, p)


def test_composite_modulus_rejected():
    A = to_dev(np.eye(4, dtype=np.uint32))
    for q in (1, 4, 65535, 2147483646):
        with pytest.raises(ff.FFGPUError):
            ff.lqup(A.clone(), q)
        with pytest.raises(ff.FFGPUError):
            ff.det(A, q)


def test_empty():
    p = 7
    assert ff.rank(torch.zeros((0, 5), dtype=torch.int32, device="cuda"), p) == 0
    assert ff.det(torch.zeros((0, 0), dtype=torch.int32, device="cuda"), p) == 1


def unpack_dense(M, r):
    m, n = M.shape
    L = np.tril(M[:, :r].astype(np.uint32), -1)
    L[np.arange(r), np.arange(r)] = 1
    U = np.triu(M[:r, :].astype(np.uint32))
    return np.ascontiguousarray(L), np.ascontiguousarray(U)


@pytest.mark.parametrize("n,p", [(2048, 65521), (8192, 2147483647)])
def test_full_size_properties(n, p):
    A = make(p, n, n, "uniform", seed=5)
    M, r, rp, cp = gpu_lqup(A, p)
    assert r == n  # a uniform matrix over a field this large is singular with probability below n/p
    assert np.array_equal(rp, np.arange(n)) and np.array_equal(np.sort(cp), np.arange(n))
    L, U = unpack_dense(M, r)
    Ap = np.ascontiguousarray(A[:, cp])
    rng = np.random.default_rng(n)
    for _ in range(2):
        x = rng.integers(0, p, size=n, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(oracle.matvec(Ap, x, p), oracle.matvec(L, oracle.matvec(U, x, p), p))
    dA = to_dev(A)
    X = ff.inverse(dA, p)
    torch.cuda.synchronize()
    Xh = from_dev(X)
    x = rng.integers(0, p, size=n, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(oracle.matvec(A, oracle.matvec(Xh, x, p), p), x)
    # det(A B) = det(A) det(B), the product formed on the GPU
    B = make(p, n, n, "uniform", seed=6)
    dB = to_dev(B)
    AB = ff.fgemm(dA, dB, p)
    assert ff.det(AB, p) == ff.det(dA, p) * ff.det(dB, p) % p
    if n <= 2048:
        assert ff.det(dA, p) == oracle.det(A, p)


def test_repeatable_and_async_safe():
    p = 2147483647
    A = make(p, 500, 520, "copies", r=300)
    a = gpu_lqup(A, p)
    b = gpu_lqup(A, p)
    assert a[1] == b[1] and np.array_equal(a[0], b[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dA = to_dev(A)
        r, rp, cp = ff.lqup(dA, p, stream=s)
    s.synchronize()
    assert r == a[1] and np.array_equal(from_dev(dA), a[0])
