"""Pins of the ftrsm oracle (CPU only).

  * the residual op(T) X = alpha B (left) or X op(T) = alpha B (right), checked
    with the fgemm oracle (itself pinned by test_oracle_fgemm against numpy);
  * sympy's exact solution over Z/pZ on small systems;
  * T = I gives X = alpha B; a singular diagonal is rejected.
"""
import numpy as np
import pytest

import oracle
from paper_cs_0601133_gb300 import workloads as W


def tri_op(T, uplo):
    return T


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("diag", ["U", "N"])
def test_residual(p, side, uplo, diag):
    rng = np.random.default_rng(hash((p, side, uplo, diag)) % 2**32)
    m, n = 23, 17
    nt = m if side == "L" else n
    T = W.triangular(rng, nt, p, uplo, diag == "U")
    B = W.uniform_words(rng, (m, n))
    alpha = int(rng.integers(1, p))
    X = oracle.ftrsm(T, B, p, alpha, side, uplo, diag)
    Bred = (alpha * B.astype(object) % p).astype(np.uint32)
    if side == "L":
        lhs = oracle.fgemm(T, X, p)
    else:
        lhs = oracle.fgemm(X, T, p)
    assert np.array_equal(lhs, Bred)
    # the unit-diagonal solve must ignore whatever sits on the diagonal
    if diag == "U":
        T2 = T.copy()
        np.fill_diagonal(T2, 12345)
        assert np.array_equal(oracle.ftrsm(T2, B, p, alpha, side, uplo, "U"), X)


@pytest.mark.parametrize("p", [5, 251])
def test_against_sympy(p):
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(11)
    T = W.triangular(rng, 6, p, "L", False)
    B = W.uniform_residues(rng, (6, 3), p)
    X = oracle.ftrsm(T, B, p, 1, "L", "L", "N")
    MT = sympy.Matrix(T.astype(int).tolist())
    expect = (MT.inv_mod(p) * sympy.Matrix(B.astype(int).tolist())).applyfunc(lambda v: v % p)
    assert np.array_equal(X, np.array(expect.tolist(), dtype=np.int64).astype(np.uint32))


def test_identity_and_singular():
    p = 65521
    rng = np.random.default_rng(12)
    B = W.uniform_residues(rng, (9, 4), p)
    I = np.eye(9, dtype=np.uint32)
    assert np.array_equal(oracle.ftrsm(I, B, p, 7, "L", "U", "N"), (7 * B.astype(object) % p).astype(np.uint32))
    T = W.triangular(rng, 9, p, "L", False)
    T[4, 4] = 0
    with pytest.raises(ValueError):
        oracle.ftrsm(T, B, p, 1, "L", "L", "N")
