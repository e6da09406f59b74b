"""GPU parity of ffgpu_ftrsm (section 4, Algorithm 1) against the CPU oracle.

Sizes cross the leaf size several times (the leaves grow from 128 to 1024
rows with the triangle, their inverses built by 128-block substitution and
0-3 doubling levels of batched products), with ragged splits and ragged last
leaves, both sides, both triangles, unit and non-unit diagonals, and alpha.
A larger solve is checked by its residual op(T) X = alpha B with Freivalds'
test (random vectors, exact matrix-vector products on the CPU)."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


def solve(T, B, p, alpha, side, uplo, diag, algorithm="default"):
    dT, dB = to_dev(T), to_dev(B)
    ff.ftrsm(dT, dB, p, alpha, side, uplo, diag, algorithm=algorithm)
    torch.cuda.synchronize()
    rc = ff.last_device_error()
    return from_dev(dB), rc


@pytest.mark.parametrize("algorithm", ["recursive", "delayed", "cascade"])
@pytest.mark.parametrize("p", [3, 251, 65521, 2147483647])
@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("diag", ["U", "N"])
def test_against_oracle(p, side, uplo, diag, algorithm):
    rng = W.rng_for("ftrsm", p, ord(side), ord(uplo), ord(diag))
    m, n = (300, 170) if side == "L" else (170, 300)
    nt = m if side == "L" else n
    T = W.triangular(rng, nt, p, uplo, diag == "U")
    # words above p and garbage in the unused triangle must not matter
    T = T + (W.uniform_words(rng, T.shape) % 7).astype(np.uint32) * (np.triu(np.ones_like(T), 1) if uplo == "L" else np.tril(np.ones_like(T), -1))
    B = W.uniform_words(rng, (m, n))
    alpha = int(rng.integers(1, p))
    got, rc = solve(T, B, p, alpha, side, uplo, diag, algorithm)
    assert rc == 0
    expect = oracle.ftrsm(T, B, p, alpha, side, uplo, diag)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("shape", [(1, 1), (64, 3), (65, 1), (129, 200), (1000, 5)])
def test_shapes_left_lower_unit(shape):
    p = 65521
    m, n = shape
    rng = W.rng_for("ftrsm", 7, m, n)
    T = W.unit_lower_triangular(rng, m, p)
    B = W.uniform_residues(rng, (m, n), p)
    got, rc = solve(T, B, p, 1, "L", "L", "U")
    assert rc == 0
    assert np.array_equal(got, oracle.ftrsm(T, B, p, 1, "L", "L", "U"))


def test_large_residual_freivalds():
    p = 2147483647
    m, n = 2048, 1536
    rng = W.rng_for("ftrsm", 8)
    T = W.unit_lower_triangular(rng, m, p)
    B = W.uniform_residues(rng, (m, n), p)
    alpha = 12345
    X, rc = solve(T, B, p, alpha, "L", "L", "U")
    assert rc == 0
    for t in range(2):
        x = W.uniform_residues(np.random.default_rng(t), (n,), p)
        lhs = oracle.matvec(T, oracle.matvec(X, x, p), p)
        rhs = (alpha * oracle.matvec(B, x, p).astype(object) % p).astype(np.uint32)
        assert np.array_equal(lhs, rhs)


def test_singular_diagonal_is_reported():
    p = 65521
    rng = W.rng_for("ftrsm", 9)
    T = W.triangular(rng, 100, p, "L", False)
    T[37, 37] = 0
    B = W.uniform_residues(rng, (100, 10), p)
    _, rc = solve(T, B, p, 1, "L", "L", "N")
    assert rc == -1  # FFGPU_ERR_INVALID
    # the record is cleared once read
    assert ff.last_device_error() == 0


@pytest.mark.parametrize("algorithm", ["recursive", "delayed", "cascade"])
@pytest.mark.parametrize("p", [65521, 2147483647])
@pytest.mark.parametrize("side,uplo,diag", [("L", "L", "U"), ("L", "U", "N"), ("R", "U", "U"), ("R", "L", "N"),
                                            ("L", "L", "N"), ("R", "U", "N")])
def test_doubling_levels_and_ragged_leaves(p, side, uplo, diag, algorithm):
    """2500-row triangle: 512-row leaves (two doubling levels 128 -> 256 ->
    512), the last leaf 452 rows, the last 128-block 68 rows."""
    rng = W.rng_for("ftrsm", 8, p, ord(side), ord(uplo), ord(diag))
    nt, nrhs = 2500, 96
    m, n = (nt, nrhs) if side == "L" else (nrhs, nt)
    T = W.triangular(rng, nt, p, uplo, diag == "U")
    B = W.uniform_words(rng, (m, n))
    alpha = int(rng.integers(1, p))
    got, rc = solve(T, B, p, alpha, side, uplo, diag, algorithm)
    assert rc == 0
    assert np.array_equal(got, oracle.ftrsm(T, B, p, alpha, side, uplo, diag))


@pytest.mark.parametrize("algorithm", ["recursive", "delayed", "cascade"])
def test_three_doubling_levels_four_row_last_leaf(algorithm):
    """4100 rows: 1024-row leaves (doubling 128 -> ... -> 1024), a last leaf
    of 4 rows."""
    p = 2147483647
    rng = W.rng_for("ftrsm", 9)
    nt, nrhs = 4100, 40
    T = W.triangular(rng, nt, p, "L", False)
    B = W.uniform_residues(rng, (nt, nrhs), p)
    got, rc = solve(T, B, p, 5, "L", "L", "N", algorithm)
    assert rc == 0
    assert np.array_equal(got, oracle.ftrsm(T, B, p, 5, "L", "L", "N"))


# ---------------------------------------------------------------------------
# The double cascade (Algorithms 2-3, section 4.3): leaves of t_del rows solved
# over Z with no reduction, updates over Z inside blocks of t_split rows.
# ---------------------------------------------------------------------------

def sign_chasing_upper(n, p):
    """Unit upper T with h = floor(p/2) at odd distance from the diagonal and
    -h at even distance, b alternating up from h at the bottom: the solution
    over Z reaches |x_1| = h (h+1)^(n-1), the growth bound of Corollary 4.5
    (the optimality argument after Theorem 4.2)."""
    h = p // 2
    T = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        T[i, i] = 1
        for j in range(i + 1, n):
            T[i, j] = h if (j - i) % 2 else -h
    b = np.array([h if (n - 1 - i) % 2 == 0 else -h for i in range(n)], dtype=np.int64)
    return T, b


@pytest.mark.parametrize("p", [5, 251, 65521])
@pytest.mark.parametrize("uplo", ["U", "L"])
def test_cascade_leaf_of_t_del_rows_at_the_growth_bound(p, uplo):
    """A triangle of exactly t_del rows (one leaf) built so that the leaf's
    solve over Z reaches the growth bound its size admits; the right-hand
    side repeats b in some columns among random ones (40 columns: two
    column strips).  The lower case is the same system with rows and columns
    reversed."""
    td = ff.ftrsm_cascade_params(p)["t_del"]
    T, b = sign_chasing_upper(td, p)
    if uplo == "L":
        T, b = T[::-1, ::-1].copy(), b[::-1].copy()
    rng = W.rng_for("ftrsm", 80, p, ord(uplo))
    B = W.uniform_residues(rng, (td, 40), p).astype(np.int64)
    for c in (0, 7, 31, 32, 39):
        B[:, c] = b
    Tw, Bw = (T % p).astype(np.uint32), (B % p).astype(np.uint32)
    got, rc = solve(Tw, Bw, p, 1, "L", uplo, "U", "cascade")
    assert rc == 0
    assert np.array_equal(got, oracle.ftrsm(Tw, Bw, p, 1, "L", uplo, "U"))


@pytest.mark.parametrize("p,nt", [(268435399, 700), (65521, 1000), (5, 600), (8388593, 520)])
@pytest.mark.parametrize("side,uplo,diag", [("L", "L", "U"), ("L", "U", "N"), ("R", "L", "N"), ("R", "U", "U")])
def test_cascade_blocks_and_panels(p, nt, side, uplo, diag):
    """p = 268435399 (largest prime below 2^28): t_split = 256, so Algorithm
    2 runs three blocks with an fgemm update mod p between them, each block
    two panels and one exact product over Z; p = 65521, 5, 8388593: one
    block, Algorithm 3's recursion over several panels (products over Z at
    two or three levels)."""
    c = ff.ftrsm_cascade_params(p)
    rng = W.rng_for("ftrsm", 81, p, ord(side), ord(uplo), ord(diag))
    nrhs = 77
    m, n = (nt, nrhs) if side == "L" else (nrhs, nt)
    T = W.triangular(rng, nt, p, uplo, diag == "U")
    B = W.uniform_words(rng, (m, n))
    alpha = int(rng.integers(1, p))
    got, rc = solve(T, B, p, alpha, side, uplo, diag, "cascade")
    assert rc == 0
    assert np.array_equal(got, oracle.ftrsm(T, B, p, alpha, side, uplo, diag))
    if p == 268435399:
        assert c["t_split"] == 256 and nt > 2 * c["t_split"]


def test_cascade_large_residual_freivalds():
    p = 65521
    m, n = 2048, 1536
    rng = W.rng_for("ftrsm", 82)
    T = W.unit_lower_triangular(rng, m, p)
    B = W.uniform_residues(rng, (m, n), p)
    X, rc = solve(T, B, p, 77, "L", "L", "U", "cascade")
    assert rc == 0
    for t in range(2):
        x = W.uniform_residues(np.random.default_rng(t), (n,), p)
        lhs = oracle.matvec(T, oracle.matvec(X, x, p), p)
        rhs = (77 * oracle.matvec(B, x, p).astype(object) % p).astype(np.uint32)
        assert np.array_equal(lhs, rhs)


def test_cascade_singular_diagonal_is_reported():
    p = 65521
    rng = W.rng_for("ftrsm", 83)
    T = W.triangular(rng, 100, p, "U", False)
    T[50, 50] = 0
    B = W.uniform_residues(rng, (100, 10), p)
    _, rc = solve(T, B, p, 1, "L", "U", "N", "cascade")
    assert rc == -1
    assert ff.last_device_error() == 0
