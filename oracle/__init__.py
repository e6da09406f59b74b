"""CPU oracle for fgemm / ftrsm / LQUP over Z/pZ -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and this package imports nothing from the
product path.

Contents
  * ``fgemm``/``fgemm_entries``/``matvec``/``ftrsm``: thin ctypes wrappers over
    ``ffgpu_oracle.c`` (the definitions, exact 128-bit integer arithmetic).
  * ``lqup``/``rank``/``det``/``inverse``: LQUP by row-by-row elimination with
    the first-non-zero pivot rule, rank by column echelon form, determinant by
    Gaussian elimination, inverse by Gauss-Jordan (sections 5-6).
  * ``winograd``: the Strassen-Winograd schedule of Table 2 over Z with the
    intermediate-size tracking of Theorem 3.1 (section 3.2).
  * ``bounds``: the delayed-reduction bounds (eq. 1, eq. 2, Corollaries
    3.2-3.4, eqs. trsmboundpos/trsmboundcen) and the operation counts of
    Table 1.

Parity status: every function here is pinned by tests/test_oracle_*.py
(brute force against numpy object-dtype products, identities, closed forms and
values printed in the paper).  No function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffgpu_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ffgpu_oracle.c into oracle/liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u32, vp, i = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
            lib.oracle_fgemm.argtypes = [i64, i64, i64, u32, u32, vp, i64, vp, i64, u32, vp, i64]
            lib.oracle_fgemm_entries.argtypes = [i64, i64, i64, u32, u32, vp, i64, vp, i64, u32,
                                                 vp, i64, i64, vp, vp, vp]
            lib.oracle_matvec.argtypes = [i64, i64, u32, vp, i64, vp, vp]
            lib.oracle_ftrsm.argtypes = [i, i, i, i64, i64, u32, u32, vp, i64, vp, i64]
            lib.oracle_num_threads.argtypes = []
            lib.oracle_lqup.argtypes = [i64, i64, u32, vp, i64, vp, vp]
            lib.oracle_rank.argtypes = [i64, i64, u32, vp, i64]
            lib.oracle_det.argtypes = [i64, u32, vp, i64, vp]
            lib.oracle_inverse.argtypes = [i64, u32, vp, i64, vp, i64]
            for f in (lib.oracle_fgemm, lib.oracle_fgemm_entries, lib.oracle_matvec,
                      lib.oracle_ftrsm, lib.oracle_num_threads, lib.oracle_det, lib.oracle_inverse):
                f.restype = ctypes.c_int
            lib.oracle_lqup.restype = ctypes.c_int64
            lib.oracle_rank.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype != np.uint32:
        raise TypeError("oracle expects uint32 arrays, got %s" % a.dtype)
    if a.ndim == 2 and a.size and a.strides[1] != 4:
        raise ValueError("rows must be contiguous")
    return a


def _ld(a: np.ndarray) -> int:
    return a.strides[0] // 4 if a.ndim == 2 and a.size else max(a.shape[-1], 1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return _load().oracle_num_threads()


def fgemm(A, B, p: int, alpha: int = 1, beta: int = 0, C=None) -> np.ndarray:
    """Return (alpha*A@B + beta*C) mod p as a new uint32 array (C is not modified)."""
    A, B = _u32(A), _u32(B)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    out = np.zeros((m, n), np.uint32) if C is None else np.array(_u32(C), dtype=np.uint32, copy=True)
    rc = _load().oracle_fgemm(m, n, k, p, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta,
                              _ptr(out), _ld(out))
    if rc != 0:
        raise ValueError("oracle_fgemm failed (%d)" % rc)
    return out


def fgemm_entries(A, B, p: int, alpha: int, beta: int, C, rows, cols) -> np.ndarray:
    """Entries (rows[e], cols[e]) of (alpha*A@B + beta*C) mod p."""
    A, B, C = _u32(A), _u32(B), _u32(C)
    m, k = A.shape
    n = B.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0], np.uint32)
    rc = _load().oracle_fgemm_entries(m, n, k, p, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta,
                                      _ptr(C), _ld(C), rows.shape[0], _ptr(rows), _ptr(cols),
                                      _ptr(out))
    if rc != 0:
        raise ValueError("oracle_fgemm_entries failed (%d)" % rc)
    return out


def matvec(M, x, p: int) -> np.ndarray:
    """(M @ x) mod p, exact."""
    M = _u32(M)
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.empty(M.shape[0], np.uint32)
    rc = _load().oracle_matvec(M.shape[0], M.shape[1], p, _ptr(M), _ld(M), _ptr(x), _ptr(y))
    if rc != 0:
        raise ValueError("oracle_matvec failed (%d)" % rc)
    return y


def ftrsm(T, B, p: int, alpha: int = 1, side: str = "L", uplo: str = "L", diag: str = "U") -> np.ndarray:
    """Solve op(T) X = alpha*B (side L) or X op(T) = alpha*B (side R) mod p; returns X."""
    T, B = _u32(T), _u32(B)
    X = np.array(B, dtype=np.uint32, copy=True)
    m, n = X.shape
    rc = _load().oracle_ftrsm(0 if side == "L" else 1, 0 if uplo == "L" else 1,
                              1 if diag == "U" else 0, m, n, p, alpha, _ptr(T), _ld(T),
                              _ptr(X), _ld(X))
    if rc != 0:
        raise ValueError("oracle_ftrsm failed (%d)" % rc)
    return X


def freivalds(A, B, C_old, C_new, p: int, alpha: int, beta: int, trials: int = 3, seed: int = 0) -> bool:
    """Randomised check C_new == alpha*A@B + beta*C_old (mod p) by matrix-vector
    products with random vectors; a wrong C_new passes one trial with probability
    at most 1/p (Freivalds' test)."""
    rng = np.random.default_rng(seed)
    n = B.shape[1]
    for _ in range(trials):
        x = rng.integers(0, p, size=n, dtype=np.uint64).astype(np.uint32)
        bx = matvec(B, x, p)
        abx = matvec(A, bx, p).astype(object)
        cx = matvec(C_old, x, p).astype(object)
        lhs = (alpha * abx + beta * cx) % p
        rhs = matvec(C_new, x, p).astype(object)
        if not np.array_equal(lhs.astype(np.uint64), rhs.astype(np.uint64)):
            return False
    return True


def lqup(A, p: int):
    """Packed LQUP of A mod p (p prime): returns (M, r, rowperm, colperm) with
    A[rowperm][:, colperm] = L U mod p, M holding L strictly below the diagonal
    of its first r columns and U on and above it (rows >= r zero beyond column
    r).  A is not modified."""
    A = _u32(A)
    M = np.array(A, dtype=np.uint32, copy=True)
    m, n = M.shape
    rowperm = np.zeros(m, np.int32)
    colperm = np.zeros(n, np.int32)
    r = _load().oracle_lqup(m, n, p, _ptr(M), _ld(M) if m else max(n, 1), _ptr(rowperm), _ptr(colperm))
    if r < 0:
        raise ValueError("oracle_lqup failed (%d)" % r)
    return M, int(r), rowperm, colperm


def rank(A, p: int) -> int:
    """Rank of A mod p (p prime), by column echelon form."""
    A = np.ascontiguousarray(_u32(A))
    m, n = A.shape
    r = _load().oracle_rank(m, n, p, _ptr(A), max(n, 1))
    if r < 0:
        raise ValueError("oracle_rank failed (%d)" % r)
    return int(r)


def det(A, p: int) -> int:
    """Determinant of the square matrix A mod p (p prime), by Gaussian elimination."""
    A = np.ascontiguousarray(_u32(A))
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("det needs a square matrix")
    out = np.zeros(1, np.uint32)
    rc = _load().oracle_det(n, p, _ptr(A), max(n, 1), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_det failed (%d)" % rc)
    return int(out[0])


def inverse(A, p: int):
    """A^{-1} mod p (p prime) by Gauss-Jordan elimination, or None if A is singular."""
    A = np.ascontiguousarray(_u32(A))
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("inverse needs a square matrix")
    X = np.zeros((n, n), np.uint32)
    rc = _load().oracle_inverse(n, p, _ptr(A), max(n, 1), _ptr(X), max(n, 1))
    if rc == 1:
        return None
    if rc != 0:
        raise ValueError("oracle_inverse failed (%d)" % rc)
    return X
