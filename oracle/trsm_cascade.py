"""The double cascade of section 4.3 over Z with intermediate tracking -- TEST INFRASTRUCTURE.

Restates Algorithm 2 (trsm-rec-BLAS-delayed) and Algorithm 3
(trsm-partial-delayed) in the paper's orientation (A unit upper triangular,
A X = B, block columns [V_i; U_i; 0] taken from the last one back to the
first) with exact Python integers (numpy object arrays), so that the largest
value any step holds can be compared with the 63-bit carrier the GPU path
uses.  Residues are in the balanced (centred) representation, the one that
eq. (trsmboundcen) bounds.

Steps, in the paper's order:
  Algorithm 2: for each block column of t_split columns, from the last:
      X_i = trsm-partial-delayed(U_i, B_i); X_i = X_i mod p;
      B_{1..i-1} = B_{1..i-1} - V_i X_i; B_{1..i-1} = B_{1..i-1} mod p.
  Algorithm 3 (m rows):
      if m <= t_del: B = B mod p; X = the exact solution over Z (back
          substitution, the paper's dtrsm); X = X mod p.
      else: split into floor(m/2) and ceil(m/2) rows;
          X_2 = trsm-partial-delayed(A_3, B_2);
          B_1 = B_1 - A_2 X_2 without reduction;
          X_1 = trsm-partial-delayed(A_1, B_1).

Pins: tests/test_oracle_trsm_cascade.py (the result equals the plain
substitution of oracle.ftrsm; on the sign-chasing system of Corollary 4.3's
optimality argument a leaf of t_del rows reaches the growth bound exactly).
"""
from __future__ import annotations

import numpy as np


class Tracker:
    """Largest |value| held by any step."""

    def __init__(self):
        self.max_abs = 0

    def see(self, x):
        x = np.asarray(x, dtype=object)
        if x.size:
            v = max(abs(int(x.max())), abs(int(x.min())))
            self.max_abs = max(self.max_abs, v)
        return x


def balanced(x, p: int):
    """The balanced representative of x mod p, in (-p/2, p/2]."""
    x = np.asarray(x, dtype=object)
    r = x % p
    return np.where(r > p // 2, r - p, r).astype(object)


def _back_substitute(A, B, tr: Tracker):
    """X with A X = B over Z for unit upper triangular A (exact, no reduction)."""
    m = A.shape[0]
    X = np.zeros(B.shape, dtype=object)
    for i in range(m - 1, -1, -1):
        acc = B[i, :].copy()
        for j in range(i + 1, m):
            acc = tr.see(acc - A[i, j] * X[j, :])
        X[i, :] = acc
    return X


def trsm_partial_delayed(A, B, p: int, t_del: int, tr: Tracker):
    """Algorithm 3 for unit upper A (m x m) and B (m x n) over Z."""
    m = A.shape[0]
    if m <= t_del:
        Bp = balanced(B, p)
        X = _back_substitute(A, Bp, tr)
        return balanced(X, p)
    h = m // 2                                  # A1: floor(m/2) rows, A3: ceil(m/2)
    A1, A2, A3 = A[:h, :h], A[:h, h:], A[h:, h:]
    X2 = trsm_partial_delayed(A3, B[h:, :], p, t_del, tr)
    B1 = tr.see(B[:h, :] - A2.dot(X2))          # without modular reduction
    X1 = trsm_partial_delayed(A1, B1, p, t_del, tr)
    return np.vstack([X1, X2])


def trsm_rec_blas_delayed(A, B, p: int, t_del: int, t_split: int):
    """Algorithm 2 for unit upper A (m x m), B (m x n) mod p.
    Returns (X canonical in [0, p) as an object array, largest |intermediate|)."""
    tr = Tracker()
    A = balanced(A, p)
    B = balanced(B, p)
    m = A.shape[0]
    X = np.zeros(B.shape, dtype=object)
    r1 = m
    while r1 > 0:                               # block columns from the last one back
        r0 = max(0, r1 - t_split)
        U, V = A[r0:r1, r0:r1], A[:r0, r0:r1]
        Xi = trsm_partial_delayed(U, B[r0:r1, :], p, t_del, tr)
        Xi = balanced(Xi, p)
        X[r0:r1, :] = Xi
        if r0 > 0:
            upd = tr.see(B[:r0, :] - V.dot(Xi))
            B[:r0, :] = balanced(upd, p)
        r1 = r0
    return X % p, tr.max_abs
