"""Strassen-Winograd schedule over Z with intermediate-size tracking -- TEST INFRASTRUCTURE.

Restates section 3.2: Winograd's variant of Strassen's algorithm with the
schedule of Table 2 for C <- alpha*A*B + beta*C (3 temporaries X1, X2, X3),
l recursive levels, the classic product at the leaves, and dynamic peeling for
odd dimensions (appendix, "case of an arbitrary k").  All arithmetic is exact
over Z (numpy object arrays of Python ints) with no modular reduction, so that
the largest intermediate value can be compared with Theorem 3.1.

Reading of a garbled entry: Table 2 row 16 prints ``P4 = alpha*A12*T4 -
beta*C21``; the appendix defines P4 = A22 x (...), and only A22 makes the
schedule compute A*B, so row 16 is taken with A22.

Pins: tests/test_oracle_winograd.py (equality with numpy's exact product;
Theorem 3.1's bound reached exactly by the appendix's matrices A_l, B_l).
"""
from __future__ import annotations

import numpy as np


class Tracker:
    """Records the largest |value| of every intermediate matrix produced."""

    def __init__(self):
        self.max_abs = 0

    def see(self, x):
        if x.size:
            v = max(abs(int(x.max())), abs(int(x.min())))
            if v > self.max_abs:
                self.max_abs = v
        return x


def _classic(A, B, tr: Tracker):
    """Leaf product by the classic algorithm, tracking every partial dot product."""
    m, k = A.shape
    n = B.shape[1]
    acc = np.zeros((m, n), dtype=object)
    for t in range(k):
        acc = acc + np.outer(A[:, t], B[t, :])
        tr.see(acc)
    return acc


def _wino(A, B, C, alpha, beta, levels, tr: Tracker):
    """Return alpha*A*B + beta*C (exact), l = levels recursive Winograd levels."""
    m, k = A.shape
    n = B.shape[1]
    if levels == 0 or min(m, k, n) < 2:
        prod = _classic(A, B, tr)
        out = alpha * prod + (beta * C if C is not None else 0)
        return tr.see(np.asarray(out, dtype=object).reshape(m, n))
    m2, k2, n2 = m - m % 2, k - k % 2, n - n % 2
    if (m2, k2, n2) != (m, k, n):
        return _peel(A, B, C, alpha, beta, levels, tr)
    h, kh, w = m // 2, k // 2, n // 2
    A11, A12, A21, A22 = A[:h, :kh], A[:h, kh:], A[h:, :kh], A[h:, kh:]
    B11, B12, B21, B22 = B[:kh, :w], B[:kh, w:], B[kh:, :w], B[kh:, w:]
    if C is None:
        C = np.zeros((m, n), dtype=object)
        beta_eff = 0
    else:
        beta_eff = beta
    C = C.copy()
    C11, C12, C21, C22 = C[:h, :w], C[:h, w:], C[h:, :w], C[h:, w:]
    rec = lambda X, Y, Z, b: _wino(X, Y, Z, alpha, b, levels - 1, tr)
    see = tr.see
    # Table 2, in its order (rows 1..21); X1, X2, X3 are the temporaries.
    X1 = see(A21 + A22)                       # 1  S1
    X2 = see(B12 - B11)                       # 2  T1
    X3 = rec(X1, X2, None, 0)                 # 3  P5 = alpha S1 T1
    C22[...] = see(X3 + beta_eff * C22)       # 4  C22 = P5 + beta C22
    C12[...] = see(X3 + beta_eff * C12)       # 5  C12 = P5 + beta C12
    X1 = see(X1 - A11)                        # 6  S2 = S1 - A11
    X2 = see(B22 - X2)                        # 7  T2 = B22 - T1
    X3 = rec(A11, B11, None, 0)               # 8  P1 = alpha A11 B11
    C11[...] = see(X3 + beta_eff * C11)       # 9  C11 = P1 + beta C11
    X3 = rec(X1, X2, X3, 1)                   # 10 U2 = alpha S2 T2 + P1
    C11[...] = rec(A12, B21, C11.copy(), 1)   # 11 U1 = alpha A12 B21 + C11
    X1 = see(A12 - X1)                        # 12 S4 = A12 - S2
    X2 = see(X2 - B21)                        # 13 T4 = T2 - B21
    C12[...] = rec(X1, B22, C12.copy(), 1)    # 14 C12 = alpha S4 B22 + C12
    C12[...] = see(X3 + C12)                  # 15 U5 = U2 + C12
    C21[...] = rec(A22, X2, C21.copy(), -beta_eff)  # 16 P4 = alpha A22 T4 - beta C21
    X1 = see(A11 - A21)                       # 17 S3 = A11 - A21
    X2 = see(B22 - B12)                       # 18 T3 = B22 - B12
    X3 = rec(X1, X2, X3, 1)                   # 19 U3 = alpha S3 T3 + U2
    C22[...] = see(X3 + C22)                  # 20 U7 = U3 + C22
    C21[...] = see(X3 - C21)                  # 21 U6 = U3 - C21
    return C


def _peel(A, B, C, alpha, beta, levels, tr: Tracker):
    """Dynamic peeling: the even top-left block by Winograd, then the odd
    row / column / inner index by matrix-vector, vector-matrix and rank-1 updates."""
    m, k = A.shape
    n = B.shape[1]
    m2, k2, n2 = m - m % 2, k - k % 2, n - n % 2
    out = np.zeros((m, n), dtype=object) if C is None else C.copy()
    b = 0 if C is None else beta
    if m2 and n2 and k2:
        out[:m2, :n2] = _wino(A[:m2, :k2], B[:k2, :n2],
                              None if C is None else C[:m2, :n2], alpha, b, levels, tr)
    elif m2 and n2:
        out[:m2, :n2] = tr.see(b * out[:m2, :n2])
    if k2 < k and m2 and n2:       # rank-1 update with the odd inner index
        out[:m2, :n2] = tr.see(out[:m2, :n2] + alpha * np.outer(A[:m2, k2], B[k2, :n2]))
    if n2 < n:                     # odd last column: matrix-vector
        col = _classic(A[:m2, :], B[:, n2:], tr)
        out[:m2, n2:] = tr.see(alpha * col + b * out[:m2, n2:])
    if m2 < m:                     # odd last row: vector-matrix
        row = _classic(A[m2:, :], B, tr)
        out[m2:, :] = tr.see(alpha * row + b * out[m2:, :])
    return out


def winograd_fgemm_z(A, B, C=None, alpha: int = 1, beta: int = 0, levels: int = 1):
    """alpha*A*B + beta*C over Z with `levels` Winograd levels.
    Returns (result as object array, largest |intermediate|)."""
    A = np.asarray(A).astype(object)
    B = np.asarray(B).astype(object)
    C = None if C is None else np.asarray(C).astype(object)
    tr = Tracker()
    out = _wino(A, B, C, alpha, beta, levels, tr)
    return out, tr.max_abs


def optimal_matrices(l: int, mA: int, MA: int, mB: int, MB: int):
    """The appendix's matrices A_l, B_l of order 2^l that reach Theorem 3.1's
    bound: A_1 = [[mA, 0], [MA, MA]], B_1 = [[MB, mB], [0, MB]],
    A_{l+1} = [[bar(A_l), 0], [A_l, A_l]], B_{l+1} = [[B_l, bar(B_l)], [0, B_l]],
    bar(x) = M + m - x."""
    A = np.array([[mA, 0], [MA, MA]], dtype=object)
    B = np.array([[MB, mB], [0, MB]], dtype=object)
    for _ in range(l - 1):
        Ab = MA + mA - A
        Bb = MB + mB - B
        Z = np.zeros_like(A)
        A = np.block([[Ab, Z], [A, A]])
        B = np.block([[B, Bb], [Z, B]])
    return A, B
