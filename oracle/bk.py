"""Dense Bunch-Kaufman LDL^T restricted to a pivot block -- oracle, test only.

The paper factors K with "block restricted" Bunch-Kaufman pivoting (ref. [6],
Bunch & Kaufman 1977; discussion preceding the main steps): the pivot search
never leaves the current diagonal block and no pivot is delayed.  For a front
F (m x m, complex symmetric, NOT Hermitian: transposes, never conjugates) whose
first p rows/columns form the pivot block this computes

    P F P^T = [L11; L21] D [L11; L21]^T + [[0, 0], [0, C]]

with P a permutation of the first p indices only, L11 unit lower triangular,
D block diagonal with 1x1 and 2x2 blocks, and C the Schur complement on the
last m - p indices.  Magnitudes are |Re| + |Im|; alpha = (1 + sqrt 17) / 8;
ties go to the lowest index; a zero column in the pivot block raises
SingularPivot (never skipped).  Unblocked right-looking elimination, one pivot
step at a time.

Pins (tests/test_oracle_bk.py): reconstruction, agreement of solves with
numpy.linalg.solve and with scipy.linalg.ldl, a matrix with zero diagonal that
must take 2x2 pivots, the 1x1-at-r swap case, singular detection.
"""
from __future__ import annotations

import math

import numpy as np

ALPHA = (1.0 + math.sqrt(17.0)) / 8.0


class SingularPivot(ArithmeticError):
    pass


def cabs1(z):
    return np.abs(np.real(z)) + np.abs(np.imag(z))


def ldlt_restricted(F, p=None):
    """Returns (perm, L, dblocks, C, steps).  perm[i] = original index at
    pivot position i; L is m x p; dblocks[k] = (size, D block) keyed by its
    first position; steps = list of (k, size)."""
    A = np.array(F, dtype=np.complex128, copy=True)
    m = A.shape[0]
    p = m if p is None else p
    perm = np.arange(m)
    L = np.zeros((m, p), np.complex128)
    dblocks = {}
    steps = []
    k = 0
    while k < p:
        absakk = cabs1(A[k, k])
        if k + 1 < p:
            cand = cabs1(A[k + 1:p, k])
            imax = k + 1 + int(np.argmax(cand))
            colmax = float(cand.max())
        else:
            imax, colmax = k, 0.0
        if max(absakk, colmax) == 0.0:
            raise SingularPivot(f"zero pivot column at {k}")
        if absakk >= ALPHA * colmax:
            kp, step = k, 1
        else:
            row = cabs1(A[k:p, imax]).copy()
            row[imax - k] = 0.0
            rowmax = float(row.max())
            if absakk * rowmax >= ALPHA * colmax * colmax:
                kp, step = k, 1
            elif cabs1(A[imax, imax]) >= ALPHA * rowmax:
                kp, step = imax, 1
            else:
                kp, step = imax, 2
        kk = k + step - 1
        if kp != kk:
            A[[kk, kp], :] = A[[kp, kk], :]
            A[:, [kk, kp]] = A[:, [kp, kk]]
            L[[kk, kp], :] = L[[kp, kk], :]
            perm[[kk, kp]] = perm[[kp, kk]]
        if step == 1:
            d = A[k, k]
            l = A[k + 1:, k] / d
            A[k + 1:, k + 1:] -= np.outer(l, A[k + 1:, k])
            L[k, k] = 1.0
            L[k + 1:, k] = l
            dblocks[k] = (1, np.array([[d]]))
        else:
            D = A[k:k + 2, k:k + 2].copy()
            Lb = A[k + 2:, k:k + 2] @ np.linalg.inv(D)
            A[k + 2:, k + 2:] -= Lb @ A[k + 2:, k:k + 2].T
            L[k:k + 2, k:k + 2] = np.eye(2)
            L[k + 2:, k:k + 2] = Lb
            dblocks[k] = (2, D)
        A[k:, k:k + step] = 0.0
        A[k:k + step, k:] = 0.0
        steps.append((k, step))
        k += step
    C = A[p:, p:].copy()
    return perm, L, dblocks, C, steps


def d_matrix(dblocks, p):
    D = np.zeros((p, p), np.complex128)
    for k, (s, blk) in dblocks.items():
        D[k:k + s, k:k + s] = blk
    return D


def solve(perm, L, dblocks, b):
    """x = F^{-1} b for a full factorisation (p = m)."""
    m = L.shape[0]
    y = np.array(b, dtype=np.complex128)[perm]
    for k in range(m):                       # forward, unit lower
        y[k + 1:] -= np.outer(L[k + 1:, k], y[k]) if y.ndim > 1 else L[k + 1:, k] * y[k]
    z = np.zeros_like(y)
    for k, (s, blk) in dblocks.items():      # block diagonal
        z[k:k + s] = np.linalg.solve(blk, y[k:k + s])
    for k in range(m - 1, -1, -1):           # backward, unit upper L^T
        z[k] -= L[k + 1:, k] @ z[k + 1:]
    x = np.zeros_like(z)
    x[perm] = z
    return x
