"""Iterative refinement with a low-precision factorisation -- oracle, test only.

The library's mixed path (factors in complex64, residuals in fp64) refines
the solution of A x = f by

    plain IR:   r = f - A x (fp64),  d = M^{-1} r (low precision),  x += d

which converges while the preconditioned operator A M^{-1} stays close to the
identity.  When the conditioning times the factor precision approaches one,
plain refinement stalls; GMRES-based refinement (GMRES-IR) instead solves
each correction equation A d = r with flexible GMRES in fp64, right
preconditioned by the same low-precision factorisation, so the outer loop
keeps converging.  This module writes both out in plain fp64 NumPy for the
tests; it is the reference for a future GPU implementation of the refinement
step and imports nothing from the library.

    fgmres(apply_a, apply_m, b, ...)   flexible GMRES, right preconditioned
    plain_ir(apply_a, apply_m, b, ...) plain iterative refinement
    gmres_ir(apply_a, apply_m, b, ...) refinement with FGMRES corrections
    lowprec_lu(A)                      complex64 sparse LU of A as M^{-1}

Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
matrix; complex arithmetic with the Hermitian inner product (GMRES minimises
the 2-norm of the residual, whatever the symmetry of A).

Pins (tests/test_oracle_gmres_ir.py): unpreconditioned GMRES on small dense
systems against numpy.linalg.solve within n steps; monotone residual norms;
an exact preconditioner converging in one step; an ill-conditioned complex
symmetric system where plain refinement with a complex64 LU fails and
GMRES-IR reaches the fp64 target; the library's FEM operator on a tiny mesh.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def fgmres(apply_a, apply_m, b, x0=None, tol=1e-12, restart=50, maxit=200):
    """Flexible GMRES for A x = b with right preconditioning, x = x0 + Z y.

    apply_a(v) -> A v and apply_m(v) -> M^{-1} v act on 1-D complex arrays
    (apply_m may differ between calls: the preconditioned directions z_j are
    stored).  Stops when ||b - A x||_2 <= tol ||b||_2 or after maxit inner
    steps in total.  Returns (x, residual 2-norm history)."""
    b = np.asarray(b, np.complex128)
    n = b.size
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, np.complex128), [0.0]
    r = b - apply_a(x)
    beta = np.linalg.norm(r)
    hist = [beta]
    steps = 0
    while beta > tol * bnorm and steps < maxit:
        m = min(restart, maxit - steps)
        V = np.zeros((n, m + 1), np.complex128)
        Z = np.zeros((n, m), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k_done = 0
        for j in range(m):
            Z[:, j] = apply_m(V[:, j])
            w = apply_a(Z[:, j])
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = np.conj(a) / den, np.conj(c) / den
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k_done = j + 1
            steps += 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * bnorm or H[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done]) if k_done else np.zeros(0)
        x = x + Z[:, :k_done] @ y
        r = b - apply_a(x)
        beta = np.linalg.norm(r)
        hist.append(beta)
    return x, hist


def _inf_ratio(r, f):
    return np.abs(r).max(axis=0) / np.abs(f).max(axis=0)


def plain_ir(apply_a, apply_m, f, tol=1e-10, max_iter=20):
    """x_0 = M^{-1} f, then x += M^{-1}(f - A x) until max|r| / max|f| <= tol
    (the library's criterion).  Returns (x, residual history)."""
    f = np.asarray(f, np.complex128)
    x = apply_m(f).astype(np.complex128)
    hist = []
    for _ in range(max_iter + 1):
        r = f - apply_a(x)
        hist.append(float(_inf_ratio(r, f)))
        if hist[-1] <= tol or not np.isfinite(hist[-1]):
            break
        x = x + apply_m(r).astype(np.complex128)
    return x, hist


def gmres_ir(apply_a, apply_m, f, tol=1e-10, max_outer=10, inner_tol=1e-4, restart=30, maxit=60):
    """Iterative refinement whose correction equation A d = r is solved by
    fgmres (fp64, right preconditioned by apply_m) to the relative accuracy
    inner_tol.  Returns (x, outer residual history, inner steps per outer)."""
    f = np.asarray(f, np.complex128)
    x = apply_m(f).astype(np.complex128)
    hist, inner = [], []
    for _ in range(max_outer + 1):
        r = f - apply_a(x)
        hist.append(float(_inf_ratio(r, f)))
        if hist[-1] <= tol:
            break
        d, h = fgmres(apply_a, apply_m, r, tol=inner_tol, restart=restart, maxit=maxit)
        inner.append(len(h) - 1)
        x = x + d
    return x, hist, inner


def lowprec_lu(A):
    """M^{-1} from a sparse LU of A rounded to complex64, applied in complex64
    (the precision of the library's mixed factors)."""
    lu = spla.splu(sp.csc_matrix(A).astype(np.complex64))
    return lambda v: lu.solve(np.asarray(v).astype(np.complex64)).astype(np.complex128)
