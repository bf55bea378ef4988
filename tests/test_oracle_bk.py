"""Pins of the oracle's restricted Bunch-Kaufman LDL^T."""
import numpy as np
import pytest
import scipy.linalg

from oracle import bk


def _sym(n, rng, scale_diag=1.0):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.T
    A[np.diag_indices(n)] *= scale_diag
    return A


def _reconstruct(F, p):
    perm, L, dbl, C, steps = bk.ldlt_restricted(F, p)
    D = bk.d_matrix(dbl, p)
    PF = F[np.ix_(perm, perm)]
    R = L @ D @ L.T
    R[p:, p:] += C
    return PF, R, perm, steps


@pytest.mark.parametrize("n,p", [(1, 1), (7, 7), (30, 30), (30, 11), (50, 50)])
def test_reconstruction(n, p):
    rng = np.random.default_rng(n + p)
    F = _sym(n, rng)
    PF, R, perm, _ = _reconstruct(F, p)
    assert np.abs(PF - R).max() < 1e-12 * np.abs(F).max()
    assert np.all(perm[p:] == np.arange(p, n))          # restricted: no row >= p moves


def test_zero_diagonal_forces_2x2():
    rng = np.random.default_rng(0)
    F = _sym(12, rng, scale_diag=0.0)
    PF, R, perm, steps = _reconstruct(F, 12)
    assert steps[0] == (0, 2)              # zero diagonal: a 1x1 pivot is impossible
    assert sum(s == 2 for _, s in steps) >= 1
    assert np.abs(PF - R).max() < 1e-12 * np.abs(F).max()


def test_swap_1x1_at_r():
    # |a00| small, column max at row 2, a22 large -> 1x1 pivot taken at r = 2
    F = np.array([[1e-3, 0.1, 1.0], [0.1, 1.0, 0.1], [1.0, 0.1, 5.0]], complex)
    PF, R, perm, steps = _reconstruct(F, 3)
    assert perm[0] == 2 and steps[0] == (0, 1)
    assert np.abs(PF - R).max() < 1e-14


def test_solve_matches_library():
    rng = np.random.default_rng(5)
    F = _sym(40, rng, scale_diag=0.1)
    b = rng.standard_normal((40, 3)) + 1j * rng.standard_normal((40, 3))
    perm, L, dbl, _, _ = bk.ldlt_restricted(F)
    x = bk.solve(perm, L, dbl, b)
    assert np.abs(x - np.linalg.solve(F, b)).max() < 1e-10 * np.abs(x).max()
    # scipy's complex-symmetric (hermitian=False) LDL^T solves the same system
    lu, d, sp_perm = scipy.linalg.ldl(F, hermitian=False)
    y = np.linalg.solve(lu @ d @ lu.T, b)
    assert np.abs(x - y).max() < 1e-9 * np.abs(x).max()


def test_schur_complement_is_library_schur():
    rng = np.random.default_rng(6)
    F = _sym(20, rng)
    p = 8
    _, _, _, C, _ = bk.ldlt_restricted(F, p)
    S = F[p:, p:] - F[p:, :p] @ np.linalg.solve(F[:p, :p], F[:p, p:])
    assert np.abs(C - S).max() < 1e-10 * np.abs(S).max()


def test_singular_detected():
    F = np.zeros((4, 4), complex)
    F[2, 2] = F[3, 3] = 1.0
    with pytest.raises(bk.SingularPivot):
        bk.ldlt_restricted(F, 2)
