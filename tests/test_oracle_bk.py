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


def _scipy_pattern(F):
    """(perm, block sizes by first position, D) of LAPACK's complex-symmetric
    Bunch-Kaufman LDL^T (scipy.linalg.ldl, hermitian=False, lower): the same
    magnitude |Re| + |Im|, the same alpha and lowest-index ties."""
    lu, d, perm = scipy.linalg.ldl(F, lower=True, hermitian=False)
    n = F.shape[0]
    sizes = {}
    k = 0
    while k < n:
        if k + 1 < n and d[k + 1, k] != 0:
            sizes[k] = 2
            k += 2
        else:
            sizes[k] = 1
            k += 1
    return perm, sizes, d, lu


@pytest.mark.parametrize("n,seed,scale", [(12, 0, 1.0), (24, 1, 0.3), (40, 2, 0.1), (48, 3, 0.0),
                                          (60, 4, 0.05), (33, 5, 2.0)])
def test_pivot_sequence_matches_lapack(n, seed, scale):
    """Pivot sequence (1x1 / 2x2 pattern and the permutation) and D of the
    full (p = n) factorisation against LAPACK's Bunch-Kaufman on random complex
    symmetric matrices.  Below LAPACK's block size (64) it runs the unblocked
    algorithm, the same right-looking order of updates; Gaussian entries keep
    every decision far from a tie for these seeds."""
    rng = np.random.default_rng(100 + seed)
    F = _sym(n, rng, scale)
    perm, L, dbl, C, steps = bk.ldlt_restricted(F)
    sp_perm, sizes, d, lu = _scipy_pattern(F)
    assert {k: s for k, s in steps} == sizes
    assert np.array_equal(perm, sp_perm)
    D = bk.d_matrix(dbl, n)
    assert np.abs(D - d).max() < 1e-11 * np.abs(d).max()
    assert np.abs(L - lu[sp_perm]).max() < 1e-10 * max(1.0, np.abs(L).max())
    if scale < 0.2:
        assert any(s == 2 for _, s in steps)     # small diagonals force 2x2 pivots


def test_one_by_one_after_row_test():
    """|a_kk| < alpha*omega_1 but |a_kk|*omega_r >= alpha*omega_1^2: a 1x1
    pivot at k with no interchange (the middle Bunch-Kaufman test).  Without
    that test the step would become the 2x2 pivot (|a_rr| < alpha*omega_r)."""
    F = np.array([[0.5, 1.0, 0.0], [1.0, 0.1, 2.0], [0.0, 2.0, 1.0]], complex)
    # omega_1 = 1 (row 1), omega_r = 2; 0.5 < 0.64 * 1, 0.5 * 2 >= 0.64 * 1
    PF, R, perm, steps = _reconstruct(F, 3)
    assert steps[0] == (0, 1) and perm[0] == 0
    assert np.abs(PF - R).max() < 1e-14
    sp_perm, sizes, _, _ = _scipy_pattern(F)
    assert sizes[0] == 1 and sp_perm[0] == 0


def test_two_by_two_when_all_tests_fail():
    """|a_kk| small, |a_kk|*omega_r < alpha*omega_1^2 and |a_rr| < alpha*omega_r:
    a 2x2 pivot on (k, r) with r moved next to k."""
    F = np.array([[0.01, 0.2, 1.0], [0.2, 3.0, 0.1], [1.0, 0.1, 0.02]], complex)
    # omega_1 = 1 at r = 2; omega_r = 1 (row 0 of column 2); 0.01 * 1 < 0.64;
    # |a_22| = 0.02 < 0.64 * 1  ->  2x2 on (0, 2)
    PF, R, perm, steps = _reconstruct(F, 3)
    assert steps[0] == (0, 2) and list(perm[:2]) == [0, 2]
    assert np.abs(PF - R).max() < 1e-14
    sp_perm, sizes, _, _ = _scipy_pattern(F)
    assert sizes[0] == 2 and list(sp_perm[:2]) == [0, 2]
