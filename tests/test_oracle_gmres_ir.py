"""Pins of the refinement oracle (oracle/gmres_ir.py)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, gmres_ir as G
from paper_2002_05018_gb300 import workloads as W


def _csym(n, rng, cond=1.0):
    """Complex symmetric (not Hermitian) matrix with singular values spread
    over [1/cond, 1] (Takagi-like: A = U S U^T with U unitary)."""
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = np.geomspace(1.0, 1.0 / cond, n)
    return (Q * s) @ Q.T


def test_gmres_solves_small_dense_in_n_steps():
    rng = np.random.default_rng(1)
    for n in (1, 5, 17):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x, h = G.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, restart=n, maxit=n)
        ref = np.linalg.solve(A, b)
        assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
        inner = h[1:-1]  # residual norms inside the cycle (the last entry is recomputed)
        assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip([h[0]] + inner[:-1], inner))  # minimal residual


def test_exact_preconditioner_converges_in_one_step():
    rng = np.random.default_rng(2)
    A = _csym(30, rng, cond=1e6)
    b = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    Ainv = np.linalg.inv(A)
    x, h = G.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, tol=1e-10, restart=10, maxit=10)
    assert len(h) == 3  # initial, one inner step, the recomputed final residual
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_gmres_ir_where_plain_refinement_fails():
    """A complex symmetric system with condition number 1e9 and f = A x_true
    (so ||A|| ||x|| / ||f|| stays near 1 and the fp64 residual floor is far
    below the target): the complex64 LU (unit roundoff 6e-8) leaves A M^{-1}
    far from the identity, so plain refinement cannot reach 1e-10 while
    GMRES-IR does."""
    rng = np.random.default_rng(3)
    n = 80
    A = _csym(n, rng, cond=1e9)
    xt = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    f = A @ xt
    M = G.lowprec_lu(sp.csc_matrix(A))
    apply_a = lambda v: A @ v
    xp, hp = G.plain_ir(apply_a, M, f, tol=1e-10, max_iter=15)
    assert not hp[-1] <= 1e-10
    xg, hg, inner = G.gmres_ir(apply_a, M, f, tol=1e-10, max_outer=10, inner_tol=1e-6, maxit=80)
    assert hg[-1] <= 1e-10


def test_fem_operator_refinement():
    """The library's operator on a tiny lossy mesh: with a complex64 LU both
    refinements reach the 1e-10 criterion; GMRES-IR needs no more outer steps
    and both agree with the fp64 direct solution."""
    w = W.tiny(6, 5, 4, 2, 2, 1, seed=3, lossy=True)
    keep = fem.free_edges(w)
    A = fem.global_matrix(w)[keep][:, keep].tocsc()
    f = fem.rhs_planewave(w)[keep, 0]
    M = G.lowprec_lu(A)
    apply_a = lambda v: A @ v
    xp, hp = G.plain_ir(apply_a, M, f, tol=1e-10)
    xg, hg, _ = G.gmres_ir(apply_a, M, f, tol=1e-10)
    assert hp[-1] <= 1e-10 and hg[-1] <= 1e-10
    assert len(hg) <= len(hp)
    ref = spla.spsolve(A, f)
    for x in (xp, xg):
        assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()
