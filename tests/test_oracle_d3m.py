"""Pins of the oracle's decomposed path (Eq. (1), Algorithm 1) and orderings."""
import numpy as np
import pytest

from oracle import d3m, decomp, fem, ordering
from paper_2002_05018_gb300 import workloads as W


CASES = [
    dict(nx=4, ny=2, nz=2, px=2, py=1, pz=1),           # one interface
    dict(nx=4, ny=4, nz=4, px=2, py=2, pz=2),           # cross-lines, 4-way copies
    dict(nx=6, ny=5, nz=4, px=3, py=2, pz=1, jitter=True),
]


@pytest.mark.parametrize("case", CASES)
def test_decomposed_equals_global(case):
    c = dict(case)
    jit = c.pop("jitter", False)
    w = W.tiny(c["nx"], c["ny"], c["nz"], c["px"], c["py"], c["pz"], seed=7, nrhs=2, jitter=jit)
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    assert r["copy_mismatch"] < 1e-10 * np.abs(xg).max()
    assert fem.rel_residual(w, r["x"], f).max() < 1e-12


def test_sum_of_subdomain_matrices_is_global():
    w = W.tiny(4, 4, 2, 2, 2, 1, seed=3)
    dec = decomp.decompose(w)
    A = fem.global_matrix(w).toarray()
    acc = np.zeros_like(A)
    for sd in dec.subs:
        acc[np.ix_(sd.edges, sd.edges)] += sd.A.toarray()
    assert np.abs(acc - A).max() < 1e-13 * np.abs(A).max()


def test_K_equals_bruteforce_dense():
    w = W.tiny(4, 4, 4, 2, 2, 2, seed=9)
    dec = decomp.decompose(w)
    kd, _ = d3m.domain_matrices(w, dec)
    K = d3m.assemble_K(dec, kd)
    Kb = np.zeros_like(K)
    for sd in dec.subs:
        D = decomp.D_matrix(dec, sd).toarray()
        Kb += D.T @ np.linalg.inv(sd.A.toarray()) @ D
    assert np.abs(K - Kb).max() < 1e-12 * np.abs(Kb).max()
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()


def test_block_ldlt_matches_dense_solve():
    w = W.tiny(6, 6, 4, 3, 2, 2, seed=11, nrhs=3)
    dec = decomp.decompose(w)
    kd, _ = d3m.domain_matrices(w, dec)
    K = d3m.assemble_K(dec, kd)
    pattern, parent = d3m.block_symbolic(dec)
    fac = d3m.block_ldlt(K, dec.block_lms, pattern)
    g = np.random.default_rng(0).standard_normal((K.shape[0], 3)) + 0j
    lam = d3m.block_solve(fac, dec.block_lms, g)
    assert np.abs(lam - np.linalg.solve(K, g)).max() < 1e-10 * np.abs(lam).max()


def test_lm_rule_full_rank_and_cross_lines():
    w = W.tiny(4, 4, 4, 2, 2, 2, seed=1)
    dec = decomp.decompose(w)
    # every copied edge with m copies gets m - 1 multipliers
    n_expected = sum(len(c) - 1 for c in dec.copies.values())
    assert len(dec.lm_edge) == n_expected
    assert max(len(c) for c in dec.copies.values()) == 4
    for e, a, b in zip(dec.lm_edge, dec.lm_plus, dec.lm_minus):
        assert a < b and decomp.face_adjacent(a, b, dec.parts)


def test_nested_dissection_is_a_partition_with_separators():
    w = W.make(1)
    dec = decomp.decompose(w, with_matrices=True)
    plan = ordering.build_plan(dec)
    # each (subdomain, edge) appears exactly once
    keys = set(zip(plan.m_sub.tolist(), plan.m_edge.tolist()))
    assert len(keys) == plan.n
    assert plan.n == sum(len(s.edges) for s in dec.subs) + len(dec.lm_edge)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic(plan, r, c)
    # ND property: two ND leaves of one subdomain never share a matrix entry
    sn_of = np.repeat(np.arange(len(plan.sn_start)), plan.sn_end - plan.sn_start)
    a, b = sn_of[r], sn_of[c]
    leaf = np.zeros(len(plan.sn_start), bool)
    leaf[plan.sn_kind == 0] = True
    leaf[plan.parent[plan.parent >= 0]] = False
    bad = leaf[a] & leaf[b] & (a != b)
    assert not bad.any()
    # parent follows children, the only root is the last block of K
    ids = np.arange(len(plan.parent))
    assert np.all((plan.parent > ids) | (plan.parent == -1))
    assert (plan.parent == -1).sum() == 1 and plan.parent[-1] == -1


def test_symbolic_matches_bruteforce_elimination():
    """Supernodal structure vs scalar elimination on a dense boolean matrix."""
    w = W.tiny(4, 3, 2, 2, 1, 1, seed=2)
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=8)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic(plan, r, c)
    n = plan.n
    G = np.zeros((n, n), bool)
    G[r, c] = True
    for v in range(n):                      # scalar elimination game
        nb = np.flatnonzero(G[v, v + 1:]) + v + 1
        G[np.ix_(nb, nb)] = True
    for s, (a, b) in enumerate(zip(plan.sn_start, plan.sn_end)):
        rows = np.flatnonzero(G[a:b, b:].any(axis=0)) + b
        assert np.array_equal(rows, plan.struct[s])


def test_config1_structure_numbers():
    w = W.make(1)
    dec = decomp.decompose(w)
    assert [len(s.edges) for s in dec.subs] == [1680] * 4
    assert len(dec.lm_edge) == 636 and len(dec.blocks) == 4


@pytest.mark.parametrize("alpha_scale", [1.0, 0.3, 4.0, 1.0 - 1.0j])
def test_interface_coefficient_does_not_change_the_solution(alpha_scale):
    """The interface loss/gain alpha T_f cancels between the two sides of every
    cut face, so the decomposed solution equals the global one for any alpha
    (here alpha = scale * jk); the multipliers and K do depend on it."""
    w = W.tiny(6, 5, 4, 3, 2, 1, seed=12, nrhs=2, jitter=True)
    w.alpha = alpha_scale * 1j * w.k
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    if alpha_scale != 1.0:
        w.alpha = None
        r1 = d3m.solve(w, f, return_all=True)
        assert np.abs(r1["lam"] - r["lam"]).max() > 1e-3 * np.abs(r1["lam"]).max()


@pytest.mark.parametrize("case", CASES)
def test_primal_schur_equals_global_and_d3m(case):
    """The primal substructuring route (interface edges as unknowns) and the
    multiplier route of Eq. (1) reach the same solution as the global solve."""
    c = dict(case)
    jit = c.pop("jitter", False)
    w = W.tiny(c["nx"], c["ny"], c["nz"], c["px"], c["py"], c["pz"], seed=5, nrhs=2, jitter=jit)
    f = fem.rhs_planewave(w)
    xs = d3m.solve_primal_schur(w, f)
    xg = fem.solve_global(w, f)
    xd = d3m.solve(w, f)
    assert np.abs(xs - xg).max() < 1e-10 * np.abs(xg).max()
    assert np.abs(xs - xd).max() < 1e-10 * np.abs(xg).max()


def test_multiplier_mass_closed_form():
    """T_lambda (the Galerkin reading of lambda = j +- e): symmetric positive
    definite, no coupling between y- and z-directed multipliers on an x cut
    plane, and on a single interface whose tangential edges all carry a
    multiplier, 1^T T_yy 1 = 1^T T_zz 1 = the face area (the basis functions
    of one direction sum to the unit vector on the face)."""
    w = W.tiny(6, 4, 4, 2, 1, 1, seed=3, nrhs=1)
    w.lm_weight = 1
    dec = decomp.decompose(w)
    T = dec.T_lambda.toarray()
    g = dec.grid
    assert np.array_equal(T, T.T)
    assert np.linalg.eigvalsh(T).min() > 0
    ey = [l for l, e in enumerate(dec.lm_edge) if g.nex <= e < g.nex + g.ney]
    ez = [l for l, e in enumerate(dec.lm_edge) if e >= g.nex + g.ney]
    assert len(ey) + len(ez) == len(dec.lm_edge)  # an x cut plane carries y and z edges only
    area = w.ly * w.lz
    assert abs(T[np.ix_(ey, ey)].sum() - area) < 1e-13 * area
    assert abs(T[np.ix_(ez, ez)].sum() - area) < 1e-13 * area
    assert np.abs(T[np.ix_(ey, ez)]).max() == 0.0


def test_multiplier_mass_is_block_diagonal():
    """Multipliers of different interface blocks are not coupled (cross-lines
    tie a copy to one face-adjacent neighbour only)."""
    w = W.tiny(4, 4, 4, 2, 2, 2, seed=5, nrhs=1)
    w.lm_weight = 1
    dec = decomp.decompose(w)
    blk = np.empty(len(dec.lm_edge), int)
    for b, ids in enumerate(dec.block_lms):
        blk[ids] = b
    T = dec.T_lambda.tocoo()
    assert np.all(blk[T.row] == blk[T.col])
    for ids in dec.block_lms:  # every block's own mass is positive definite
        Tb = dec.T_lambda[ids][:, ids].toarray()
        assert np.linalg.eigvalsh(Tb).min() > 0


@pytest.mark.parametrize("case", CASES)
def test_mass_weighted_multipliers_leave_the_solution(case):
    """D = D_bool T_lambda differs from the Boolean map by an invertible
    congruence per block: the decomposed solution still equals the global
    one, and the multipliers satisfy T_lambda lambda_1 = lambda_0."""
    c = dict(case)
    jit = c.pop("jitter", False)
    w = W.tiny(c["nx"], c["ny"], c["nz"], c["px"], c["py"], c["pz"], seed=5, nrhs=2, jitter=jit)
    f = fem.rhs_planewave(w)
    xg = fem.solve_global(w, f)
    r0 = d3m.solve(w, f, return_all=True)
    w.lm_weight = 1
    r1 = d3m.solve(w, f, return_all=True)
    assert np.abs(r1["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    T = r1["dec"].T_lambda
    assert np.abs(T @ r1["lam"] - r0["lam"]).max() < 1e-10 * np.abs(r0["lam"]).max()
    assert np.abs(r1["lam"] - r0["lam"]).max() > 1e-3 * np.abs(r0["lam"]).max()
