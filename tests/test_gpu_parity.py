"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: relative solution error <= 1e-10 for the fp64 path and <= 1e-8
for the mixed path after refinement; relative residual
||A x - f||_inf / ||f||_inf <= 1e-12 (fp64) and <= 1e-10 (mixed) with A
assembled by the oracle (independent of the library's own operator)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bk, d3m as od3m, fem  # noqa: E402
from paper_2002_05018_gb300 import d3m, workloads as W  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sym(n, rng, diag_scale=1.0):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.T
    A[np.diag_indices(n)] *= diag_scale
    return A


def _factors(G, dv, p):
    L = np.tril(G[:, :p], -1)
    L[np.arange(p), np.arange(p)] = 1.0
    D = np.zeros((p, p), complex)
    k = 0
    while k < p:
        code = int(dv[k, 4])
        if code == 1:
            D[k, k] = 1.0 / (dv[k, 0] + 1j * dv[k, 1])
            k += 1
        else:
            assert code == 2
            Di = np.array([[dv[k, 0] + 1j * dv[k, 1], dv[k, 2] + 1j * dv[k, 3]],
                           [dv[k, 2] + 1j * dv[k, 3], dv[k + 1, 0] + 1j * dv[k + 1, 1]]])
            D[k:k + 2, k:k + 2] = np.linalg.inv(Di)
            assert L[k + 1, k] == 0
            k += 2
    return L, D


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("m,p,scale", [(600, 600, 0.2), (1000, 500, 1.0), (2000, 300, 0.0), (4000, 200, 0.5)])
def test_dense_front_kernel_large(m, p, scale, kernel):
    """Large fronts (cluster sizes 2..16 for the cluster panel): reconstruction
    checked on random vectors, Schur complement against the library-free formula."""
    _need_gpu()
    rng = np.random.default_rng(m + p)
    F = _sym(m, rng, scale)
    A = torch.tensor(np.ascontiguousarray(F.T[None]), device="cuda")
    A, perm, dinv, info = d3m.dense_ldlt(A, p, panel_kernel=kernel)
    torch.cuda.synchronize()
    assert info.item() == 0
    G = A.cpu().numpy()[0].T
    pv = perm.cpu().numpy()[0]
    L, D = _factors(G, dinv.cpu().numpy()[0], p)
    PF = F[np.ix_(pv, pv)]
    X = rng.standard_normal((m, 3)) + 1j * rng.standard_normal((m, 3))
    C = np.tril(G[p:, p:])
    C = C + np.tril(C, -1).T
    lhs = PF @ X
    rhs = L @ (D @ (L.T @ X))
    rhs[p:] += C @ X[p:]
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()
    if p < m:
        Cs = F[p:, p:] - F[p:, :p] @ np.linalg.solve(F[:p, :p], F[:p, p:])
        assert np.abs(C - Cs).max() < 1e-9 * np.abs(Cs).max()


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("m,p,scale", [(1, 1, 1.0), (40, 40, 1.0), (100, 37, 1.0), (257, 129, 0.05),
                                       (300, 300, 0.0), (130, 64, 0.0)])
def test_dense_front_kernel(m, p, scale, kernel):
    """Restricted Bunch-Kaufman partial LDL^T of dense fronts: reconstruction
    and the Schur complement (unique) against the oracle."""
    _need_gpu()
    rng = np.random.default_rng(m * 7 + p)
    mats = [_sym(m, rng, scale) for _ in range(3)]
    # column-major per matrix: element (i, j) at [b, j, i]
    A = torch.tensor(np.ascontiguousarray(np.stack([M.T for M in mats])), device="cuda")
    A, perm, dinv, info = d3m.dense_ldlt(A, p, panel_kernel=kernel)
    torch.cuda.synchronize()
    out = A.cpu().numpy()
    perm = perm.cpu().numpy()
    dv = dinv.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for b, F in enumerate(mats):
        G = out[b].T                       # back to row-major (i, j)
        pv = perm[b]
        assert sorted(pv[:p]) == list(range(p)) and np.all(pv[p:] == np.arange(p, m))
        L = np.tril(G[:, :p], -1)
        L[np.arange(p), np.arange(p)] = 1.0
        D = np.zeros((p, p), complex)
        k = 0
        while k < p:
            code = int(dv[b, k, 4])
            if code == 1:
                D[k, k] = 1.0 / (dv[b, k, 0] + 1j * dv[b, k, 1])
                k += 1
            else:
                assert code == 2
                Di = np.array([[dv[b, k, 0] + 1j * dv[b, k, 1], dv[b, k, 2] + 1j * dv[b, k, 3]],
                               [dv[b, k, 2] + 1j * dv[b, k, 3], dv[b, k + 1, 0] + 1j * dv[b, k + 1, 1]]])
                D[k:k + 2, k:k + 2] = np.linalg.inv(Di)
                L[k + 1, k] = 0.0
                k += 2
        R = L @ D @ L.T
        C = np.tril(G[p:, p:])
        R[p:, p:] += C + np.tril(C, -1).T
        PF = F[np.ix_(pv, pv)]
        assert np.abs(PF - R).max() < 1e-11 * np.abs(F).max()
        _, _, _, Co, _ = bk.ldlt_restricted(F, p)
        if p < m:
            assert np.abs(np.tril(C - Co)).max() < 1e-10 * max(1.0, np.abs(Co).max())


def _solve_case(w, precision, f=None, **kw):
    s = d3m.Solver.from_workload(w, precision=precision, **kw)
    s.factor()
    f = fem.rhs_planewave(w) if f is None else f
    rhs = torch.tensor(np.asfortranarray(f).T.copy(), device="cuda").t()
    x, info = s.solve(rhs)
    return s, x.cpu().numpy(), info, f


TINY = [
    lambda: W.tiny(4, 4, 4, 2, 2, 2, seed=1, nrhs=2),
    lambda: W.tiny(9, 7, 5, 3, 2, 2, seed=4, jitter=True, nrhs=3),
    lambda: W.tiny(6, 6, 6, 1, 1, 1, seed=2),            # no interface at all
    lambda: W.tiny(10, 4, 4, 5, 1, 1, seed=3, nrhs=2),   # a chain of subdomains
]


@pytest.mark.parametrize("mk", TINY)
@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_tiny_meshes(mk, precision):
    _need_gpu()
    w = mk()
    s, x, info, f = _solve_case(w, precision)
    _check_tiny(w, x, f, precision)


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_global_panel_variant(precision):
    _need_gpu()
    w = TINY[1]()
    s = d3m.Solver.from_workload(w, precision=precision, panel_kernel=1)
    s.factor()
    f = fem.rhs_planewave(w)
    x, info = s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    _check_tiny(w, x.cpu().numpy(), f, precision)


def _check_tiny(w, x, f, precision):
    xg = fem.solve_global(w, f)
    err = np.abs(x - xg).max() / np.abs(xg).max()
    tol = 1e-10 if precision == d3m.FP64 else 1e-8
    assert err < tol
    assert fem.rel_residual(w, x, f).max() < (1e-12 if precision == d3m.FP64 else 1e-10)


def test_pec_plate_on_cut_plane():
    _need_gpu()
    w = W.tiny(8, 8, 6, 2, 2, 2, seed=5, nrhs=2)
    w.pec_edge = W.pec_plate_mask(8, 8, 6, 2, 6, 2, 6, 3)
    s, x, info, f = _solve_case(w, d3m.FP64)
    xg = fem.solve_global(w, f)
    assert np.abs(x - xg).max() < 1e-10 * np.abs(xg).max()
    assert np.all(x[w.pec_edge == 1] == 0)


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_config1_against_oracle(precision):
    _need_gpu()
    w = W.make(1)
    s, x, info, f = _solve_case(w, precision)
    ref = od3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    tol = 1e-10 if precision == d3m.FP64 else 1e-8
    assert np.abs(x - xg).max() < tol * np.abs(xg).max()
    assert np.abs(x - ref["x"]).max() < tol * np.abs(xg).max()
    # multipliers: fp64 path to the solution tolerance; the mixed path refines
    # the primal residual only, so its multipliers keep the factor precision
    lam = s.lam(f.shape[1])
    ltol = 1e-9 if precision == d3m.FP64 else 1e-4
    assert np.abs(lam - ref["lam"]).max() < ltol * np.abs(ref["lam"]).max()
    assert info["max_resid"] < (1e-12 if precision == d3m.FP64 else 1e-10)


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_mass_weighted_multipliers(precision):
    """lm_weight = 1 (the Galerkin multiplier map D = D_bool T_lambda): the
    GPU solution still equals the global solve, and the multipliers equal the
    oracle's for the weighted map (a partition with cross-lines)."""
    _need_gpu()
    w = W.tiny(6, 6, 4, 2, 2, 1, seed=4, nrhs=3)
    w.lm_weight = 1
    s, x, info, f = _solve_case(w, precision)
    ref = od3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    tol = 1e-10 if precision == d3m.FP64 else 1e-8
    assert np.abs(x - xg).max() < tol * np.abs(xg).max()
    lam = s.lam(f.shape[1])
    ltol = 1e-9 if precision == d3m.FP64 else 1e-4
    assert np.abs(lam - ref["lam"]).max() < ltol * np.abs(ref["lam"]).max()


TET = [
    lambda: W.tetrahedral(W.tiny(4, 4, 4, 2, 2, 2, seed=1, nrhs=2), 0.1, seed=2),
    lambda: W.tetrahedral(W.tiny(7, 6, 5, 3, 2, 2, seed=4, jitter=True, nrhs=3), 0.1),
    lambda: W.tetrahedral(W.tiny(8, 3, 3, 4, 1, 1, seed=3, nrhs=2), 0.15),   # a chain
]


@pytest.mark.parametrize("mk", TET)
@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_tetrahedral_meshes(mk, precision):
    """Six Whitney tetrahedra per cell on jittered vertices: the GPU solution
    equals the oracle's global solve element by element and its multipliers
    equal the oracle's D3M multipliers."""
    _need_gpu()
    w = mk()
    s, x, info, f = _solve_case(w, precision)
    _check_tiny(w, x, f, precision)
    ref = od3m.solve(w, f, return_all=True)
    lam = s.lam(f.shape[1])
    ltol = 1e-9 if precision == d3m.FP64 else 1e-4
    assert np.abs(lam - ref["lam"]).max() < ltol * np.abs(ref["lam"]).max()
    s.close()


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_tetrahedral_uneven_partition(precision):
    """A 14x12x12-cell box on six jittered tetrahedra per cell (15,590
    edges), jittered uneven 3x2x2 cuts, per-cell eps, against the oracle's
    global solve element by element (the 20^3 tetrahedral mesh takes the
    oracle's sparse LU minutes, so this is the largest tetrahedral case
    checked element by element)."""
    _need_gpu()
    w = W.tetrahedral(W.tiny(14, 12, 12, 3, 2, 2, seed=3, nrhs=2, jitter=True), 0.1)
    s, x, info, f = _solve_case(w, precision)
    xg = fem.solve_global(w, f)
    tol = 1e-10 if precision == d3m.FP64 else 1e-8
    assert np.abs(x - xg).max() < tol * np.abs(xg).max()
    assert fem.rel_residual(w, x, f).max() < (1e-12 if precision == d3m.FP64 else 1e-10)
    s.close()


MESH = [
    lambda: W.delaunay(5, 4, 4, 2, 2, 2, seed=3, nrhs=2),
    lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6, nrhs=2),
    # complete first order (two dofs per edge)
    lambda: W.delaunay(5, 4, 4, 2, 2, 2, seed=3, nrhs=2, order=2),
    lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6, nrhs=2, order=2),
]


@pytest.mark.parametrize("mk", MESH)
@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_general_tetrahedral_meshes(mk, precision):
    """Delaunay meshes (arbitrary connectivity, subdomains by centroid, blocks
    between grid-diagonal subdomains), Whitney and complete first-order
    functions: E against the oracle's global solve element by element, lambda
    against the oracle's D3M multipliers."""
    _need_gpu()
    w = mk()
    s, x, info, f = _solve_case(w, precision)
    _check_tiny(w, x, f, precision)
    ref = od3m.solve(w, f, return_all=True)
    lam = s.lam(f.shape[1])
    ltol = 1e-9 if precision == d3m.FP64 else 1e-4
    assert np.abs(lam - ref["lam"]).max() < ltol * np.abs(ref["lam"]).max()
    s.close()


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_curl_complete_second_order_mesh(precision):
    """order 3 (two dofs per edge and two per face) on a Delaunay mesh with
    2x2x2 coordinate boxes: E against the oracle's global solve element by
    element in both precisions; lambda against the oracle's multipliers in
    FP64 (the mixed path's multipliers keep the factor precision, estimated at
    2-3e-5 on CPU for this order)."""
    _need_gpu()
    w = W.delaunay(5, 4, 4, 2, 2, 2, seed=3, nrhs=2, order=3)
    s, x, info, f = _solve_case(w, precision)
    _check_tiny(w, x, f, precision)
    if precision == d3m.FP64:
        ref = od3m.solve(w, f, return_all=True)
        lam = s.lam(f.shape[1])
        assert np.abs(lam - ref["lam"]).max() < 1e-9 * np.abs(ref["lam"]).max()
    s.close()


def test_lattice_mesh_through_the_general_path():
    """A lattice-tetrahedral workload through D3M_TET and, as vertex and
    tetrahedron lists, through D3M_TET_MESH: the same solution edge for edge
    (different numberings, orderings and assemblies)."""
    _need_gpu()
    wt = W.tetrahedral(W.tiny(6, 5, 4, 2, 2, 1, seed=1, nrhs=2), 0.1)
    wm = W.as_mesh(wt)
    _, xt, _, ft = _solve_case(wt, d3m.FP64)
    _, xm, _, fm = _solve_case(wm, d3m.FP64)
    g = fem.Grid.of(wt)
    s0, s1 = g.edge_nodes()
    from oracle import tetmesh
    ids = tetmesh.grid_of(wm).edge_id(s0, s1)
    assert np.abs(xm[ids] - xt).max() < 1e-10 * np.abs(xt).max()


def test_config3_fp64():
    _need_gpu()
    w = W.make(3)
    s, x, info, f = _solve_case(w, d3m.FP64)
    xg = fem.solve_global(w, f)
    assert np.abs(x - xg).max() < 1e-10 * np.abs(xg).max()


def _golden(cfg):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"x_samples_config{cfg}.npz")
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run tests/golden/make_full_size_samples.py {cfg}")
    return dict(np.load(path))


def _check_against_golden(w, g, x, f, tol):
    """Element-wise check of x at the stored sample rows against the oracle's
    solution (relative to the oracle column's max |x|), after checking that
    the library's RHS equals the oracle's at those rows."""
    cols, rows = g["columns"], g["rows"]
    assert np.abs(f[np.ix_(rows, cols)] - g["f"]).max() < 1e-12 * g["fmax"].max()
    err = np.abs(x[np.ix_(rows, cols)] - g["x"]) / g["xmax"][None, :]
    assert err.max() < tol, err.max()


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_config2_full_size(precision):
    """Full-size 32^3 / 64-RHS workload in the bench configuration (the launch
    configuration bench.py times, default schedule): x element by element at
    2048 sampled rows of 8 of the 64 columns against the oracle's solution
    (tests/golden, written by the oracle alone), and the residual of the
    oracle's own assembled operator on 3 columns."""
    _need_gpu()
    w = W.make(2)
    g = _golden(2)
    s = d3m.Solver.from_workload(w, precision=precision)
    s.factor()
    f = s.rhs_planewave(w.khat_pol6())
    rhs = torch.tensor(f.T.copy(), device="cuda").t()
    x, info = s.solve(rhs)
    x = x.cpu().numpy()
    _check_against_golden(w, g, x, f, 1e-10 if precision == d3m.FP64 else 1e-8)
    cols = [0, 17, 63]
    fo = fem.rhs_planewave(w, which=cols)
    assert np.abs(f[:, cols] - fo).max() < 1e-12 * np.abs(fo).max()
    res = fem.rel_residual(w, x[:, cols], fo)
    assert res.max() < 1e-10
    assert info["max_resid"] < 1e-10
    s.close()


def test_config4_pec_plate_full_size():
    """Full-size 48x48x24 workload with a PEC plate on the mid-z node layer
    (8 plane waves), mixed precision with refinement: x element by element at
    2048 sampled rows of 4 of the 8 columns against the oracle's solution, the
    residual of the oracle's own assembled operator on the free edges, zero
    field on the removed (PEC) edges."""
    _need_gpu()
    w = W.make(4)
    g = _golden(4)
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED)
    s.factor()
    f = s.rhs_planewave(w.khat_pol6())
    x, info = s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    x = x.cpu().numpy()
    _check_against_golden(w, g, x, f, 1e-8)
    cols = [0, 7]
    fo = fem.rhs_planewave(w, which=cols)
    assert np.abs(f[:, cols] - fo).max() < 1e-12 * np.abs(fo).max()
    assert info["max_resid"] < 1e-10
    assert fem.rel_residual(w, x[:, cols], fo).max() < 1e-10
    pec = np.flatnonzero(w.pec_edge)
    assert pec.size > 0 and np.all(x[pec] == 0)
    s.close()


def test_config3_mixed():
    """The 20^3 per-cell-eps workload in mixed precision with refinement
    against the oracle's global solve (16 RHS would be the adjoint probes; one
    plane wave here)."""
    _need_gpu()
    w = W.make(3)
    s, x, info, f = _solve_case(w, d3m.MIXED)
    xg = fem.solve_global(w, f)
    assert np.abs(x - xg).max() < 1e-8 * np.abs(xg).max()
    assert info["max_resid"] < 1e-10
    s.close()


def test_config5_full_size_mixed():
    """The 64^3 workload (811k edges, 4x4x4 jittered subdomains, 128 plane
    waves in one batch), mixed precision with refinement: every column meets
    the residual criterion by the library's count, and 2 columns are checked
    with the oracle's own assembled operator and plane-wave RHS (the oracle's
    direct solvers cannot factor this size in a test's time, so x itself is
    not compared).  Peak device memory stays under 180 GB."""
    _need_gpu()
    w = W.make(5)
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED)
    s.factor()
    f = s.rhs_planewave(w.khat_pol6())
    rhs = torch.tensor(f.T.copy(), device="cuda").t()
    x, info = s.solve(rhs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 180e9
    assert info["max_resid"] < 1e-10 and len(info["resid"]) == 128
    cols = [0, 127]
    xs = x[:, cols].cpu().numpy()
    del x, rhs
    s.close()
    fo = fem.rhs_planewave(w, which=cols)
    assert np.abs(f[:, cols] - fo).max() < 1e-12 * np.abs(fo).max()
    assert fem.rel_residual(w, xs, fo).max() < 1e-10


@pytest.mark.parametrize("wk", [1, 3])
def test_tensor_core_update_matches_fp32_fma(wk):
    """The deferred tcgen05 products (BF16x3 split operands, update rows through
    the explicit L11^{-1}) against the right-looking fp32-FMA updates: the
    fronts of the two mixed factorisations agree to fp32 rounding amplified
    by the fronts' conditioning (5e-4 relative), and both solve."""
    _need_gpu()
    w = W.make(wk)
    solvers = []
    for uk in (2, 1):
        s = d3m.Solver.from_workload(w, precision=d3m.MIXED, update_kernel=uk)
        s.factor()
        solvers.append(s)
    rng = solvers[0].structure(d3m.SN_RANGE)
    worst = 0.0
    for q in range(0, len(rng), max(1, len(rng) // 40)):
        Fa, pa, _ = solvers[0].export_front(q)
        Fb, pb, _ = solvers[1].export_front(q)
        if not np.array_equal(pa, pb):
            continue  # a near-tie pivot may differ; the solve check below covers it
        La, Lb = np.tril(Fa), np.tril(Fb)
        worst = max(worst, np.abs(La - Lb).max() / max(np.abs(Lb).max(), 1e-30))
    assert worst < 5e-4
    f = fem.rhs_planewave(w)
    x, info = solvers[0].solve(torch.tensor(f.T.copy(), device="cuda").t())
    assert info["max_resid"] < 1e-10


@pytest.mark.gpu
@pytest.mark.parametrize("wk", ["config3", "tiny70"])
def test_tensor_core_substitution_matches_fp32_fma(wk):
    """The substitution products on the tensor cores (complex BF16x3, operands
    split in the kernel) against the fp32-FMA products on the same factors
    (fixed schedule, so both contexts factor bitwise alike): one unrefined pass
    agrees to fp32 rounding amplified by the factors' conditioning, both passes
    are equally far from the fp64 solution, and refinement takes both to the
    same tolerance in the same number of passes (give or take one)."""
    _need_gpu()
    # one right-hand side; 70 (two column tiles of 64, the second ragged)
    w = W.make(3) if wk == "config3" else W.tiny(14, 12, 10, 2, 2, 2, seed=5, nrhs=70)
    f = fem.rhs_planewave(w)
    b = torch.tensor(f.T.copy(), device="cuda").t()
    one, full = {}, {}
    for sk in (0, 1):
        s = d3m.Solver.from_workload(w, precision=d3m.MIXED, autotune=1, solve_kernel=sk, refine_tol=0.5)
        s.factor()
        x, info = s.solve(b)
        assert info["iters"] == 0
        one[sk] = x.cpu().numpy()
        s.close()
        s = d3m.Solver.from_workload(w, precision=d3m.MIXED, autotune=1, solve_kernel=sk)
        s.factor()
        x, info = s.solve(b)
        assert info["max_resid"] < 1e-10
        full[sk] = (x.cpu().numpy(), info["iters"])
        s.close()
    ref = full[1][0]
    scale = np.abs(ref).max()
    d01 = np.abs(one[0] - one[1]).max() / scale
    e0 = np.abs(one[0] - ref).max() / scale
    e1 = np.abs(one[1] - ref).max() / scale
    assert d01 < 1e-3
    assert e0 < 3 * e1 + 1e-6
    assert np.abs(full[0][0] - ref).max() / scale < 1e-8
    assert abs(full[0][1] - full[1][1]) <= 1


@pytest.mark.gpu
def test_autotuner_choices_and_cache(tmp_path):
    """The per-level autotuner: its schedule gives the same refined solution as
    the fixed fp32-FMA schedule, its choices round-trip through the cache file,
    a cache written for another problem is ignored, and autotune=1 skips it."""
    _need_gpu()
    w = W.make(1)
    f = fem.rhs_planewave(w)
    b = torch.tensor(f.T.copy(), device="cuda").t()
    cache = tmp_path / "tune.txt"
    a = d3m.Solver.from_workload(w, precision=d3m.MIXED, autotune_cache=cache)
    a.factor()
    sa = a.stats()
    nlev = sa["n_levels"]
    assert sa["ms_tuning"] > 0
    assert 0 <= sa["tuned_levels_tc"] <= nlev and 0 <= sa["tuned_levels_cs2"] <= nlev
    lines = cache.read_text().splitlines()
    assert len(lines) == nlev + 1 and lines[0].startswith("d3m-autotune-v1")
    xa, ia = a.solve(b)
    ref = d3m.Solver.from_workload(w, precision=d3m.MIXED, update_kernel=1, autotune=1)
    ref.factor()
    assert ref.stats()["ms_tuning"] == 0 and ref.stats()["tuned_levels_tc"] == 0
    xr, ir = ref.solve(b)
    assert ia["max_resid"] < 1e-10 and ir["max_resid"] < 1e-10
    rel = (xa - xr).abs().max().item() / xr.abs().max().item()
    assert rel < 1e-8
    # the second solver reads the cached schedule instead of tuning
    c2 = d3m.Solver.from_workload(w, precision=d3m.MIXED, autotune_cache=cache)
    c2.factor()
    s2 = c2.stats()
    assert s2["ms_tuning"] == 0
    assert (s2["tuned_levels_tc"], s2["tuned_levels_cs2"]) == (sa["tuned_levels_tc"], sa["tuned_levels_cs2"])
    x2, i2 = c2.solve(b)
    assert i2["max_resid"] < 1e-10
    # a cache whose signature does not match is ignored (and rewritten)
    cache.write_text("d3m-autotune-v1 nm=1 fronts=1 levels=1 prec=1 arena=1\n0 1 1\n")
    c3 = d3m.Solver.from_workload(w, precision=d3m.MIXED, autotune_cache=cache)
    c3.factor()
    assert c3.stats()["ms_tuning"] > 0
    assert cache.read_text().splitlines()[0] == lines[0]
    for s in (a, ref, c2, c3):
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,uk", [(d3m.MIXED, 1), (d3m.MIXED, 2), (d3m.FP64, 1)])
def test_lookahead_bitwise_identical(prec, uk):
    """The overlapped schedule (Schur-complement updates on a second stream)
    partitions every step's trailing update by columns and keeps the step
    order per entry, so its factors equal the sequential schedule's bit for
    bit."""
    _need_gpu()
    w = W.make(1)
    sv = []
    for la in (0, 1):
        s = d3m.Solver.from_workload(w, precision=prec, update_kernel=uk, autotune=1, lookahead=la)
        s.factor()
        sv.append(s)
    n = len(sv[0].structure(d3m.SN_RANGE))
    for q in range(n):
        Fa, pa, da = sv[0].export_front(q)
        Fb, pb, db = sv[1].export_front(q)
        assert np.array_equal(pa, pb) and np.array_equal(da, db), q
        assert np.array_equal(Fa, Fb), q
    f = fem.rhs_planewave(w)
    b = torch.tensor(f.T.copy(), device="cuda").t()
    xa, _ = sv[0].solve(b)
    xb, _ = sv[1].solve(b)
    assert torch.equal(xa, xb)
    for s in sv:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [d3m.MIXED, d3m.FP64])
def test_factor_graph_replay_bitwise(prec):
    """Unprofiled factorisations replay the launch sequence captured at their
    first call; the replay, the capture run and an eager profiled run give
    the same factors bit for bit."""
    _need_gpu()
    w = W.make(1)
    s = d3m.Solver.from_workload(w, precision=prec, autotune=1)
    n = len(s.structure(d3m.SN_RANGE))
    fronts = []
    for prof in (True, False, False):  # eager, capture + launch, replay
        s.set_profile(prof)
        s.factor()
        fronts.append([s.export_front(q) for q in range(0, n, max(1, n // 60))])
    for other in fronts[1:]:
        for (Fa, pa, da), (Fb, pb, db) in zip(fronts[0], other):
            assert np.array_equal(pa, pb) and np.array_equal(da, db) and np.array_equal(Fa, Fb)
    f = fem.rhs_planewave(w)
    x, info = s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    assert info["max_resid"] < 1e-10
    s.close()


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_interface_coefficient_sweep(precision):
    """E does not depend on the interface loss/gain coefficient alpha (the two
    sides of every cut face cancel): workload 1 with alpha = s jk for several
    s, and a complex alpha, against the oracle's global solution; the
    multipliers do change with alpha."""
    _need_gpu()
    w = W.make(1)
    f = fem.rhs_planewave(w)
    xg = fem.solve_global(w, f)
    tol = 1e-10 if precision == d3m.FP64 else 1e-8
    lams = []
    for a in (None, 0.3j * w.k, 4j * w.k, (1 - 1j) * w.k):
        w.alpha = a
        s, x, info, _ = _solve_case(w, precision, f=f)
        assert np.abs(x - xg).max() < tol * np.abs(xg).max(), a
        lams.append(s.lam(1))
        s.close()
    w.alpha = None
    assert np.abs(lams[1] - lams[0]).max() > 1e-3 * np.abs(lams[0]).max()
