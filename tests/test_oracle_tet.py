"""Pins of the oracle's tetrahedral (Whitney) discretisation against closed
forms and invariants: the Whitney space holds every constant field and every
field with constant curl exactly, so their energies are known in closed form;
gradients lie in the kernel of the stiffness; quadrature rules integrate
monomials exactly up to their degree."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint, d3m, fem
from paper_2002_05018_gb300 import workloads as W


def _tet(nx=4, ny=3, nz=3, px=1, py=1, pz=1, seed=1, jitter=0.1, **kw):
    return W.tetrahedral(W.tiny(nx, ny, nz, px, py, pz, seed=seed, **kw), jitter, seed=seed + 10)


def _tangents(g):
    s0, s1 = g.edge_nodes()
    t = g.nodes[s1] - g.nodes[s0]
    return t / np.linalg.norm(t, axis=1)[:, None], 0.5 * (g.nodes[s0] + g.nodes[s1])


def test_monomials_on_reference_simplices():
    # int_T x^a y^b = a! b! / (a + b + 2)!  (unit right triangle)
    for deg, (pts, wts) in ((2, fem.tri_quadrature(2)), (5, fem.tri_quadrature(5))):
        assert np.isclose(wts.sum(), 1.0)
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                xy = pts[:, 1:]           # barycentrics (1 - x - y, x, y)
                q = 0.5 * np.sum(wts * xy[:, 0] ** a * xy[:, 1] ** b)
                exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                assert abs(q - exact) < 1e-15, (deg, a, b)
    # int_T x^a y^b z^c = a! b! c! / (a + b + c + 3)!  (unit right tetrahedron)
    pts, wts = fem.tet_quadrature()
    for a in range(3):
        for b in range(3 - a):
            for c in range(3 - a - b):
                q = np.sum(wts * pts[:, 1] ** a * pts[:, 2] ** b * pts[:, 3] ** c) / 6.0
                exact = (math.factorial(a) * math.factorial(b) * math.factorial(c)
                         / math.factorial(a + b + c + 3))
                assert abs(q - exact) < 1e-15, (a, b, c)


def test_six_tetrahedra_fill_the_cells():
    w = _tet()
    g = fem.Grid.of(w)
    vol = fem.tet_volumes(g)
    assert vol.min() > 0
    assert np.isclose(vol.sum(), w.lx * w.ly * w.lz, rtol=1e-13)
    # undistorted: each tetrahedron is 1/6 of its cell
    g0 = fem.Grid(2, 2, 1, 0.6, 0.4, 0.5, "tet")
    assert np.allclose(fem.tet_volumes(g0), 0.3 * 0.2 * 0.5 / 6.0, rtol=1e-13)
    # every cell edge appears in some tetrahedron or on some face; 19 distinct columns
    ce = g.cell_edges()
    assert ce.shape[1] == 19 and all(len(set(r)) == 19 for r in ce[:5])
    assert len(np.unique(ce)) == g.n_edges     # no orphan edges


def test_edge_counts_match_the_workload():
    w = _tet(5, 4, 3)
    g = fem.Grid.of(w)
    assert g.n_edges == w.n_edges
    n = (5 + 1) * (4 + 1) * (3 + 1)
    # Euler: V - E + F - T = 1 for a cell complex of a ball
    tets = 6 * w.n_cells
    faces = (4 * tets + _boundary_triangles(w)) // 2
    assert n - g.n_edges + faces - tets == 1


def _boundary_triangles(w):
    return 4 * (w.nx * w.ny + w.ny * w.nz + w.nx * w.nz)


def test_gradients_are_in_the_stiffness_kernel():
    g = fem.Grid.of(_tet(seed=2))
    S, M = fem.mass_stiffness(g)
    G = sp.diags(1.0 / fem.edge_lengths(g)) @ fem.discrete_gradient(g)  # line-average dofs
    assert abs(S @ G).max() < 1e-13 * abs(S).max()
    assert abs(M @ G).max() > 1e-3 * abs(M).max()   # the mass does not annihilate them


def test_constant_field_energy():
    w = _tet(seed=3)
    g = fem.Grid.of(w)
    S, M = fem.mass_stiffness(g)
    t, _ = _tangents(g)
    E0 = np.array([0.3, -0.7, 0.5])
    x = t @ E0
    assert np.isclose(x @ M @ x, w.lx * w.ly * w.lz * E0 @ E0, rtol=1e-13)
    assert abs(S @ x).max() < 1e-13 * abs(S).max()


def test_constant_curl_energy():
    w = _tet(seed=4)
    g = fem.Grid.of(w)
    S, _ = fem.mass_stiffness(g)
    t, mid = _tangents(g)
    B, r0 = np.array([0.2, 0.5, -0.4]), np.array([0.1, 0.2, 0.3])
    x = np.sum(np.cross(B, mid - r0) * t, 1)   # E = B x (r - r0): curl E = 2B
    assert np.isclose(x @ S @ x, w.lx * w.ly * w.lz * 4.0 * B @ B, rtol=1e-12)


def test_boundary_face_mass_of_a_constant_field():
    w = _tet(seed=5)
    g = fem.Grid.of(w)
    faces = [(a, s, cid, 1.0) for a, s, cid, _ in fem.abc_faces(g, 1.0)]
    r, c, v = fem.assemble(g, w.eps, 0.0, cells=np.zeros(0, np.int64), extra_faces=faces)
    T = sp.csr_matrix((v.real, (r, c)), shape=(g.n_edges, g.n_edges))
    t, _ = _tangents(g)
    E0 = np.array([0.4, 0.1, -0.8])
    x = t @ E0
    lx, ly, lz = w.lx, w.ly, w.lz
    exact = 2.0 * (ly * lz * (E0[1] ** 2 + E0[2] ** 2) + lx * lz * (E0[0] ** 2 + E0[2] ** 2)
                   + lx * ly * (E0[0] ** 2 + E0[1] ** 2))
    assert np.isclose(x @ T @ x, exact, rtol=1e-13)


def test_single_cell_spectrum():
    g = fem.Grid(1, 1, 1, 0.3, 0.2, 0.5, "tet")
    S, M = (a.toarray() for a in fem.mass_stiffness(g))
    ev = np.linalg.eigvalsh(S)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 7      # 8 nodes -> 7 gradients
    assert np.linalg.eigvalsh(M).min() > 0
    assert np.abs(S - S.T).max() == 0 and np.abs(M - M.T).max() < 1e-17


def test_planewave_convergence_homogeneous_box():
    """As for bricks: the discrete solution converges to the interpolant of
    E_inc, at least 2x per halving of h."""
    errs = []
    for n in (3, 6):
        w = W.tetrahedral(W.tiny(n, n, n, 1, 1, 1, seed=3, lossy=False, h=1.0 / n), 0.1, seed=8)
        w.eps[:] = 1.0
        f = fem.rhs_planewave(w)
        x = fem.solve_global(w, f)[:, 0]
        xi = fem.edge_interpolant(w, w.khat[0], w.pol[0])
        errs.append(np.linalg.norm(x - xi) / np.linalg.norm(xi))
    assert errs[0] < 0.5 and errs[1] < errs[0] / 2.0


def test_reciprocity_and_symmetry():
    w = _tet(4, 3, 3, nrhs=2, seed=6)
    A = fem.global_matrix(w)
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    f = fem.rhs_planewave(w)
    x = fem.solve_global(w, f)
    assert abs(x[:, 0] @ f[:, 1] - x[:, 1] @ f[:, 0]) < 1e-10 * abs(x[:, 0] @ f[:, 1])


@pytest.mark.parametrize("case", [dict(nx=4, ny=3, nz=3, px=2, py=2, pz=1),
                                  dict(nx=5, ny=4, nz=4, px=2, py=2, pz=2, jitter=True)])
@pytest.mark.parametrize("lm_weight", [0, 1])
def test_decomposed_equals_global(case, lm_weight):
    c = dict(case)
    jit = c.pop("jitter", False)
    w = _tet(c["nx"], c["ny"], c["nz"], c["px"], c["py"], c["pz"], seed=7, nrhs=2, jitter=0.1)
    if jit:
        w = W.tetrahedral(W.tiny(c["nx"], c["ny"], c["nz"], c["px"], c["py"], c["pz"], seed=5,
                                 nrhs=2, jitter=True), 0.1, seed=9)
    w.lm_weight = lm_weight
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    assert r["copy_mismatch"] < 1e-10 * np.abs(xg).max()
    xs = d3m.solve_primal_schur(w, f)
    assert np.abs(xs - xg).max() < 1e-10 * np.abs(xg).max()


def test_adjoint_matches_central_differences():
    w = _tet(3, 3, 2, nrhs=2, seed=21)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(0)
    probes = np.sort(rng.choice(w.n_edges, 6, replace=False))
    J, g = adjoint.gradient(w, f, probes)
    h = 1e-6
    for c in rng.choice(w.n_cells, 5, replace=False):
        e0 = w.eps.copy()
        w.eps = e0.copy(); w.eps[c] += h
        Jp = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0.copy(); w.eps[c] -= h
        Jm = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * max(abs(fd), 1e-3 * abs(g).max()), (c, fd, g[c])
