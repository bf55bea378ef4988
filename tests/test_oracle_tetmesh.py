"""Pins of the oracle's general tetrahedral meshes (oracle/tetmesh.py): the
lattice-tetrahedral path and the general-mesh path are two independent
numberings and assemblies of the same discretisation; the Whitney energy
identities hold on an unstructured (Delaunay) mesh; D3M is exact there too,
including multiplier blocks between subdomains that touch only along an edge."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint, d3m, decomp, fem, ordering, tetmesh
from paper_2002_05018_gb300 import workloads as W


def _lattice_ids(wt, wm):
    g = fem.Grid.of(wt)
    s0, s1 = g.edge_nodes()
    gm = tetmesh.grid_of(wm)
    ids = gm.edge_id(np.minimum(s0, s1), np.maximum(s0, s1))
    assert np.array_equal(gm.edges[ids], np.stack([s0, s1], 1))   # same orientation too
    return ids


def test_lattice_mesh_equals_lattice_path():
    wt = W.tetrahedral(W.tiny(4, 3, 3, 2, 2, 1, seed=1, nrhs=2), 0.1)
    wm = W.as_mesh(wt)
    ids = _lattice_ids(wt, wm)
    assert wm.n_edges == wt.n_edges and len(np.unique(ids)) == len(ids)
    At, Am = fem.global_matrix(wt), fem.global_matrix(wm)
    assert abs(Am[ids][:, ids] - At).max() < 1e-13 * abs(At).max()
    ft, fm = fem.rhs_planewave(wt), fem.rhs_planewave(wm)
    assert np.abs(fm[ids] - ft).max() < 1e-13 * np.abs(ft).max()
    xt, xm = fem.solve_global(wt, ft), fem.solve_global(wm, fm)
    assert np.abs(xm[ids] - xt).max() < 1e-12 * np.abs(xt).max()
    # decomposed: the same multipliers (same blocks, the same edges in each;
    # inside a block they follow each numbering's own edge order)
    dt, dm = decomp.decompose(wt, False), decomp.decompose(wm, False)
    assert dt.blocks == dm.blocks
    for lt, lm in zip(dt.block_lms, dm.block_lms):
        assert np.array_equal(np.sort(ids[dt.lm_edge[lt]]), dm.lm_edge[lm])


def _delaunay(**kw):
    args = dict(nx=5, ny=4, nz=4, px=2, py=2, pz=2, seed=3, nrhs=2)
    args.update(kw)
    return W.delaunay(**args)


def _tangents(g):
    t = g.V[g.edges[:, 1]] - g.V[g.edges[:, 0]]
    return t / np.linalg.norm(t, axis=1)[:, None], 0.5 * (g.V[g.edges[:, 0]] + g.V[g.edges[:, 1]])


def test_energy_identities_on_an_unstructured_mesh():
    w = _delaunay()
    g = tetmesh.grid_of(w)
    V = w.lx * w.ly * w.lz
    X = g.V[g.T]
    vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6
    assert np.isclose(vol.sum(), V, rtol=1e-12)
    S, M = tetmesh.mass_stiffness(g)
    G = sp.diags(1.0 / tetmesh.edge_lengths(g)) @ tetmesh.discrete_gradient(g)
    assert abs(S @ G).max() < 1e-12 * abs(S).max()
    t, mid = _tangents(g)
    E0 = np.array([0.3, -0.7, 0.5])
    x = t @ E0
    assert np.isclose(x @ M @ x, V * E0 @ E0, rtol=1e-12)
    B, r0 = np.array([0.2, 0.5, -0.4]), np.array([0.1, 0.2, 0.3])
    xl = np.sum(np.cross(B, mid - r0) * t, 1)
    assert np.isclose(xl @ S @ xl, V * 4.0 * B @ B, rtol=1e-11)
    # boundary face mass of a constant field: sum of area |E0_t|^2 over the box faces
    bf = tetmesh.boundary_faces(g)
    r, c, v = tetmesh.assemble(g, w.eps, 0.0, tets=np.zeros(0, np.int64), faces=[(bf, 1.0)])
    T = sp.csr_matrix((v.real, (r, c)), shape=(g.n_edges, g.n_edges))
    lx, ly, lz = w.lx, w.ly, w.lz
    exact = 2.0 * (ly * lz * (E0[1] ** 2 + E0[2] ** 2) + lx * lz * (E0[0] ** 2 + E0[2] ** 2)
                   + lx * ly * (E0[0] ** 2 + E0[1] ** 2))
    assert np.isclose(x @ T @ x, exact, rtol=1e-12)
    # outward normals of the box faces are the axis directions
    n = tetmesh.outward_normals(g, bf)
    assert np.allclose(np.sort(np.abs(n), axis=1)[:, :2], 0.0, atol=1e-12)


def test_planewave_convergence_on_delaunay_meshes():
    errs = []
    for n in (3, 6):
        w = W.delaunay(n, n, n, 1, 1, 1, seed=4, lossy=False, h=1.0 / n)
        w.eps[:] = 1.0
        f = fem.rhs_planewave(w)
        x = fem.solve_global(w, f)[:, 0]
        xi = fem.edge_interpolant(w, w.khat[0], w.pol[0])
        errs.append(np.linalg.norm(x - xi) / np.linalg.norm(xi))
    assert errs[0] < 0.5 and errs[1] < errs[0] / 2.0


def test_reciprocity_and_symmetry():
    w = _delaunay(px=1, py=1, pz=1)
    A = fem.global_matrix(w)
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    f = fem.rhs_planewave(w)
    x = fem.solve_global(w, f)
    assert abs(x[:, 0] @ f[:, 1] - x[:, 1] @ f[:, 0]) < 1e-10 * abs(x[:, 0] @ f[:, 1])


@pytest.mark.parametrize("kw", [dict(), dict(nx=6, ny=5, nz=4, px=3, py=2, pz=1, seed=5)])
def test_decomposed_equals_global_on_delaunay_meshes(kw):
    w = _delaunay(**kw)
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    assert r["copy_mismatch"] < 1e-10 * np.abs(xg).max()
    xs = d3m.solve_primal_schur(w, f)
    assert np.abs(xs - xg).max() < 1e-10 * np.abs(xg).max()


def test_jagged_interfaces_tie_non_neighbour_copies():
    """On a Delaunay mesh some edge is shared by two subdomains that are not
    face neighbours in the grid (the fallback of the multiplier rule), and
    the block order still lists every block once."""
    w = _delaunay()
    dec = decomp.decompose(w, False)
    assert any(not decomp.face_adjacent(a, b, dec.parts) for a, b in dec.blocks)
    assert sorted(dec.blocks) == sorted(set(dec.blocks))


@pytest.mark.parametrize("order", [1, 3])
def test_mesh_nested_dissection_is_a_partition_with_separators(order):
    """The centroid bisection over edges (and, at order 3, faces): every dof
    in exactly one supernode, no two ND leaves of a subdomain coupled."""
    import dataclasses
    w = dataclasses.replace(_delaunay(nx=6, ny=6, nz=5, px=2, py=1, pz=1), order=order)
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=24)
    keys = set(zip(plan.m_sub.tolist(), plan.m_edge.tolist()))
    assert len(keys) == plan.n == sum(len(s.edges) for s in dec.subs) + len(dec.lm_edge)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic(plan, r, c)
    sn_of = np.repeat(np.arange(len(plan.sn_start)), plan.sn_end - plan.sn_start)
    a, b = sn_of[r], sn_of[c]
    leaf = np.zeros(len(plan.sn_start), bool)
    leaf[plan.sn_kind == 0] = True
    leaf[plan.parent[plan.parent >= 0]] = False
    assert leaf.sum() > 4
    assert not (leaf[a] & leaf[b] & (a != b)).any()
    ids = np.arange(len(plan.parent))
    assert np.all((plan.parent > ids) | (plan.parent == -1))


def test_adjoint_matches_central_differences():
    w = _delaunay(nx=3, ny=3, nz=2, px=1, py=1, pz=1, seed=21)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(0)
    probes = np.sort(rng.choice(w.n_edges, 6, replace=False))
    J, g = adjoint.gradient(w, f, probes)
    assert g.shape == (w.n_cells,)
    h = 1e-6
    for c in rng.choice(w.n_cells, 5, replace=False):
        e0 = w.eps.copy()
        w.eps = e0.copy(); w.eps[c] += h
        Jp = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0.copy(); w.eps[c] -= h
        Jm = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0
        fd = (Jp - Jm) / (2 * h)
        # 1e-5 relative, plus the rounding floor of a 1e-6 central difference
        # (about 1e-16 J / 1e-6) relative to the largest gradient entry: the
        # per-tetrahedron entries are small next to J
        assert abs(fd - g[c]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (c, fd, g[c], J)


# ------------------------------------------------------- complete first order


def _linear_field_dofs(g, a, C):
    """Dofs of E = a + C r: the line average of E . t and the coefficient of
    1 - 2 s / l (half the difference of E . t between the edge's ends)."""
    P0, P1 = g.V[g.edges[:, 0]], g.V[g.edges[:, 1]]
    t = (P1 - P0) / np.linalg.norm(P1 - P0, axis=1)[:, None]
    E0, E1 = a + P0 @ C.T, a + P1 @ C.T
    x = np.zeros(g.n_edges)
    x[0::2] = 0.5 * np.sum((E0 + E1) * t, 1)
    x[1::2] = 0.5 * np.sum((E0 - E1) * t, 1)
    return x


def test_order2_holds_every_linear_field():
    """The order-2 space contains every field a + C r: its energies are exact
    (the integral of |a + C r|^2 over the box by tensor Gauss-Legendre, exact
    for the quadratic integrand), the Whitney space alone does not."""
    w = W.delaunay(5, 4, 4, 1, 1, 1, seed=3, order=2)
    g = tetmesh.grid_of(w)
    assert g.n_edges == 2 * g.n_geo == w.n_edges
    S, M = tetmesh.mass_stiffness(g)
    a = np.array([0.3, -0.2, 0.5])
    C = np.array([[0.1, 0.4, -0.3], [0.2, -0.5, 0.6], [-0.7, 0.3, 0.2]])
    x = _linear_field_dofs(g, a, C)
    L = np.array([w.lx, w.ly, w.lz])
    q, wq = fem.gauss01(2)
    exact = 0.0
    for i, xi in enumerate(q):
        for j, yj in enumerate(q):
            for k, zk in enumerate(q):
                e = a + C @ (np.array([xi, yj, zk]) * L)
                exact += wq[i] * wq[j] * wq[k] * (e @ e)
    exact *= L.prod()
    assert np.isclose(x @ M @ x, exact, rtol=1e-12)
    curl = np.array([C[2, 1] - C[1, 2], C[0, 2] - C[2, 0], C[1, 0] - C[0, 1]])
    assert np.isclose(x @ S @ x, L.prod() * curl @ curl, rtol=1e-11)
    # the edge-gradient functions have no curl: their stiffness rows are zero
    assert abs(S[1::2]).max() == 0.0
    # a symmetric C (a gradient field) leaves no curl energy
    xs = _linear_field_dofs(g, a, C + C.T)
    assert abs(xs @ S @ xs) < 1e-12 * abs(S).max()
    # Whitney functions alone miss the linear field's energy
    g1 = tetmesh.grid_of(W.delaunay(5, 4, 4, 1, 1, 1, seed=3))
    _, M1 = tetmesh.mass_stiffness(g1)
    assert not np.isclose(x[0::2] @ M1 @ x[0::2], exact, rtol=1e-3)


def test_order2_converges_faster_than_whitney():
    err = {}
    for order in (1, 2):
        err[order] = []
        for n in (3, 6):
            w = W.delaunay(n, n, n, 1, 1, 1, seed=4, lossy=False, h=1.0 / n, order=order)
            w.eps[:] = 1.0
            f = fem.rhs_planewave(w)
            x = fem.solve_global(w, f)[:, 0]
            xi = fem.edge_interpolant(w, w.khat[0], w.pol[0])
            err[order].append(np.linalg.norm(x - xi) / np.linalg.norm(xi))
    assert err[2][1] < err[2][0] / 3.0
    assert all(e2 < e1 for e1, e2 in zip(err[1], err[2]))


@pytest.mark.parametrize("kw", [dict(), dict(nx=6, ny=5, nz=4, px=3, py=2, pz=1, seed=5)])
def test_order2_decomposed_equals_global(kw):
    w = _delaunay(order=2, **kw)
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    assert r["copy_mismatch"] < 1e-10 * np.abs(xg).max()
    xs = d3m.solve_primal_schur(w, f)
    assert np.abs(xs - xg).max() < 1e-10 * np.abs(xg).max()


def test_order2_adjoint_matches_central_differences():
    w = _delaunay(nx=3, ny=3, nz=2, px=1, py=1, pz=1, seed=21, order=2)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(0)
    probes = np.sort(rng.choice(w.n_edges, 6, replace=False))
    J, g = adjoint.gradient(w, f, probes)
    h = 1e-6
    for c in rng.choice(w.n_cells, 4, replace=False):
        e0 = w.eps.copy()
        w.eps = e0.copy(); w.eps[c] += h
        Jp = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0.copy(); w.eps[c] -= h
        Jm = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (c, fd, g[c], J)


# ------------------------------------------------- curl-complete second order


def test_collapsed_coordinate_rules_are_exact():
    import math
    P, Wt = tetmesh.duffy_tet(4)
    for a in range(6):
        for b in range(6 - a):
            for c in range(6 - a - b):
                q = np.sum(Wt * P[:, 1] ** a * P[:, 2] ** b * P[:, 3] ** c) / 6.0
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                assert abs(q - exact) < 1e-14 * exact, (a, b, c)
    P, Wt = tetmesh.duffy_tri(3)
    for a in range(5):
        for b in range(5 - a):
            q = 0.5 * np.sum(Wt * P[:, 1] ** a * P[:, 2] ** b)
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(q - exact) < 1e-14 * exact, (a, b)


def _order3(**kw):
    import dataclasses
    return dataclasses.replace(_delaunay(**kw), order=3)


def _projection(g, E):
    """L2 projection of the field E(points) onto the mesh's space: dofs x and
    the energy defect int |E|^2 - x^T M x (zero when E lies in the space)."""
    import scipy.sparse.linalg as spla
    X = g.V[g.T]
    G, vol = fem.tet_barycentric(X)
    vol = np.abs(vol)
    ell = np.stack([np.linalg.norm(X[:, b] - X[:, a], axis=1) for a, b in tetmesh.PAIRS], 1)
    tets = np.arange(g.n_cells)
    b = np.zeros(g.n_edges)
    energy = 0.0
    for lam, wt in zip(*tetmesh.duffy_tet(4)):
        if g.order == 3:
            N, _ = tetmesh._tet_basis3(g, lam, G, X, ell, tets)
        else:
            N = tetmesh._basis(lam, G, ell, tetmesh.PAIRS, g.order)
        N = N * g.tet_sign[:, :, None]
        e = E(np.einsum("i,cid->cd", lam, X))
        np.add.at(b, g.tet_dofs.ravel(), (wt * vol[:, None] * np.einsum("cid,cd->ci", N, e)).ravel())
        energy += np.sum(wt * vol * np.sum(e * e, 1))
    _, M = tetmesh.mass_stiffness(g)
    x = spla.spsolve(M.tocsc(), b)
    return x, (energy - x @ M @ x) / energy


def test_order3_holds_the_curl_complete_quadratic_fields():
    """E = d x (C d), d = r - r0, is a homogeneous quadratic field with
    E . d = 0, in the first-kind space of degree 2: its L2 projection keeps
    all of its energy, and the projection's curl energy is the exact
    int |tr(C) d - 3 C d|^2 (curl E in closed form).  The order-2 space
    misses it."""
    C = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.6], [0.7, 0.2, -0.1]])
    r0 = np.array([0.1, 0.05, 0.12])

    def E(r):
        d = r - r0
        return np.cross(d, d @ C.T)

    w = _order3(nx=4, ny=3, nz=3, px=1, py=1, pz=1)
    g = tetmesh.grid_of(w)
    x, defect = _projection(g, E)
    assert abs(defect) < 1e-12
    S, _ = tetmesh.mass_stiffness(g)
    L = np.array([w.lx, w.ly, w.lz])
    q, wq = fem.gauss01(2)
    exact = 0.0
    for i, xi in enumerate(q):
        for j, yj in enumerate(q):
            for k, zk in enumerate(q):
                d = np.array([xi, yj, zk]) * L - r0
                c = np.trace(C) * d - 3.0 * C @ d
                exact += wq[i] * wq[j] * wq[k] * (c @ c)
    exact *= L.prod()
    assert np.isclose(x @ S @ x, exact, rtol=1e-11)
    g2 = tetmesh.MeshGrid(w.vertices, w.tets, 2)
    _, defect2 = _projection(g2, E)
    assert defect2 > 1e-4


def test_order3_keeps_the_linear_fields_and_the_gradient_kernel():
    w = _order3(nx=4, ny=3, nz=3, px=1, py=1, pz=1)
    g = tetmesh.grid_of(w)
    S, M = tetmesh.mass_stiffness(g)
    a = np.array([0.3, -0.2, 0.5])
    C = np.array([[0.1, 0.4, -0.3], [0.2, -0.5, 0.6], [-0.7, 0.3, 0.2]])
    x = np.zeros(g.n_edges)
    g2 = tetmesh.MeshGrid(w.vertices, w.tets, 2)
    x[:2 * g.n_geo] = _linear_field_dofs(g2, a, C)       # face dofs zero: hierarchical
    L = np.array([w.lx, w.ly, w.lz])
    q, wq = fem.gauss01(2)
    exact = sum(wq[i] * wq[j] * wq[k] * np.sum((a + C @ (np.array([xi, yj, zk]) * L)) ** 2)
                for i, xi in enumerate(q) for j, yj in enumerate(q) for k, zk in enumerate(q)) * L.prod()
    assert np.isclose(x @ M @ x, exact, rtol=1e-12)
    xs = np.zeros(g.n_edges)
    xs[:2 * g.n_geo] = _linear_field_dofs(g2, a, C + C.T)  # a gradient field
    assert abs(S @ xs).max() < 1e-12 * abs(S).max()


@pytest.mark.parametrize("kw", [dict(), dict(nx=6, ny=5, nz=4, px=3, py=2, pz=1, seed=5)])
def test_order3_decomposed_equals_global(kw):
    """Face dofs on the interfaces are copied and tied like edge dofs."""
    w = _order3(**kw)
    f = fem.rhs_planewave(w)
    r = d3m.solve(w, f, return_all=True)
    xg = fem.solve_global(w, f)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max()
    assert r["copy_mismatch"] < 1e-10 * np.abs(xg).max()
    assert any(e >= 2 * tetmesh.grid_of(w).n_geo for e in r["dec"].lm_edge)   # face multipliers exist
    xs = d3m.solve_primal_schur(w, f)
    assert np.abs(xs - xg).max() < 1e-10 * np.abs(xg).max()
