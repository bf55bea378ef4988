"""Host symbolic stage of the library vs the oracle: bit-exact structure.

Runs on CPU (d3m_setup makes no CUDA call).  Compares the ordering of the
saddle matrix, supernode ranges and kinds, the supernodal elimination tree,
every front's update-row list, the multiplier map and the block order."""
import numpy as np
import pytest

from oracle import decomp, ordering
from paper_2002_05018_gb300 import d3m, workloads as W

CASES = [
    ("config1", lambda: W.make(1), 64),
    ("tiny-2x2x2", lambda: W.tiny(4, 4, 4, 2, 2, 2, seed=1), 16),
    ("tiny-jitter", lambda: W.tiny(9, 7, 5, 3, 2, 2, seed=4, jitter=True), 24),
    ("tiny-pec", lambda: _pec_case(), 32),
    # full-size workloads: jittered uneven 4x4x2 cuts (32^3 sphere; 48x48x24
    # PEC plate) and the 2x2x2 per-cell-eps workload; their M is too large for
    # the n x n bitset of the elimination game, so the oracle's children-merge
    # form (pinned against the game in test_oracle_ordering.py) is used
    ("config2", lambda: W.make(2), 64),
    ("config3", lambda: W.make(3), 64),
    ("config4", lambda: W.make(4), 64),
    # six tetrahedra per cell on jittered vertices: seven edge families, the
    # face diagonals of the cut planes among the interface edges
    ("tet-2x2x2", lambda: W.tetrahedral(W.tiny(4, 4, 4, 2, 2, 2, seed=1), 0.1, seed=2), 16),
    ("tet-jitter", lambda: W.tetrahedral(W.tiny(7, 6, 5, 3, 2, 2, seed=4, jitter=True), 0.1), 24),
    ("tet-config3", lambda: W.tetrahedral(W.make(3), 0.1), 64),
    # general tetrahedral meshes: a lattice mesh passed as vertex and
    # tetrahedron lists, and Delaunay meshes whose subdomains meet along
    # jagged interfaces (blocks between grid-diagonal subdomains)
    ("mesh-lattice", lambda: W.as_mesh(W.tetrahedral(W.tiny(6, 5, 4, 2, 2, 1, seed=1), 0.1)), 16),
    ("delaunay-2x2x2", lambda: W.delaunay(5, 4, 4, 2, 2, 2, seed=3), 16),
    ("delaunay-3x2x2", lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6), 32),
    # complete first order: two dofs per edge, kept together by the ordering
    ("delaunay-order2", lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6, order=2), 32),
    # curl-complete second order: face dofs, ordered with the edges
    ("delaunay-order3", lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6, order=3), 32),
]
LARGE = {"config2", "config3", "config4", "tet-config3"}


def _pec_case():
    w = W.tiny(8, 8, 6, 2, 2, 2, seed=5)
    w.pec_edge = W.pec_plate_mask(8, 8, 6, 2, 6, 2, 6, 3)   # plate on the z cut plane
    return w


@pytest.mark.parametrize("name,make,leaf", CASES)
def test_structure_bit_exact(name, make, leaf):
    w = make()
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=leaf)
    r, c = ordering.saddle_pattern(dec, plan)
    (ordering.symbolic_merge if name in LARGE else ordering.symbolic)(plan, r, c)
    s = d3m.Solver.from_workload(w, leaf_max=leaf)
    rng = s.structure(d3m.SN_RANGE)
    assert np.array_equal(rng[:, 0], plan.sn_start) and np.array_equal(rng[:, 1], plan.sn_end)
    kind = s.structure(d3m.SN_KIND)
    assert np.array_equal(kind[:, 0], plan.sn_kind) and np.array_equal(kind[:, 1], plan.sn_owner)
    assert np.array_equal(s.structure(d3m.SN_PARENT), plan.parent)
    st = s.structure(d3m.SN_STRUCT)
    n = len(plan.sn_start)
    ptr, idx = st[: n + 1], st[n + 1:]
    for q in range(n):
        assert np.array_equal(idx[ptr[q]:ptr[q + 1]], plan.struct[q]), q
    mm = s.structure(d3m.M_MAP)
    assert np.array_equal(mm[:, 0], plan.m_sub) and np.array_equal(mm[:, 1], plan.m_edge)
    lm = s.structure(d3m.LM)
    assert np.array_equal(lm[:, 0], dec.lm_edge)
    assert np.array_equal(lm[:, 1], dec.lm_plus) and np.array_equal(lm[:, 2], dec.lm_minus)
    bl = s.structure(d3m.BLOCKS)
    assert [tuple(x) for x in bl[:, :2]] == [tuple(b) for b in dec.blocks]
    s.close()


def test_library_exports_every_declared_symbol():
    import os
    import re
    lib = d3m.load()
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "d3m.h")).read()
    names = set(re.findall(r"\b(d3m_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for nme in names:
        assert hasattr(lib, nme), nme


def test_setup_rejects_unknown_fault(monkeypatch):
    monkeypatch.setenv("D3M_FAULT", "meteor")
    with pytest.raises(d3m.D3MError) as e:
        d3m.Solver.from_workload(W.tiny(4, 4, 4, 2, 1, 1))
    assert e.value.code == d3m.D3M_EINVAL and "D3M_FAULT" in str(e.value)


def test_setup_rejects_bad_input():
    w = W.tiny(4, 4, 4, 2, 1, 1)
    with pytest.raises(d3m.D3MError) as e:
        d3m.Solver(4, 4, 4, 1, 1, 1, w.eps, w.k, [0, 4, 4], [0, 4], [0, 4])
    assert e.value.code == d3m.D3M_EINVAL


@pytest.mark.parametrize("tet", [False, True, "mesh", "order2", "order3"])
def test_rhs_planewave_matches_oracle(tet):
    from oracle import fem
    w = W.tiny(5, 4, 3, 1, 1, 1, seed=8, nrhs=3)
    if tet in ("mesh", "order2", "order3"):
        w = W.delaunay(5, 4, 3, 2, 1, 1, seed=8, nrhs=3, order={"mesh": 1, "order2": 2, "order3": 3}[tet])
    elif tet:
        w = W.tetrahedral(w, 0.1)
    s = d3m.Solver.from_workload(w)
    assert s.n_edges == w.n_edges
    f = s.rhs_planewave(w.khat_pol6())
    fo = fem.rhs_planewave(w)
    assert np.abs(f - fo).max() < 1e-13 * np.abs(fo).max()


def _tet_vertices(w, move):
    v = W.lattice_vertices(w)
    for node, delta in move:
        v[node] += delta
    return v


def _mesh_kw(w, **over):
    kw = dict(element=d3m.TET_MESH, vertices=w.vertices, tets=w.tets, gcuts=w.gcuts)
    kw.update(over)
    return kw


@pytest.mark.parametrize("what", ["degenerate", "vertex-id", "no-cuts", "cuts-order", "lm_weight", "nonmanifold",
                                  "order", "pec-split", "empty-box"])
def test_setup_rejects_bad_general_meshes(what):
    """A degenerate tetrahedron, a vertex id out of range, missing or
    unordered coordinate cuts, the mass-weighted multiplier map and a
    triangle shared by three tetrahedra are refused at set-up."""
    w = W.delaunay(3, 3, 3, 2, 1, 1, seed=2)
    tets = w.tets.copy()
    if what == "degenerate":
        v = w.vertices.copy()
        t = tets[0]
        v[t[3]] = v[t[0]] + 0.5 * (v[t[1]] - v[t[0]]) + 0.5 * (v[t[2]] - v[t[0]])  # coplanar
        kw = _mesh_kw(w, vertices=v)
    elif what == "vertex-id":
        tets[3, 2] = len(w.vertices)
        kw = _mesh_kw(w, tets=tets)
    elif what == "no-cuts":
        kw = _mesh_kw(w, gcuts=None)
    elif what == "cuts-order":
        kw = _mesh_kw(w, gcuts=(w.gcuts[0][::-1], w.gcuts[1], w.gcuts[2]))
    elif what == "lm_weight":
        kw = _mesh_kw(w, lm_weight=1)
    elif what == "order":
        kw = _mesh_kw(w, order=4)
    elif what == "empty-box":   # a box too thin to hold a centroid
        gx = np.array([0.0, 0.15, 0.1501, 0.3])
        kw = _mesh_kw(w, gcuts=(gx, w.gcuts[1], w.gcuts[2]))
    elif what == "pec-split":   # order 2: the two dofs of an edge marked differently
        pec = np.zeros(2 * w.n_edges, np.uint8)
        pec[4] = 1
        kw = _mesh_kw(w, order=2, pec=pec)
    else:   # two more tetrahedra on the face (t0, t1, t2) of tetrahedron 0
        t, V = tets[0], w.vertices
        n = np.cross(V[t[1]] - V[t[0]], V[t[2]] - V[t[0]])
        far = np.argsort(-np.abs((V - V[t[0]]) @ n))[:2]   # off the face plane
        extra = np.array([[t[0], t[1], t[2], far[0]], [t[0], t[1], t[2], far[1]]])
        kw = _mesh_kw(w, tets=np.concatenate([tets, extra]))
    eps = np.ones(len(kw["tets"]), np.complex128)
    with pytest.raises(d3m.D3MError) as ei:
        d3m.Solver(0, 0, 0, 0.0, 0.0, 0.0, eps, w.k, w.cx, w.cy, w.cz, **kw)
    assert ei.value.code == d3m.D3M_EINVAL and "d3m_setup" in str(ei.value)
    if what == "nonmanifold":
        assert "more than two" in str(ei.value)
    if what == "degenerate":
        assert "degenerate" in str(ei.value)
    if what == "pec-split":
        assert "both dofs" in str(ei.value)
    if what == "empty-box":
        assert "no tetrahedron" in str(ei.value)


def test_general_mesh_with_pec_region_matches_oracle():
    """A PEC block inside a Delaunay mesh (the dofs of every edge whose
    midpoint lies in it removed): plan bit-exact against the oracle, and the
    oracle's D3M solution equals its global solution with zero field there."""
    from oracle import d3m as od3m, fem, tetmesh
    w = W.delaunay(6, 5, 5, 2, 2, 1, seed=7, nrhs=2)
    g = tetmesh.grid_of(w)
    mid = 0.5 * (g.V[g.edges[:, 0]] + g.V[g.edges[:, 1]])
    inside = np.all((mid > [0.2, 0.15, 0.15]) & (mid < [0.35, 0.3, 0.3]), axis=1)
    assert inside.sum() > 10
    w.pec_edge = inside.astype(np.uint8)
    f = fem.rhs_planewave(w)
    xg = fem.solve_global(w, f)
    r = od3m.solve(w, f, return_all=True)
    assert np.abs(r["x"] - xg).max() < 1e-10 * np.abs(xg).max() and np.all(xg[inside] == 0)
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=16)
    rr, cc = ordering.saddle_pattern(dec, plan)
    ordering.symbolic(plan, rr, cc)
    s = d3m.Solver.from_workload(w, leaf_max=16)
    rng, mm = s.structure(d3m.SN_RANGE), s.structure(d3m.M_MAP)
    assert np.array_equal(rng[:, 0], plan.sn_start) and np.array_equal(rng[:, 1], plan.sn_end)
    assert np.array_equal(mm[:, 0], plan.m_sub) and np.array_equal(mm[:, 1], plan.m_edge)
    assert np.array_equal(s.structure(d3m.SN_PARENT), plan.parent)
    assert s.stats()["n_free"] == w.n_edges - inside.sum()
    s.close()


def test_order2_is_for_general_meshes():
    w = W.tetrahedral(W.tiny(3, 3, 3, 1, 1, 1, seed=1), 0.1)
    with pytest.raises(d3m.D3MError) as ei:
        d3m.Solver.from_workload(w, order=2)
    assert ei.value.code == d3m.D3M_EINVAL and "D3M_TET_MESH" in str(ei.value)


@pytest.mark.parametrize("what", ["inverted", "off-plane", "brick-with-vertices", "element"])
def test_setup_rejects_bad_tetrahedral_meshes(what):
    """Inverted tetrahedra, boundary vertices moved off their plane, vertex
    positions with bricks and unknown element kinds are refused at set-up."""
    w = W.tiny(3, 3, 3, 1, 1, 1, seed=1)
    n = lambda i, j, k: i + 4 * (j + 4 * k)
    kw = dict(element=d3m.TET)
    if what == "inverted":      # interior node pushed through its neighbour
        kw["vertices"] = _tet_vertices(w, [(n(1, 1, 1), np.array([0.15, 0.15, 0.15]))])
    elif what == "off-plane":   # a node of the face x = 0 moved in x
        kw["vertices"] = _tet_vertices(w, [(n(0, 1, 1), np.array([0.01, 0.0, 0.0]))])
    elif what == "brick-with-vertices":
        kw = dict(element=d3m.BRICK, vertices=W.lattice_vertices(w))
    else:
        kw = dict(element=7)
    with pytest.raises(d3m.D3MError) as ei:
        d3m.Solver.from_workload(w, **kw)
    assert ei.value.code == d3m.D3M_EINVAL and "d3m_setup" in str(ei.value)


@pytest.mark.parametrize("mk", [lambda: W.make(1), lambda: W.delaunay(9, 7, 6, 3, 2, 2, seed=6, order=2)])
def test_level_table_matches_tree_heights(mk):
    """D3M_LEVELS: fronts grouped by height in the supernodal elimination tree
    (leaves 0, a parent one above its highest child), computed here from the
    oracle's plan; per-level flops add up to the factorisation's total (bricks
    and a complete first-order Delaunay mesh)."""
    w = mk()
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=64)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic(plan, r, c)
    n = len(plan.sn_start)
    h = np.zeros(n, np.int64)
    for q in range(n):  # children precede parents in elimination order
        if plan.parent[q] >= 0:
            h[plan.parent[q]] = max(h[plan.parent[q]], h[q] + 1)
    s = d3m.Solver.from_workload(w, leaf_max=64)
    lv = s.structure(d3m.LEVELS)
    assert lv.shape == (h.max() + 1, 10)
    pp = np.asarray(plan.sn_end) - np.asarray(plan.sn_start)
    mm = pp + np.array([len(plan.struct[q]) for q in range(n)])
    for L in range(h.max() + 1):
        sel = h == L
        assert lv[L, 0] == sel.sum() and lv[L, 1] == pp[sel].max() and lv[L, 2] == mm[sel].max()
    st = s.stats()
    total = st["flops_interior"] + st["flops_domain"] + st["flops_k"]
    assert abs(lv[:, 3].sum() - total) <= 1e-9 * total
    assert np.all(lv[:, 4:] == 0)  # nothing factored yet
    s.close()


@pytest.mark.parametrize("kw", [dict(update_kernel=3), dict(panel_kernel=2), dict(autotune=-1),
                                dict(lookahead=2), dict(leaf_max=-5), dict(refine_method=2),
                                dict(gmres_restart=201), dict(gmres_restart=-1), dict(gmres_tol=1.5),
                                dict(gmres_tol=-1e-3), dict(solve_kernel=2), dict(lm_weight=2)])
def test_setup_rejects_bad_options(kw):
    """Option values outside their documented sets are refused at set-up."""
    w = W.make(1)
    with pytest.raises(d3m.D3MError) as ei:
        d3m.Solver.from_workload(w, **kw)
    assert ei.value.code == d3m.D3M_EINVAL
    assert "d3m_setup" in str(ei.value)


@pytest.mark.parametrize("tet", [False, True, "mesh", "order2", "order3"])
def test_interface_coefficient_matches_oracle_entries(tet):
    """d3m_options.alpha sets the interface loss/gain term: the library's
    assembled entries of M equal the oracle's subdomain matrices for a
    non-default alpha (same check as for the default, row by row); on
    tetrahedra the element and face matrices are the library's closed forms
    against the oracle's quadrature."""
    from oracle import decomp
    w = W.tiny(4, 3, 3, 2, 1, 1, seed=6)
    if tet in ("mesh", "order2", "order3"):
        w = W.delaunay(5, 4, 4, 2, 2, 2, seed=3, order={"mesh": 1, "order2": 2, "order3": 3}[tet])
    elif tet:
        w = W.tetrahedral(W.tiny(4, 3, 3, 2, 2, 1, seed=6), 0.1)
    w.alpha = 2.5 - 0.7j
    s = d3m.Solver.from_workload(w)
    ent = s.structure(d3m.M_ENTRIES)
    mm = s.structure(d3m.M_MAP)
    s.close()
    dec = decomp.decompose(w)
    for sd in dec.subs:
        A = sd.A.tocsr()
        loc = -np.ones(int(mm[:, 1].max()) + 1, np.int64)
        loc[sd.edges] = np.arange(len(sd.edges))
        rows, cols = ent[:, 0].astype(np.int64), ent[:, 1].astype(np.int64)
        sel = (mm[rows, 0] == sd.index) & (mm[cols, 0] == sd.index)
        ar, ac = loc[mm[rows[sel], 1]], loc[mm[cols[sel], 1]]
        assert (ar >= 0).all() and (ac >= 0).all()
        ref = np.asarray(A[ar, ac]).ravel()
        got = ent[sel, 2] + 1j * ent[sel, 3]
        assert np.abs(ref - got).max() < 1e-12 * abs(A).max()


@pytest.mark.parametrize("tet", [False, True])
def test_mass_weighted_multiplier_map_matches_oracle_entries(tet):
    """d3m_options.lm_weight = 1: the library's multiplier couplings (rows of
    lambda, columns of the subdomain copies) equal the oracle's D_i = D_bool,i
    T_lambda entry for entry, on a partition with cross-lines."""
    from oracle import decomp
    w = W.tiny(6, 6, 4, 2, 2, 1, seed=4)
    if tet:
        w = W.tetrahedral(w, 0.1)
    w.lm_weight = 1
    s = d3m.Solver.from_workload(w)
    ent = s.structure(d3m.M_ENTRIES)
    mm = s.structure(d3m.M_MAP)
    st = s.stats()
    s.close()
    dec = decomp.decompose(w)
    lam_start = st["n_m"] - st["n_lm"]
    sel = (ent[:, 0] >= lam_start) & (ent[:, 1] < lam_start)
    Ds = {sd.index: (decomp.D_matrix(dec, sd).toarray(), {int(e): i for i, e in enumerate(sd.edges)})
          for sd in dec.subs}
    for r, c, re, im in ent[sel]:
        sub, e = mm[int(c)]
        D, loc = Ds[int(sub)]
        assert abs(D[loc[int(e)], int(r) - lam_start] - (re + 1j * im)) < 1e-15
    assert sel.sum() == sum(int((np.abs(D) > 0).sum()) for D, _ in Ds.values())


def test_c_program_drives_the_abi(tmp_path):
    """tests/c_abi/abi_check.c, compiled with gcc against include/d3m.h and
    linked to libd3m.so, sets up a brick mesh and a complete first-order
    general mesh from plain C; its counts and RHS norms equal the binding's for
    the same inputs (the header's struct layouts as C sees them)."""
    import math
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2002_05018_gb300")
    d3m.load()   # the library must have been built (raises otherwise)
    exe = str(tmp_path / "abi_check")
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                         os.path.join(root, "tests", "c_abi", "abi_check.c"), "-L", pkg, "-ld3m",
                         "-Wl,-rpath," + pkg, "-lm", "-o", exe], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    out = dict(ln.split() for ln in run.stdout.splitlines())
    assert out["ok"] == "1"
    kp = np.array([[0, 0, 1, 1, 0, 0, 0, 0, 0]], float)
    k = 2.0 * math.pi
    eps = (1.0 + 0.1 * np.arange(16)) - 0.05j
    brick = d3m.Solver(4, 2, 2, 0.4, 0.2, 0.2, eps, k, [0, 2, 4], [0, 2], [0, 2])
    v = np.array([[0.2 * (n & 1), 0.2 * ((n >> 1) & 1), 0.2 * ((n >> 2) & 1)] for n in range(8)])
    tets = np.array([[0, 1, 3, 7], [0, 1, 5, 7], [0, 2, 3, 7], [0, 2, 6, 7], [0, 4, 5, 7], [0, 4, 6, 7]])
    mesh = d3m.Solver(0, 0, 0, 0.0, 0.0, 0.0, np.full(6, 2.0 + 0j), k, [0], [0], [0], element=d3m.TET_MESH,
                      vertices=v, tets=tets, gcuts=([0.0, 0.1, 0.2], [0.0, 0.2], [0.0, 0.2]), order=2)
    mesh3 = d3m.Solver(0, 0, 0, 0.0, 0.0, 0.0, np.full(6, 2.0 + 0j), k, [0], [0], [0], element=d3m.TET_MESH,
                       vertices=v, tets=tets, gcuts=([0.0, 0.1, 0.2], [0.0, 0.2], [0.0, 0.2]), order=3)
    assert mesh3.n_edges == 2 * 19 + 2 * 18   # 19 edges and 18 faces of a cube's six tetrahedra
    for tag, s in (("brick", brick), ("mesh", mesh), ("mesh3", mesh3)):
        st = s.stats()
        for key in ("n_edges", "n_lm", "n_m", "n_fronts"):
            assert int(out[f"{tag}_{key}"]) == st[key], (tag, key)
        assert int(out[f"{tag}_m_map_bytes"]) == 16 * st["n_m"]
        f = s.rhs_planewave(kp)
        assert abs(float(out[f"{tag}_rhs_l1"]) - (np.abs(f.real).sum() + np.abs(f.imag).sum())) < 1e-12
        s.close()


def test_entry_points_refuse_bad_arguments_before_any_device_work():
    """Host-side argument checks of the ABI (run on CPU: each returns before
    any CUDA call): null pointers, nrhs <= 0, leading dimensions shorter than
    n_edges, out-of-range fronts and structure kinds, bad dense-front sizes."""
    import ctypes
    lib = d3m.load()
    s = d3m.Solver.from_workload(W.tiny(4, 3, 3, 2, 1, 1, seed=2))
    h, n = s.h, s.n_edges
    buf = np.zeros(4 * n + 64)
    p = buf.ctypes.data
    E = d3m.D3M_EINVAL
    for fn in (lib.d3m_solve, lib.d3m_solve_host, lib.d3m_solve_adjoint):
        assert fn(h, p, n, p, n, 0, None) == E            # no right-hand side
        assert fn(h, p, n, p, n, -3, None) == E
        assert fn(h, p, n - 1, p, n, 1, None) == E        # ldb < n_edges
        assert fn(h, p, n, p, n - 1, 1, None) == E        # ldx < n_edges
        assert fn(h, None, n, p, n, 1, None) == E
        assert fn(h, p, n, None, n, 1, None) == E
        assert fn(None, p, n, p, n, 1, None) == E
    assert lib.d3m_grad_eps(h, p, n, p, n, 0, p) == E
    assert lib.d3m_grad_eps(h, p, n - 1, p, n, 1, p) == E
    assert lib.d3m_grad_eps(h, p, n, p, n, 1, None) == E
    assert lib.d3m_rhs_planewave(h, p, 1, p, n - 1) == E
    assert lib.d3m_rhs_planewave(h, p, -1, p, n) == E
    assert lib.d3m_rhs_planewave(h, None, 1, p, n) == E
    m_out, p_out = ctypes.c_int32(), ctypes.c_int32()
    nf = s.stats()["n_fronts"]
    assert lib.d3m_export_front(h, nf, ctypes.byref(m_out), ctypes.byref(p_out), None, None, None) == E
    assert lib.d3m_export_front(h, -1, ctypes.byref(m_out), ctypes.byref(p_out), None, None, None) == E
    nbytes = ctypes.c_size_t(0)
    assert lib.d3m_structure(h, 99, None, ctypes.byref(nbytes)) == E
    assert lib.d3m_structure(h, d3m.SN_RANGE, None, None) == E
    assert lib.d3m_stats_get(h, None) == E
    ip = np.zeros(8, np.int32).ctypes.data
    for m, pp, batch in ((0, 0, 1), (4, 5, 1), (4, -1, 1), (4, 2, 0)):
        assert lib.d3m_dense_ldlt(m, pp, batch, p, ip, p, ip, None, 0) == E, (m, pp, batch)
    assert lib.d3m_dense_ldlt(4, 2, 1, None, ip, p, ip, None, 0) == E
    s.close()


@pytest.mark.parametrize("case", range(15))
def test_structure_bit_exact_on_random_meshes(case):
    """Seeded random meshes (bricks, lattice tetrahedra, Delaunay meshes of
    orders 1 to 3; random sizes, partitions, cut jitter and leaf sizes): the
    library's plan equals the oracle's bit for bit."""
    rng = np.random.default_rng(1000 + case)
    nx, ny, nz = [int(v) for v in rng.integers(2, 8, 3)]
    px, py, pz = [int(rng.integers(1, min(3, n) + 1)) for n in (nx, ny, nz)]
    kind, seed, leaf = case % 5, int(rng.integers(0, 1000)), int(rng.integers(4, 40))
    if kind < 2:
        w = W.tiny(nx, ny, nz, px, py, pz, seed=seed)
        if kind == 1:
            w = W.tetrahedral(w, 0.1)
    else:
        w = W.delaunay(nx, ny, nz, px, py, pz, seed=seed, order=kind - 1,
                       jitter=float(rng.uniform(0.05, 0.35)))
    dec = decomp.decompose(w)
    plan = ordering.build_plan(dec, leaf_max=leaf)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic_merge(plan, r, c)
    s = d3m.Solver.from_workload(w, leaf_max=leaf)
    rng_, mm = s.structure(d3m.SN_RANGE), s.structure(d3m.M_MAP)
    assert np.array_equal(rng_[:, 0], plan.sn_start) and np.array_equal(rng_[:, 1], plan.sn_end)
    assert np.array_equal(mm[:, 0], plan.m_sub) and np.array_equal(mm[:, 1], plan.m_edge)
    assert np.array_equal(s.structure(d3m.SN_PARENT), plan.parent)
    st = s.structure(d3m.SN_STRUCT)
    n = len(plan.sn_start)
    for q in range(n):
        assert np.array_equal(st[n + 1:][st[q]:st[q + 1]], plan.struct[q]), q
    lm = s.structure(d3m.LM)
    assert np.array_equal(lm[:, 0], dec.lm_edge) and np.array_equal(lm[:, 1], dec.lm_plus)
    s.close()


@pytest.mark.parametrize("case", range(8))
def test_entries_match_oracle_on_random_meshes(case):
    """Every assembled entry of M (element, interface and absorbing terms,
    multiplier couplings) on seeded random lattice-tetrahedral and Delaunay
    meshes (orders 1 to 3) equals the oracle's subdomain matrices and D_i."""
    rng = np.random.default_rng(2000 + case)
    nx, ny, nz = [int(v) for v in rng.integers(2, 6, 3)]
    px, py, pz = [int(rng.integers(1, min(3, n) + 1)) for n in (nx, ny, nz)]
    seed = int(rng.integers(0, 1000))
    if case % 4 == 0:
        w = W.tetrahedral(W.tiny(nx, ny, nz, px, py, pz, seed=seed), 0.1)
    else:
        w = W.delaunay(nx, ny, nz, px, py, pz, seed=seed, order=case % 4)
    s = d3m.Solver.from_workload(w)
    ent, mm, st = s.structure(d3m.M_ENTRIES), s.structure(d3m.M_MAP), s.stats()
    s.close()
    dec = decomp.decompose(w)
    lam0 = st["n_m"] - st["n_lm"]
    A = {sd.index: (sd.A.toarray(), {int(e): i for i, e in enumerate(sd.edges)}) for sd in dec.subs}
    Ds = {sd.index: decomp.D_matrix(dec, sd).toarray() for sd in dec.subs}
    scale = max(np.abs(a).max() for a, _ in A.values())
    for r, c, re, im in ent:
        r, c = int(r), int(c)
        v = re + 1j * im
        if r < lam0:
            sub, er = mm[r]
            _, ec = mm[c]
            Ai, loc = A[int(sub)]
            assert abs(Ai[loc[int(er)], loc[int(ec)]] - v) < 1e-12 * scale
        else:
            sub, e = mm[c]
            _, loc = A[int(sub)]
            assert abs(Ds[int(sub)][loc[int(e)], r - lam0] - v) < 1e-15


@pytest.mark.parametrize("mk", [
    lambda: W.tiny(4, 4, 3, 2, 2, 1, seed=3, nrhs=2),
    lambda: W.tetrahedral(W.tiny(4, 3, 3, 2, 2, 1, seed=4, nrhs=2), 0.1),
    lambda: W.delaunay(5, 4, 4, 2, 2, 2, seed=3, nrhs=2),
    lambda: W.delaunay(5, 4, 4, 2, 2, 2, seed=3, nrhs=2, order=2),
    lambda: W.delaunay(4, 4, 3, 2, 2, 1, seed=3, nrhs=2, order=3),
])
def test_exported_saddle_matrix_solves_to_the_oracle(mk):
    """The whole host set-up end to end on CPU: the library's saddle matrix M
    (d3m_structure: its entries in its own M order), solved densely in fp64
    with the owner-split RHS, gives the oracle's solution E (each edge's
    owner copy) and the oracle's multipliers lambda (Eq. (1))."""
    from oracle import d3m as od3m, fem
    w = mk()
    f = fem.rhs_planewave(w)
    s = d3m.Solver.from_workload(w)
    ent, mm, st = s.structure(d3m.M_ENTRIES), s.structure(d3m.M_MAP), s.stats()
    s.close()
    n, lam0 = st["n_m"], st["n_m"] - st["n_lm"]
    M = np.zeros((n, n), np.complex128)
    M[ent[:, 0].astype(int), ent[:, 1].astype(int)] += ent[:, 2] + 1j * ent[:, 3]
    M = M + np.tril(M, -1).T
    dec = decomp.decompose(w, with_matrices=False)
    owner = np.array([dec.copies[int(e)][0] == sub for sub, e in mm[:lam0]])
    b = np.zeros((n, f.shape[1]), np.complex128)
    b[:lam0][owner] = f[mm[:lam0, 1][owner]]
    z = np.linalg.solve(M, b)
    ref = od3m.solve(w, f, return_all=True)
    assert np.abs(z[lam0:] - ref["lam"]).max() < 1e-10 * np.abs(ref["lam"]).max()
    x = np.zeros_like(f)
    x[mm[:lam0, 1][owner]] = z[:lam0][owner]
    xg = fem.solve_global(w, f)
    assert np.abs(x - xg).max() < 1e-10 * np.abs(xg).max()
