"""FEM discretisation of the paper's BVP (Theory section) -- oracle, test only.

    curl(curl E) - k^2 eps_r E = 0 in Omega   (mu_r = 1, J_imp = 0)
    n x curl E - jk E_t = n x curl E_inc - jk E_inc,t   on dOmega (1st-order ABC)

Weak form with outward normal n and time convention e^{jwt}:
    A x = f,  A = S - k^2 sum_c eps_c M_c + jk T,   f_v = -int_dOmega U . N_v dS,
    U = n x curl E_inc - jk (E_inc)_t.
A is complex symmetric (A = A^T, stated for K in the paper's discussion of
LDL^T).  Two element kinds (the general FEM setting of the Introduction):

- brick: lowest-order Nedelec brick elements on an axis-aligned grid; element
  integrals by tensor Gauss-Legendre quadrature (2 points per axis is exact
  for the bilinear-by-linear integrands; the incident-field RHS uses 3x3
  points per face, a stated reading because the paper gives no quadrature);
- tet: lowest-order Nedelec (Whitney) tetrahedra, six per lattice cell split
  along the cell's (0,0,0)-(1,1,1) diagonal, on jittered vertex positions.
  The edge function of edge (a, b) is l_ab (lam_a grad lam_b - lam_b grad lam_a)
  (so its dof is the line average of E . t along the edge, as for bricks).
  Element and face integrals by the degree-2 4-point tetrahedron rule and the
  3-point edge-midpoint triangle rule (exact for these quadratic integrands);
  the incident-field RHS uses the degree-5 7-point triangle rule (stated
  reading, as above).

Global edge numbering: edge families one after another, each x-fastest over
its own box of start nodes (i, j, k); directions (1,0,0), (0,1,0), (0,0,1)
(bricks and tets), then (1,1,0), (1,0,1), (0,1,1), (1,1,1) (tets only).  Every
edge points from its start node to start + direction.

Pins (tests/test_oracle_fem.py, tests/test_oracle_tet.py): S G = 0 for the
discrete gradient, M SPD, 1-D mass factors h/3, h/6, constant-field mass =
eps * volume, constant-curl stiffness = |curl|^2 * volume, boundary face mass
of a constant field = tangential |E|^2 * area, A = A^T, plane-wave
convergence in a homogeneous box, reciprocity, quadrature exactness.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------- numbering


_DIRS = {"brick": [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
         "tet": [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]}


class Grid:
    """Grid [0,lx]x[0,ly]x[0,lz] with nx*ny*nz cells: bricks, or six
    tetrahedra per cell on (optionally jittered) vertex positions."""

    def __init__(self, nx, ny, nz, lx, ly, lz, element="brick", vertices=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.ly, self.lz = float(lx), float(ly), float(lz)
        self.h = np.array([lx / nx, ly / ny, lz / nz])
        self.element = element
        self.dirs = np.array(_DIRS[element], np.int64)
        self.fam_shape = [(self.nx + 1 - d[0], self.ny + 1 - d[1], self.nz + 1 - d[2])
                          for d in self.dirs]
        sizes = [a * b * c for a, b, c in self.fam_shape]
        self.fam_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.nex, self.ney, self.nez = sizes[:3]
        self.n_edges = int(self.fam_off[-1])
        self.n_cells = nx * ny * nz
        self.n_nodes = (self.nx + 1) * (self.ny + 1) * (self.nz + 1)
        if vertices is not None and element == "brick":
            raise ValueError("brick elements are axis-aligned: no vertex positions")
        if vertices is None:
            kk, jj, ii = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1),
                                     np.arange(self.nx + 1), indexing="ij")
            vertices = np.stack([ii.ravel() * self.h[0], jj.ravel() * self.h[1],
                                 kk.ravel() * self.h[2]], 1)
        self.nodes = np.asarray(vertices, np.float64).reshape(self.n_nodes, 3)

    @classmethod
    def of(cls, w):
        return cls(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, getattr(w, "element", "brick"),
                   getattr(w, "vertices", None))

    def node_id(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    # edge ids from family and start-node indices (vectorised)
    def edge_id(self, d, i, j, k):
        sx, sy, _ = self.fam_shape[d]
        return self.fam_off[d] + i + sx * (j + sy * k)

    def ex(self, i, j, k):
        return self.edge_id(0, i, j, k)

    def ey(self, i, j, k):
        return self.edge_id(1, i, j, k)

    def ez(self, i, j, k):
        return self.edge_id(2, i, j, k)

    def edge_info(self):
        """(family, i, j, k) of every edge, as int arrays (family = direction
        0/1/2 on brick grids)."""
        out = []
        for d, (sx, sy, sz) in enumerate(self.fam_shape):
            kk, jj, ii = np.meshgrid(np.arange(sz), np.arange(sy), np.arange(sx), indexing="ij")
            out.append(np.stack([np.full(ii.size, d), ii.ravel(), jj.ravel(), kk.ravel()], 1))
        return np.concatenate(out, 0)

    def edge_nodes(self):
        """(start node, end node) ids of every edge."""
        info = self.edge_info()
        d, i, j, k = info.T
        dv = self.dirs[d]
        return (self.node_id(i, j, k),
                self.node_id(i + dv[:, 0], j + dv[:, 1], k + dv[:, 2]))

    def cell_ijk(self):
        kk, jj, ii = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                                 indexing="ij")
        return ii.ravel(), jj.ravel(), kk.ravel()

    def cell_edges(self, ci=None, cj=None, ck=None):
        """(ncells, 12) global edges of each cell in local order:
        x-edges (dy, dz) = (0,0),(1,0),(0,1),(1,1); y-edges (dx, dz) likewise;
        z-edges (dx, dy) likewise.  Tetrahedral grids append 7 columns: the
        (1,1,0) diagonals at dz = 0, 1, the (1,0,1) diagonals at dy = 0, 1, the
        (0,1,1) diagonals at dx = 0, 1 and the cell diagonal: (ncells, 19)."""
        if ci is None:
            ci, cj, ck = self.cell_ijk()
        o = [(0, 0), (1, 0), (0, 1), (1, 1)]
        cols = [self.ex(ci, cj + a, ck + b) for a, b in o]
        cols += [self.ey(ci + a, cj, ck + b) for a, b in o]
        cols += [self.ez(ci + a, cj + b, ck) for a, b in o]
        if self.element == "tet":
            cols += [self.edge_id(3, ci, cj, ck + b) for b in (0, 1)]
            cols += [self.edge_id(4, ci, cj + a, ck) for a in (0, 1)]
            cols += [self.edge_id(5, ci + a, cj, ck) for a in (0, 1)]
            cols += [self.edge_id(6, ci, cj, ck)]
        return np.stack(cols, 1).astype(np.int64)

    def cell_nodes(self, cells):
        """(ncells, 2, 2, 2, 3) vertex positions of the given cells, indexed
        [dx, dy, dz]."""
        ci, cj, ck = (a[cells] for a in self.cell_ijk())
        out = np.zeros((len(ci), 2, 2, 2, 3))
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    out[:, a, b, c] = self.nodes[self.node_id(ci + a, cj + b, ck + c)]
        return out


# ------------------------------------------------------- local basis on a brick

_OFF = [(0, 0), (1, 0), (0, 1), (1, 1)]


def _phi(t, a):
    return t if a else 1.0 - t


def _dphi(a):
    return 1.0 if a else -1.0


def basis(xi, eta, zeta, h):
    """Values (12, 3) and curls (12, 3) of the 12 edge functions at a
    reference point of a brick with sides h = (hx, hy, hz)."""
    hx, hy, hz = h
    N = np.zeros((12, 3))
    C = np.zeros((12, 3))
    for e, (a, b) in enumerate(_OFF):      # x-edge: x^ phi_a(eta) phi_b(zeta)
        N[e, 0] = _phi(eta, a) * _phi(zeta, b)
        C[e] = [0.0, _phi(eta, a) * _dphi(b) / hz, -_dphi(a) * _phi(zeta, b) / hy]
    for e, (a, b) in enumerate(_OFF):      # y-edge: y^ phi_a(xi) phi_b(zeta)
        N[4 + e, 1] = _phi(xi, a) * _phi(zeta, b)
        C[4 + e] = [-_phi(xi, a) * _dphi(b) / hz, 0.0, _dphi(a) * _phi(zeta, b) / hx]
    for e, (a, b) in enumerate(_OFF):      # z-edge: z^ phi_a(xi) phi_b(eta)
        N[8 + e, 2] = _phi(xi, a) * _phi(eta, b)
        C[8 + e] = [_phi(xi, a) * _dphi(b) / hy, -_dphi(a) * _phi(eta, b) / hx, 0.0]
    return N, C


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def element_matrices(h):
    """Element stiffness S_e = int curl N . curl N and mass M_e = int N . N
    by 2x2x2 Gauss-Legendre quadrature."""
    q, w = gauss01(2)
    vol = h[0] * h[1] * h[2]
    S = np.zeros((12, 12))
    M = np.zeros((12, 12))
    for a, xa in enumerate(q):
        for b, xb in enumerate(q):
            for c, xc in enumerate(q):
                N, C = basis(xa, xb, xc, h)
                wt = w[a] * w[b] * w[c] * vol
                S += wt * C @ C.T
                M += wt * N @ N.T
    return S, M


_FACE_PARAM = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


def _face_point(axis, side, s, t):
    p = [0.0, 0.0, 0.0]
    u, v = _FACE_PARAM[axis]
    p[axis] = float(side)
    p[u], p[v] = s, t
    return p


def face_matrix(h, axis, side):
    """T_f = int_face (N_t . N_t) dS on the face {axis coordinate = side} of a
    brick (tangential parts only), 2x2 Gauss-Legendre (exact)."""
    q, w = gauss01(2)
    u, v = _FACE_PARAM[axis]
    area = h[u] * h[v]
    T = np.zeros((12, 12))
    n = np.zeros(3)
    n[axis] = 1.0
    for a, s in enumerate(q):
        for b, t in enumerate(q):
            N, _ = basis(*_face_point(axis, side, s, t), h)
            Nt = N - np.outer(N @ n, n)
            T += w[a] * w[b] * area * Nt @ Nt.T
    return T


# ------------------------------------------- Whitney tetrahedra, six per cell


def _cell_local_index():
    """(start offset (dx, dy, dz), direction) -> column of Grid.cell_edges."""
    idx = {}
    for q, (a, b) in enumerate(_OFF):
        idx[((0, a, b), (1, 0, 0))] = q
        idx[((a, 0, b), (0, 1, 0))] = 4 + q
        idx[((a, b, 0), (0, 0, 1))] = 8 + q
    for b in (0, 1):
        idx[((0, 0, b), (1, 1, 0))] = 12 + b
        idx[((0, b, 0), (1, 0, 1))] = 14 + b
        idx[((b, 0, 0), (0, 1, 1))] = 16 + b
    idx[((0, 0, 0), (1, 1, 1))] = 18
    return idx


_LOCAL = _cell_local_index()


def _kuhn_tets():
    """The six tetrahedra of a cell, each as its 4 vertex offsets: the
    monotone lattice paths (0,0,0) -> e_a -> e_a + e_b -> (1,1,1)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        v = [(0, 0, 0)]
        for ax in perm:
            nxt = list(v[-1])
            nxt[ax] = 1
            v.append(tuple(nxt))
        out.append(v)
    return out


TETS = _kuhn_tets()
_TET_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
_TRI_EDGES = [(0, 1), (0, 2), (1, 2)]


def local_edge(o1, o2):
    """Cell-edge column of the edge from vertex offset o1 to o2 (o2 >= o1)."""
    d = tuple(int(b) - int(a) for a, b in zip(o1, o2))
    return _LOCAL[(tuple(int(a) for a in o1), d)]


def _corner(cn, o):
    return cn[:, o[0], o[1], o[2]]


def tet_barycentric(X):
    """Gradients (n, 4, 3) of the barycentric coordinates and signed volumes
    (n,) of tetrahedra with vertices X (n, 4, 3): lam_i(x) = C[0, i] + C[1:, i] . x
    where [1 X] C = I."""
    A = np.concatenate([np.ones(X.shape[:2] + (1,)), X], 2)
    C = np.linalg.inv(A)
    return np.transpose(C[:, 1:, :], (0, 2, 1)), np.linalg.det(A) / 6.0


def _parity(perm_vertices):
    """+1 / -1: orientation of a tetrahedron of the undistorted unit cell."""
    X = np.array(perm_vertices, float)[None]
    return float(np.sign(tet_barycentric(X)[1][0]))


def tet_volumes(g: Grid, cells=None):
    """(ncells, 6) volumes of the six tetrahedra of each cell, signed so that
    a tetrahedron keeping the orientation it has in the undistorted cell is
    positive (a valid mesh has all six positive)."""
    cells = np.arange(g.n_cells) if cells is None else np.asarray(cells)
    cn = g.cell_nodes(cells)
    return np.stack([_parity(tv) * tet_barycentric(np.stack([_corner(cn, o) for o in tv], 1))[1]
                     for tv in TETS], 1)


def tet_quadrature():
    """Degree-2 4-point rule on a tetrahedron: barycentric points, weights
    (fractions of the volume)."""
    al, be = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0, (5.0 - np.sqrt(5.0)) / 20.0
    return np.array([np.roll([al, be, be, be], r) for r in range(4)]), np.full(4, 0.25)


def tri_quadrature(degree):
    """Triangle rules as barycentric points and weights (fractions of the area):
    degree 2, the 3 edge midpoints; degree 5, the 7-point rule of Radon."""
    if degree == 2:
        return np.array([[0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]), np.full(3, 1.0 / 3.0)
    r = np.sqrt(15.0)
    pts, wts = [[1.0 / 3.0] * 3], [9.0 / 40.0]
    for a, wt in (((6.0 - r) / 21.0, (155.0 - r) / 1200.0), ((6.0 + r) / 21.0, (155.0 + r) / 1200.0)):
        b = 1.0 - 2.0 * a
        pts += [[a, a, b], [a, b, a], [b, a, a]]
        wts += [wt] * 3
    return np.array(pts), np.array(wts)


def _whitney(lam, G, ell, pairs):
    """Edge functions l_ab (lam_a grad lam_b - lam_b grad lam_a): (n, len(pairs), 3)."""
    return np.stack([lam[a] * G[:, b] - lam[b] * G[:, a] for a, b in pairs], 1) * ell[..., None]


def tet_cell_matrices(g: Grid, cells):
    """Per-cell S_c = int curl N . curl N and M_c = int N . N over the six
    tetrahedra, in Grid.cell_edges column order: (ncells, 19, 19) each."""
    cells = np.asarray(cells)
    cn = g.cell_nodes(cells)
    nc = len(cells)
    S = np.zeros((nc, 19, 19))
    M = np.zeros((nc, 19, 19))
    qp, qw = tet_quadrature()
    for tv in TETS:
        X = np.stack([_corner(cn, o) for o in tv], 1)
        G, vol = tet_barycentric(X)
        vol = np.abs(vol)
        loc = [local_edge(tv[a], tv[b]) for a, b in _TET_EDGES]
        ell = np.stack([np.linalg.norm(X[:, b] - X[:, a], axis=1) for a, b in _TET_EDGES], 1)
        curl = np.stack([2.0 * np.cross(G[:, a], G[:, b]) for a, b in _TET_EDGES], 1) * ell[..., None]
        Sl = vol[:, None, None] * np.einsum("cid,cjd->cij", curl, curl)
        Ml = np.zeros((nc, 6, 6))
        for lam, wt in zip(qp, qw):
            N = _whitney(lam, G, ell, _TET_EDGES)
            Ml += wt * vol[:, None, None] * np.einsum("cid,cjd->cij", N, N)
        for i in range(6):
            for j in range(6):
                S[:, loc[i], loc[j]] += Sl[:, i, j]
                M[:, loc[i], loc[j]] += Ml[:, i, j]
    return S, M


def face_triangles(axis, side):
    """The two triangles of cell face {axis = side} as vertex offsets: the
    face is split along its diagonal from the lowest to the highest corner."""
    u, v = _FACE_PARAM[axis]
    o0 = [0, 0, 0]
    o0[axis] = side
    eu, ev = list(o0), list(o0)
    eu[u] = 1
    ev[v] = 1
    euv = list(eu)
    euv[v] = 1
    return [(tuple(o0), tuple(eu), tuple(euv)), (tuple(o0), tuple(ev), tuple(euv))]


def tri_frame(Q):
    """In-plane gradients (n, 3, 3) of the barycentric coordinates and the
    areas (n,) of triangles Q (n, 3, 3): the minimum-norm solutions of
    (Q_1 - Q_0, Q_2 - Q_0) . grad mu_i = (mu_i(Q_1) - mu_i(Q_0), mu_i(Q_2) - mu_i(Q_0))."""
    E = np.stack([Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0]], 1)
    Pinv = np.linalg.pinv(E)
    rhs = np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
    G = np.einsum("cpk,ki->cip", Pinv, rhs)
    area = 0.5 * np.linalg.norm(np.cross(E[:, 0], E[:, 1]), axis=1)
    return G, area


def _tri_setup(cn, tri):
    Q = np.stack([_corner(cn, o) for o in tri], 1)
    G, area = tri_frame(Q)
    loc = [local_edge(tri[a], tri[b]) for a, b in _TRI_EDGES]
    ell = np.stack([np.linalg.norm(Q[:, b] - Q[:, a], axis=1) for a, b in _TRI_EDGES], 1)
    return Q, G, area, loc, ell


def tet_face_matrices(g: Grid, axis, side, cells):
    """Tangential face mass int_face N_t . N_t dS of face {axis = side} of
    each cell (two triangles, edge-midpoint rule): (ncells, 19, 19)."""
    cells = np.asarray(cells)
    cn = g.cell_nodes(cells)
    T = np.zeros((len(cells), 19, 19))
    qp, qw = tri_quadrature(2)
    for tri in face_triangles(axis, side):
        _, G, area, loc, ell = _tri_setup(cn, tri)
        Tl = np.zeros((len(cells), 3, 3))
        for mu, wt in zip(qp, qw):
            N = _whitney(mu, G, ell, _TRI_EDGES)
            Tl += wt * area[:, None, None] * np.einsum("cid,cjd->cij", N, N)
        for i in range(3):
            for j in range(3):
                T[:, loc[i], loc[j]] += Tl[:, i, j]
    return T


def face_block(g: Grid, axis, side, cells):
    """Face mass of face {axis = side} of each given cell, (ncells, ne, ne)."""
    if g.element == "brick":
        T = face_matrix(g.h, axis, side)
        return np.broadcast_to(T, (len(cells), 12, 12))
    return tet_face_matrices(g, axis, side, cells)


# ----------------------------------------------------------------- assembly


def boundary_faces(g: Grid, cell_lo=(0, 0, 0), cell_hi=None, planes=None):
    """Yield (axis, side, cell ids) for the faces of the cell box
    [cell_lo, cell_hi) that lie on the given planes {axis: [node coords]}.
    Default: the outer boundary of the grid."""
    hi = (g.nx, g.ny, g.nz) if cell_hi is None else cell_hi
    lo = cell_lo
    ci, cj, ck = g.cell_ijk()
    cid = np.arange(g.n_cells)
    inbox = (ci >= lo[0]) & (ci < hi[0]) & (cj >= lo[1]) & (cj < hi[1]) & (ck >= lo[2]) & (ck < hi[2])
    coords = (ci, cj, ck)
    for axis in range(3):
        for side, node in ((0, lo[axis]), (1, hi[axis])):
            if planes is not None and node not in planes.get(axis, ()):
                continue
            cell_layer = node if side == 0 else node - 1
            sel = inbox & (coords[axis] == cell_layer)
            if sel.any():
                yield axis, side, cid[sel]


def assemble(g: Grid, eps, k, cells=None, extra_faces=()):
    """COO pieces of S - k^2 sum eps_c M_c + jk T_dOmega over the given cells
    (default all).  extra_faces: iterable of (axis, side, cell ids, coeff)
    face terms coeff * T_f (used for interface loss/gain)."""
    cells = np.arange(g.n_cells) if cells is None else np.asarray(cells)
    ce = g.cell_edges()[cells]
    ne = ce.shape[1]
    rows = np.repeat(ce, ne, axis=1).ravel()
    cols = np.tile(ce, (1, ne)).ravel()
    if g.element == "brick":
        S_e, M_e = element_matrices(g.h)
        vals = (S_e.ravel()[None, :] - (k * k) * eps[cells][:, None] * M_e.ravel()[None, :]).ravel()
    else:
        S_c, M_c = tet_cell_matrices(g, cells)
        vals = (S_c.reshape(len(cells), ne * ne)
                - (k * k) * eps[cells][:, None] * M_c.reshape(len(cells), ne * ne)).ravel()
    R, C, V = [rows], [cols], [vals.astype(np.complex128)]
    for axis, side, cid, coeff in extra_faces:
        T = face_block(g, axis, side, cid)
        ce = g.cell_edges()[cid]
        R.append(np.repeat(ce, ne, axis=1).ravel())
        C.append(np.tile(ce, (1, ne)).ravel())
        V.append((coeff * T.reshape(len(cid), ne * ne)).ravel().astype(np.complex128))
    return np.concatenate(R), np.concatenate(C), np.concatenate(V)


def mass_stiffness(g: Grid, cells=None):
    """Real sparse global S and M (eps = 1, no boundary terms)."""
    cells = np.arange(g.n_cells) if cells is None else np.asarray(cells)
    ce = g.cell_edges()[cells]
    ne = ce.shape[1]
    rows = np.repeat(ce, ne, axis=1).ravel()
    cols = np.tile(ce, (1, ne)).ravel()
    if g.element == "brick":
        S_e, M_e = element_matrices(g.h)
        sv = np.broadcast_to(S_e.ravel(), (len(cells), ne * ne)).ravel()
        mv = np.broadcast_to(M_e.ravel(), (len(cells), ne * ne)).ravel()
    else:
        S_c, M_c = tet_cell_matrices(g, cells)
        sv, mv = S_c.ravel(), M_c.ravel()
    shape = (g.n_edges, g.n_edges)
    return (sp.csr_matrix((sv, (rows, cols)), shape=shape),
            sp.csr_matrix((mv, (rows, cols)), shape=shape))


def abc_faces(g: Grid, k, cells_lo=(0, 0, 0), cells_hi=None):
    """(axis, side, cells, jk) for the outer-boundary faces inside a cell box."""
    out = []
    planes = {0: (0, g.nx), 1: (0, g.ny), 2: (0, g.nz)}
    for axis, side, cid in boundary_faces(g, cells_lo, cells_hi, planes):
        node = cells_lo[axis] if side == 0 else (cells_hi or (g.nx, g.ny, g.nz))[axis]
        if node in (0, (g.nx, g.ny, g.nz)[axis]):
            out.append((axis, side, cid, 1j * k))
    return out


def global_matrix(w):
    """Sparse CSR A (all edges, PEC rows not yet removed)."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.global_matrix(w)
    g = Grid.of(w)
    r, c, v = assemble(g, w.eps, w.k, extra_faces=abc_faces(g, w.k))
    return sp.csr_matrix((v, (r, c)), shape=(g.n_edges, g.n_edges))


def free_edges(w):
    """Indices of edges that carry a dof (PEC edges removed)."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.free_edges(w)
    n = Grid.of(w).n_edges
    if w.pec_edge is None:
        return np.arange(n)
    return np.flatnonzero(w.pec_edge == 0)


# ----------------------------------------------------------------- incident field


def incident(points, khat, pol, k):
    """E_inc = pol exp(-jk khat.r) and curl E_inc = -jk khat x E_inc at (P,3)."""
    ph = np.exp(-1j * k * (points @ khat))
    E = ph[:, None] * pol[None, :]
    curl = -1j * k * np.cross(khat[None, :], E)
    return E, curl


def rhs_planewave(w, which=None):
    """f (n_edges, nrhs): f_v = -sum_faces int U . N_v dS; bricks: 3x3
    Gauss-Legendre per outer-boundary face; tets: the 7-point rule per
    boundary triangle."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.rhs_planewave(w, which)
    g = Grid.of(w)
    which = range(w.nrhs) if which is None else which
    which = list(which)
    if g.element == "tet":
        return _rhs_planewave_tet(w, g, which)
    f = np.zeros((g.n_edges, len(which)), np.complex128)
    q, wq = gauss01(3)
    ci, cj, ck = g.cell_ijk()
    origin = np.stack([ci * g.h[0], cj * g.h[1], ck * g.h[2]], 1)
    ce_all = g.cell_edges()
    for axis, side, cid, _ in abc_faces(g, w.k):
        u, v = _FACE_PARAM[axis]
        n = np.zeros(3)
        n[axis] = 1.0 if side == 1 else -1.0
        area = g.h[u] * g.h[v]
        for a, s in enumerate(q):
            for b, t in enumerate(q):
                ref = _face_point(axis, side, s, t)
                N, _ = basis(*ref, g.h)                    # (12,3)
                pts = origin[cid] + np.asarray(ref) * g.h   # (F,3)
                for col, r in enumerate(which):
                    E, cE = incident(pts, w.khat[r], w.pol[r], w.k)
                    Et = E - np.outer(E @ n, n)
                    U = np.cross(n[None, :], cE) - 1j * w.k * Et   # (F,3)
                    contrib = -(wq[a] * wq[b] * area) * (U @ N.T)   # (F,12)
                    np.add.at(f[:, col], ce_all[cid].ravel(), contrib.ravel())
    return f


def _rhs_planewave_tet(w, g: Grid, which):
    f = np.zeros((g.n_edges, len(which)), np.complex128)
    ce_all = g.cell_edges()
    qp, qw = tri_quadrature(5)
    for axis, side, cid, _ in abc_faces(g, w.k):
        n = np.zeros(3)
        n[axis] = 1.0 if side == 1 else -1.0
        cn = g.cell_nodes(cid)
        for tri in face_triangles(axis, side):
            Q, G, area, loc, ell = _tri_setup(cn, tri)
            dofs = ce_all[cid][:, loc]
            for mu, wt in zip(qp, qw):
                pts = np.einsum("i,cid->cd", mu, Q)
                N = _whitney(mu, G, ell, _TRI_EDGES)       # (F,3,3)
                for col, r in enumerate(which):
                    E, cE = incident(pts, w.khat[r], w.pol[r], w.k)
                    Et = E - np.outer(E @ n, n)
                    U = np.cross(n[None, :], cE) - 1j * w.k * Et
                    contrib = -(wt * area)[:, None] * np.einsum("cd,ced->ce", U, N)
                    np.add.at(f[:, col], dofs.ravel(), contrib.ravel())
    return f


def edge_interpolant(w, khat, pol):
    """Line averages of E_inc . t along every edge (the exact dof of E_inc),
    computed by 4-point Gauss-Legendre along the edge."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.edge_interpolant(w, khat, pol)
    g = Grid.of(w)
    q, wq = gauss01(4)
    out = np.zeros(g.n_edges, np.complex128)
    if g.element == "tet":
        s0, s1 = g.edge_nodes()
        P0 = g.nodes[s0]
        t = g.nodes[s1] - P0
        that = t / np.linalg.norm(t, axis=1)[:, None]
        for tq, wt in zip(q, wq):
            E, _ = incident(P0 + tq * t, khat, pol, w.k)
            out += wt * np.sum(E * that, 1)
        return out
    info = g.edge_info()
    d = info[:, 0]
    start = info[:, 1:4] * g.h[None, :]
    for t, wt in zip(q, wq):
        p = start.copy()
        p[np.arange(len(d)), d] += t * g.h[d]
        E, _ = incident(p, khat, pol, w.k)
        out += wt * E[np.arange(len(d)), d]
    return out


def edge_lengths(g: Grid):
    s0, s1 = g.edge_nodes()
    return np.linalg.norm(g.nodes[s1] - g.nodes[s0], axis=1)


def discrete_gradient(g: Grid):
    """Edge-node incidence G (n_edges x n_nodes): (G phi)_e = phi(end) - phi(start)."""
    start, end = g.edge_nodes()
    rows = np.concatenate([np.arange(g.n_edges)] * 2)
    return sp.csr_matrix((np.concatenate([-np.ones(g.n_edges), np.ones(g.n_edges)]),
                          (rows, np.concatenate([start, end]))), shape=(g.n_edges, g.n_nodes))


def solve_global(w, f=None):
    """Reference solution of the undecomposed system by sparse LU (SuperLU),
    PEC dofs fixed to zero.  Returns x (n_edges, nrhs)."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.solve_global(w, f)
    import scipy.sparse.linalg as spla
    A = global_matrix(w)
    f = rhs_planewave(w) if f is None else f
    keep = free_edges(w)
    lu = spla.splu(A[keep][:, keep].tocsc())
    x = np.zeros_like(f)
    x[keep] = lu.solve(np.ascontiguousarray(f[keep]))
    return x


def rel_residual(w, x, f):
    """||A x - f||_inf / ||f||_inf per column on the free dofs (Numerical
    Results section's accuracy measure; |z| is the modulus)."""
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.rel_residual(w, x, f)
    A = global_matrix(w)
    keep = free_edges(w)
    r = A[keep][:, keep] @ x[keep] - f[keep]
    return np.abs(r).max(axis=0) / np.abs(f[keep]).max(axis=0)
