"""General tetrahedral meshes (arbitrary connectivity) -- oracle, test only.

The paper's setting is a general FEM mesh (Introduction).  A mesh here is a
list of vertex positions and a list of tetrahedra (four vertex ids each, any
orientation).  Discretisation as for the lattice tetrahedra of fem.py:

- edges: the distinct vertex pairs (i < j) of the tetrahedra in lexicographic
  order; edge (i, j) points from vertex i to vertex j, and its edge function
  is l_ij (lam_i grad lam_j - lam_j grad lam_i), so its dof is the line average
  of E . t; inside a tetrahedron with local vertices (v_a, v_b), a < b, the
  local function points from v_a to v_b and carries the sign +1 when
  v_a < v_b, else -1;
- order 2 (complete first order, hierarchical; the second-kind space of
  degree 1): each edge also carries l_ij grad(lam_i lam_j), whose tangential
  component along its own edge is 1 - 2 s / l_ij (s from i) and which has no
  curl and no orientation sign; dof 2 e is the edge's Whitney function, dof
  2 e + 1 its gradient function;
- order 3 (curl-complete second order, hierarchical; the first-kind space of
  degree 2): order 2 plus two functions per face with vertices a < b < c
  (global ids): l_ab lam_c W_ab and l_ac lam_b W_ac (W the unscaled Whitney
  function), whose tangential traces vanish on every edge and every other
  face; face dofs follow the edge dofs (2 n_edges + 2 f, + 1); element and face
  integrals by collapsed-coordinate Gauss rules exact to degree 5;
- element integrals by the degree-2 four-point rule, face integrals by the
  edge-midpoint rule (both exact here), the incident-field RHS by the 7-point
  rule per boundary triangle (fem.tri_quadrature);
- boundary triangles (faces of one tetrahedron) carry the first-order ABC
  with the outward normal of their tetrahedron.

Decomposition (Theory section, Eq. (1)), reading for general meshes: the
subdomains form a px x py x pz grid of coordinate boxes; a tetrahedron
belongs to the box holding its centroid (c_a >= g_a[i] and c_a < g_a[i + 1],
the last box closed), the centroid taken as ((v0 + v1) + v2) + v3 over 4.
Copies, the owner rule and the multiplier map follow decomp.py, except that
an extra copy with no earlier face-adjacent copy (possible on a jagged
interface) is tied to the lowest-index copy.  Interface faces are the
triangles shared by tetrahedra of two different subdomains, with the +-alpha
term of decomp.py on each side.  The interior ordering bisects the
subdomain's tetrahedra by centroid: split at the middle of the centroids'
bounding box along its longest axis (ties x < y < z; left: centroid below the
middle); the still unassigned edges of both halves form the separator;
left, right, separator; a region of at most leaf_max unassigned edges (or
one that does not split) is a leaf; inside a node edges follow the global
index.

Pins (tests/test_oracle_tetmesh.py): a lattice-tetrahedral workload passed
as a general mesh gives the lattice path's solution edge for edge (two
independent numberings and assemblies), the Whitney energy identities on a
Delaunay mesh, S G = 0, D3M = global on Delaunay meshes, the adjoint
gradient against central differences.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem

PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
TRI = [(0, 1), (0, 2), (1, 2)]
_FACE_OF = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]   # face q omits vertex q


class MeshGrid:
    """Topology and geometry of a general tetrahedral mesh; n_edges counts
    the dofs (order per edge), n_geo the edges themselves."""

    element = "mesh"

    def __init__(self, vertices, tets, order=1):
        self.V = np.asarray(vertices, np.float64)
        self.T = np.asarray(tets, np.int64)
        self.order = int(order)
        if self.order not in (1, 2, 3):
            raise ValueError("order must be 1, 2 or 3")
        nt = len(self.T)
        self.n_nodes = len(self.V)
        self.n_cells = nt
        loc = np.stack([np.sort(self.T[:, [a, b]], axis=1) for a, b in PAIRS], 1)
        self.edges, inv = np.unique(loc.reshape(-1, 2), axis=0, return_inverse=True)
        self.n_geo = len(self.edges)
        self.tet_edges = inv.reshape(nt, 6)
        fl = np.stack([np.sort(self.T[:, list(f)], axis=1) for f in _FACE_OF], 1).reshape(-1, 3)
        self.faces, finv, cnt = np.unique(fl, axis=0, return_inverse=True, return_counts=True)
        finv = finv.ravel()
        self.tet_faces = finv.reshape(nt, 4)
        # local vertex indices of each face, sorted by global id
        self.face_loc = np.stack([np.array(f)[np.argsort(self.T[:, list(f)], axis=1)] for f in _FACE_OF], 1)
        sg = np.stack([np.where(self.T[:, a] < self.T[:, b], 1.0, -1.0) for a, b in PAIRS], 1)
        dpe = min(self.order, 2)
        self.dpe = dpe
        self.n_edges = dpe * self.n_geo + (2 * len(self.faces) if self.order == 3 else 0)   # dofs
        if self.order == 1:
            self.tet_dofs, self.tet_sign = self.tet_edges, sg
            self.tet_ents = self.tet_edges
        else:
            self.tet_dofs = np.concatenate([2 * self.tet_edges, 2 * self.tet_edges + 1], 1)
            self.tet_sign = np.concatenate([sg, np.ones_like(sg)], 1)
            self.tet_ents = self.tet_edges
        if self.order == 3:
            fd = 2 * self.n_geo + 2 * self.tet_faces
            self.tet_dofs = np.concatenate([self.tet_dofs, np.stack([fd, fd + 1], 2).reshape(nt, 8)], 1)
            self.tet_sign = np.concatenate([self.tet_sign, np.ones((nt, 8))], 1)
            self.tet_ents = np.concatenate([self.tet_edges, self.n_geo + self.tet_faces], 1)
        owner = np.repeat(np.arange(nt), 4)
        opp = self.T.ravel()                  # the vertex each face omits
        order = np.argsort(finv, kind="stable")
        first = np.searchsorted(finv[order], np.arange(len(self.faces)))
        self.face_tets = -np.ones((len(self.faces), 2), np.int64)
        self.face_opp = np.zeros(len(self.faces), np.int64)
        for f in range(len(self.faces)):
            k = first[f]
            self.face_tets[f, 0] = owner[order[k]]
            self.face_opp[f] = opp[order[k]]
            if cnt[f] == 2:
                self.face_tets[f, 1] = owner[order[k + 1]]
        X = self.V[self.T]
        self.centroids = (((X[:, 0] + X[:, 1]) + X[:, 2]) + X[:, 3]) / 4.0

    def edge_id(self, i, j):
        key = self.edges[:, 0] * self.n_nodes + self.edges[:, 1]
        return np.searchsorted(key, np.asarray(i) * self.n_nodes + np.asarray(j))

    def ent_dofs(self, E):
        """Dofs of entities E (edges e < n_geo, faces n_geo + f), in order."""
        E = np.asarray(E, np.int64)
        if self.order == 1:
            return E
        d = np.where(E < self.n_geo, 2 * E, 2 * self.n_geo + 2 * (E - self.n_geo))
        return np.stack([d, d + 1], 1).ravel()

    def dof_ent(self, D):
        """Entity of each dof."""
        D = np.asarray(D, np.int64)
        if self.order == 1:
            return D
        return np.where(D < 2 * self.n_geo, D // 2, self.n_geo + (D - 2 * self.n_geo) // 2)


def grid_of(w) -> MeshGrid:
    return MeshGrid(w.vertices, w.tets, getattr(w, "order", 1))


def _basis(lam, G, ell, pairs, order):
    """Edge functions at barycentric point lam: the Whitney functions of the
    pairs, then (order >= 2) the gradient functions: (n, dpe * len(pairs), 3)."""
    N = [np.stack([lam[a] * G[:, b] - lam[b] * G[:, a] for a, b in pairs], 1) * ell[..., None]]
    if order >= 2:
        N.append(np.stack([lam[a] * G[:, b] + lam[b] * G[:, a] for a, b in pairs], 1) * ell[..., None])
    return np.concatenate(N, 1)


def duffy_tet(n):
    """Collapsed-coordinate Gauss rule on a tetrahedron: x = u, y = v (1 - u),
    z = w (1 - u)(1 - v) with n Gauss-Legendre points per direction (exact to
    degree 2 n - 3); barycentric points (n^3, 4), weights as fractions of the
    volume."""
    q, wq = fem.gauss01(n)
    P, Wt = [], []
    for i, u in enumerate(q):
        for j, v in enumerate(q):
            for k, t in enumerate(q):
                x, y, z = u, v * (1 - u), t * (1 - u) * (1 - v)
                P.append([1 - x - y - z, x, y, z])
                Wt.append(6.0 * wq[i] * wq[j] * wq[k] * (1 - u) ** 2 * (1 - v))
    return np.array(P), np.array(Wt)


def duffy_tri(n):
    """The same on a triangle: x = u, y = v (1 - u) (exact to degree 2 n - 2);
    barycentric points (n^2, 3), weights as fractions of the area."""
    q, wq = fem.gauss01(n)
    P, Wt = [], []
    for i, u in enumerate(q):
        for j, v in enumerate(q):
            x, y = u, v * (1 - u)
            P.append([1 - x - y, x, y])
            Wt.append(2.0 * wq[i] * wq[j] * (1 - u))
    return np.array(P), np.array(Wt)


def _face_fns(lam, G, X, A, B, C):
    """The two face functions of a face with vertices A < B < C (global order;
    local indices per simplex) and their curls at barycentric point lam:
    l_AB lam_C W_AB and l_AC lam_B W_AC.  X: vertex positions (n, k, 3)."""
    r = np.arange(len(A))
    la, lb, lc = lam[A], lam[B], lam[C]
    ga, gb, gc = G[r, A], G[r, B], G[r, C]
    lab = np.linalg.norm(X[r, B] - X[r, A], axis=1)[:, None]
    lac = np.linalg.norm(X[r, C] - X[r, A], axis=1)[:, None]
    wab = la[:, None] * gb - lb[:, None] * ga
    wac = la[:, None] * gc - lc[:, None] * ga
    f1, f2 = lab * lc[:, None] * wab, lac * lb[:, None] * wac
    c1 = lab * (np.cross(gc, wab) + 2.0 * lc[:, None] * np.cross(ga, gb))
    c2 = lac * (np.cross(gb, wac) + 2.0 * lb[:, None] * np.cross(ga, gc))
    return f1, f2, c1, c2


def _tet_basis3(g, lam, G, X, ell, tets):
    """Order 3: the 20 functions of each tetrahedron and their curls at
    barycentric point lam (edge functions, then two per face)."""
    N = _basis(lam, G, ell, PAIRS, 3)
    Cw = np.stack([2.0 * np.cross(G[:, a], G[:, b]) for a, b in PAIRS], 1) * ell[..., None]
    C = [Cw, np.zeros_like(Cw)]
    Nf = [N]
    fl = g.face_loc[tets]
    for q in range(4):
        f1, f2, c1, c2 = _face_fns(lam, G, X, fl[:, q, 0], fl[:, q, 1], fl[:, q, 2])
        Nf.append(np.stack([f1, f2], 1))
        C.append(np.stack([c1, c2], 1))
    return np.concatenate(Nf, 1), np.concatenate(C, 1)


# ------------------------------------------------------------------ elements


def tet_matrices(g: MeshGrid, tets):
    """S and M (n, 6 order, 6 order) of the given tetrahedra (the Whitney
    functions in PAIRS order, then the gradient functions), signs of the
    global edge orientation applied."""
    tets = np.asarray(tets)
    X = g.V[g.T[tets]]
    G, vol = fem.tet_barycentric(X)
    vol = np.abs(vol)
    ell = np.stack([np.linalg.norm(X[:, b] - X[:, a], axis=1) for a, b in PAIRS], 1)
    if g.order == 3:
        nl = 20
        S = np.zeros((len(tets), nl, nl))
        M = np.zeros_like(S)
        qp, qw = duffy_tet(4)
        for lam, wt in zip(qp, qw):
            N, C = _tet_basis3(g, lam, G, X, ell, tets)
            M += wt * vol[:, None, None] * np.einsum("cid,cjd->cij", N, N)
            S += wt * vol[:, None, None] * np.einsum("cid,cjd->cij", C, C)
        sg = g.tet_sign[tets]
        sgn = sg[:, :, None] * sg[:, None, :]
        return S * sgn, M * sgn
    curl = np.stack([2.0 * np.cross(G[:, a], G[:, b]) for a, b in PAIRS], 1) * ell[..., None]
    if g.order == 2:
        curl = np.concatenate([curl, np.zeros_like(curl)], 1)   # gradients have no curl
    S = vol[:, None, None] * np.einsum("cid,cjd->cij", curl, curl)
    M = np.zeros_like(S)
    qp, qw = fem.tet_quadrature()
    for lam, wt in zip(qp, qw):
        N = _basis(lam, G, ell, PAIRS, g.order)
        M += wt * vol[:, None, None] * np.einsum("cid,cjd->cij", N, N)
    sg = g.tet_sign[tets]
    sgn = sg[:, :, None] * sg[:, None, :]
    return S * sgn, M * sgn


def _tri(g: MeshGrid, faces):
    Q = g.V[g.faces[faces]]
    G, area = fem.tri_frame(Q)
    ell = np.stack([np.linalg.norm(Q[:, b] - Q[:, a], axis=1) for a, b in TRI], 1)
    ids = np.stack([g.edge_id(g.faces[faces, a], g.faces[faces, b]) for a, b in TRI], 1)
    if g.order >= 2:
        ids = np.concatenate([2 * ids, 2 * ids + 1], 1)
    if g.order == 3:
        fd = 2 * g.n_geo + 2 * np.asarray(faces)
        ids = np.concatenate([ids, fd[:, None], fd[:, None] + 1], 1)
    return Q, G, area, ell, ids


def _tri_basis(g, mu, G, Q, ell):
    """Tangential traces on a triangle (sorted vertices): Whitney, gradient
    and (order 3) the face's two functions."""
    N = _basis(mu, G, ell, TRI, g.order)
    if g.order == 3:
        z = np.zeros(len(Q), np.int64)
        f1, f2, _, _ = _face_fns(mu, G, Q, z, z + 1, z + 2)
        N = np.concatenate([N, f1[:, None], f2[:, None]], 1)
    return N


def face_matrices(g: MeshGrid, faces):
    """Tangential face mass (n, 3 order, 3 order) of the given faces (TRI
    order of the sorted vertices, every local edge along its global
    orientation; then the gradient functions) and the global dof ids."""
    faces = np.asarray(faces)
    Q, G, area, ell, ids = _tri(g, faces)
    T = np.zeros((len(faces), ids.shape[1], ids.shape[1]))
    qp, qw = fem.tri_quadrature(2) if g.order < 3 else duffy_tri(3)
    for mu, wt in zip(qp, qw):
        N = _tri_basis(g, mu, G, Q, ell)
        T += wt * area[:, None, None] * np.einsum("cid,cjd->cij", N, N)
    return T, ids


def boundary_faces(g: MeshGrid):
    return np.flatnonzero(g.face_tets[:, 1] < 0)


def outward_normals(g: MeshGrid, faces):
    Q = g.V[g.faces[faces]]
    n = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    inward = np.einsum("ij,ij->i", n, g.V[g.face_opp[faces]] - Q[:, 0]) > 0
    n[inward] *= -1.0
    return n


def assemble(g: MeshGrid, eps, k, tets=None, faces=()):
    """COO pieces of S - k^2 sum eps_t M_t over the given tetrahedra plus
    coeff * T_f for each (face ids, coeff) in faces."""
    tets = np.arange(g.n_cells) if tets is None else np.asarray(tets)
    S, M = tet_matrices(g, tets)
    ce = g.tet_dofs[tets]
    nl = ce.shape[1]
    R = [np.repeat(ce, nl, axis=1).ravel()]
    C = [np.tile(ce, (1, nl)).ravel()]
    V = [(S.reshape(len(tets), nl * nl) - (k * k) * eps[tets][:, None] * M.reshape(len(tets), nl * nl))
         .ravel().astype(np.complex128)]
    for fids, coeff in faces:
        fids = np.asarray(fids)
        if len(fids) == 0:
            continue
        T, ids = face_matrices(g, fids)
        nf = ids.shape[1]
        R.append(np.repeat(ids, nf, axis=1).ravel())
        C.append(np.tile(ids, (1, nf)).ravel())
        V.append((coeff * T.reshape(len(fids), nf * nf)).ravel().astype(np.complex128))
    return np.concatenate(R), np.concatenate(C), np.concatenate(V)


def mass_stiffness(g: MeshGrid):
    S, M = tet_matrices(g, np.arange(g.n_cells))
    ce = g.tet_dofs
    nl = ce.shape[1]
    r, c = np.repeat(ce, nl, axis=1).ravel(), np.tile(ce, (1, nl)).ravel()
    shape = (g.n_edges, g.n_edges)
    return sp.csr_matrix((S.ravel(), (r, c)), shape=shape), sp.csr_matrix((M.ravel(), (r, c)), shape=shape)


def global_matrix(w):
    g = grid_of(w)
    r, c, v = assemble(g, w.eps, w.k, faces=[(boundary_faces(g), 1j * w.k)])
    return sp.csr_matrix((v, (r, c)), shape=(g.n_edges, g.n_edges))


def rhs_planewave(w, which=None):
    """f (n_edges, nrhs): f_v = -int U . N_v dS over the boundary triangles."""
    g = grid_of(w)
    which = list(range(w.nrhs) if which is None else which)
    f = np.zeros((g.n_edges, len(which)), np.complex128)
    bf = boundary_faces(g)
    n = outward_normals(g, bf)
    Q, G, area, ell, ids = _tri(g, bf)
    qp, qw = fem.tri_quadrature(5)
    for mu, wt in zip(qp, qw):
        pts = np.einsum("i,cid->cd", mu, Q)
        N = _tri_basis(g, mu, G, Q, ell)
        for col, r in enumerate(which):
            E, cE = fem.incident(pts, w.khat[r], w.pol[r], w.k)
            Et = E - np.einsum("cd,cd->c", E, n)[:, None] * n
            U = np.cross(n, cE) - 1j * w.k * Et
            contrib = -(wt * area)[:, None] * np.einsum("cd,ced->ce", U, N)
            np.add.at(f[:, col], ids.ravel(), contrib.ravel())
    return f


def edge_interpolant(w, khat, pol):
    """Dofs of E_inc: the line average of E . t along every edge and (order
    2) the moment 3 <E . t (1 - 2 s / l)> (the projection onto the edge's
    linear tangential variation), 4-point Gauss-Legendre along the edge."""
    g = grid_of(w)
    if g.order == 3:
        raise NotImplementedError("order 3: use an L2 projection (face moments are not defined here)")
    P0, P1 = g.V[g.edges[:, 0]], g.V[g.edges[:, 1]]
    t = P1 - P0
    that = t / np.linalg.norm(t, axis=1)[:, None]
    q, wq = fem.gauss01(4)
    avg = np.zeros(g.n_geo, np.complex128)
    mom = np.zeros(g.n_geo, np.complex128)
    for tq, wt in zip(q, wq):
        E, _ = fem.incident(P0 + tq * t, khat, pol, w.k)
        et = np.sum(E * that, 1)
        avg += wt * et
        mom += wt * et * (1.0 - 2.0 * tq)
    if g.order == 1:
        return avg
    out = np.zeros(g.n_edges, np.complex128)
    out[0::2], out[1::2] = avg, 3.0 * mom
    return out


def edge_lengths(g: MeshGrid):
    return np.linalg.norm(g.V[g.edges[:, 1]] - g.V[g.edges[:, 0]], axis=1)


def discrete_gradient(g: MeshGrid):
    """Edge-node incidence (geometric edges x nodes)."""
    ne = g.n_geo
    rows = np.concatenate([np.arange(ne)] * 2)
    return sp.csr_matrix((np.concatenate([-np.ones(ne), np.ones(ne)]),
                          (rows, np.concatenate([g.edges[:, 0], g.edges[:, 1]]))), shape=(ne, g.n_nodes))


# ------------------------------------------------------------- decomposition


def subdomain_of(w, g: MeshGrid):
    """Subdomain index of every tetrahedron (centroid rule) and the grid size."""
    parts = tuple(len(c) - 1 for c in w.gcuts)
    ix = [np.searchsorted(np.asarray(w.gcuts[a], np.float64)[1:-1], g.centroids[:, a], side="right")
          for a in range(3)]
    return ix[0] + parts[0] * (ix[1] + parts[1] * ix[2]), parts


def decompose(w, with_matrices=True):
    from . import decomp, ordering
    if int(getattr(w, "lm_weight", 0) or 0):
        raise NotImplementedError("the mass-weighted multiplier map is for lattice meshes")
    g = grid_of(w)
    sub, parts = subdomain_of(w, g)
    nsub = parts[0] * parts[1] * parts[2]
    if np.bincount(sub, minlength=nsub).min() == 0:
        raise ValueError("a subdomain box holds no tetrahedron")
    free = np.ones(g.n_edges, bool)
    if w.pec_edge is not None:   # one byte per dof
        free[np.asarray(w.pec_edge) != 0] = False
    subs = []
    for s in range(nsub):
        tets = np.flatnonzero(sub == s)
        e = np.unique(g.tet_dofs[tets].ravel()) if len(tets) else np.zeros(0, np.int64)
        sd = decomp.Subdomain(s, decomp.sub_pos(s, parts), None, None, e[free[e]])
        sd.tets = tets
        subs.append(sd)
    copies = {}
    for sd in subs:
        for e in sd.edges:
            copies.setdefault(int(e), []).append(sd.index)
    pairs = {}
    for e in sorted(copies):
        cs = copies[e]
        for kk in range(1, len(cs)):
            sk = cs[kk]
            sj = next((cs[j] for j in range(kk) if decomp.face_adjacent(cs[j], sk, parts)), cs[0])
            pairs.setdefault((sj, sk), []).append(e)
    block_order = ordering.block_nested_dissection(parts, set(pairs))
    lm_edge, lm_plus, lm_minus, block_lms = [], [], [], []
    for (a, b) in block_order:
        es = sorted(pairs[(a, b)])
        block_lms.append(np.arange(len(lm_edge), len(lm_edge) + len(es)))
        lm_edge += es
        lm_plus += [a] * len(es)
        lm_minus += [b] * len(es)
    dec = decomp.Decomposition(g, parts, subs, copies, np.array(lm_edge, np.int64),
                               np.array(lm_plus, np.int64), np.array(lm_minus, np.int64),
                               list(block_order), block_lms, 0)
    dec.tet_sub = sub
    if with_matrices:
        for sd in subs:
            sd.A = subdomain_matrix(w, dec, sd)
    return dec


def subdomain_faces(w, dec, sd, alpha):
    """[(face ids, coeff)] of subdomain sd: ABC on its boundary triangles,
    +-alpha on the triangles it shares with another subdomain."""
    g = dec.grid
    mine = np.zeros(g.n_cells, bool)
    mine[sd.tets] = True
    t0, t1 = g.face_tets[:, 0], g.face_tets[:, 1]
    out = [(np.flatnonzero((t1 < 0) & mine[t0]), 1j * w.k)]
    other = np.where(mine[t0], t1, t0)
    inter = (t1 >= 0) & (mine[t0] ^ mine[np.maximum(t1, 0)])
    nb = dec.tet_sub[other]
    out.append((np.flatnonzero(inter & (nb > sd.index)), alpha))
    out.append((np.flatnonzero(inter & (nb < sd.index)), -alpha))
    return out


def subdomain_matrix(w, dec, sd):
    g = dec.grid
    alpha = 1j * w.k if getattr(w, "alpha", None) is None else complex(w.alpha)
    r, c, v = assemble(g, w.eps, w.k, tets=sd.tets, faces=subdomain_faces(w, dec, sd, alpha))
    loc = -np.ones(g.n_edges, np.int64)
    loc[sd.edges] = np.arange(len(sd.edges))
    keep = (loc[r] >= 0) & (loc[c] >= 0)
    n = len(sd.edges)
    return sp.csr_matrix((v[keep], (loc[r[keep]], loc[c[keep]])), shape=(n, n))


def subdomain_nd(g: MeshGrid, sd, interface_edges, leaf_max):
    """ND nodes (sorted global dof arrays, post-order) of the non-interface
    dofs of sd: centroid bisection over the entities carrying dofs (edges;
    at order 3 also faces, after all edges) (module docstring); an entity's
    dofs stay together."""
    n_ent = g.n_geo + (len(g.faces) if g.order == 3 else 0)
    avail = np.zeros(n_ent, bool)
    avail[g.dof_ent(sd.edges)] = True
    avail[g.dof_ent(np.asarray(sorted(interface_edges), dtype=np.int64))] = False
    nodes = []
    ents = g.tet_ents

    def dofs(E):
        return g.ent_dofs(E)

    def leaf(E):
        if len(E):
            avail[E] = False
            nodes.append(dofs(E))

    def rec(T):
        E = np.unique(ents[T].ravel()) if len(T) else np.zeros(0, np.int64)
        E = E[avail[E]]
        if len(E) <= leaf_max or len(T) < 2:
            return leaf(E)
        c = g.centroids[T]
        lo, hi = c.min(axis=0), c.max(axis=0)
        axis = int(np.argmax(hi - lo))
        mid = (lo[axis] + hi[axis]) / 2.0
        below = c[:, axis] < mid
        left, right = T[below], T[~below]
        if len(left) == 0 or len(right) == 0:
            return leaf(E)
        sep = np.intersect1d(ents[left].ravel(), ents[right].ravel())
        sep = sep[avail[sep]]
        avail[sep] = False
        rec(left)
        rec(right)
        if len(sep):
            nodes.append(dofs(np.sort(sep)))

    rec(np.asarray(sd.tets, np.int64))
    return nodes


# ------------------------------------------------------------------ solves


def free_edges(w):
    g = grid_of(w)
    if w.pec_edge is None:
        return np.arange(g.n_edges)
    return np.flatnonzero(np.asarray(w.pec_edge) == 0)


def solve_global(w, f=None):
    import scipy.sparse.linalg as spla
    A = global_matrix(w)
    f = rhs_planewave(w) if f is None else f
    keep = free_edges(w)
    lu = spla.splu(A[keep][:, keep].tocsc())
    x = np.zeros_like(f)
    x[keep] = lu.solve(np.ascontiguousarray(f[keep]))
    return x


def rel_residual(w, x, f):
    A = global_matrix(w)
    keep = free_edges(w)
    r = A[keep][:, keep] @ x[keep] - f[keep]
    return np.abs(r).max(axis=0) / np.abs(f[keep]).max(axis=0)
