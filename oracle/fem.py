"""FEM discretisation of the paper's BVP (Theory section) -- oracle, test only.

    curl(curl E) - k^2 eps_r E = 0 in Omega   (mu_r = 1, J_imp = 0)
    n x curl E - jk E_t = n x curl E_inc - jk E_inc,t   on dOmega (1st-order ABC)

Weak form with outward normal n and time convention e^{jwt}:
    A x = f,  A = S - k^2 sum_c eps_c M_c + jk T,   f_v = -int_dOmega U . N_v dS,
    U = n x curl E_inc - jk (E_inc)_t.
A is complex symmetric (A = A^T, stated for K in the paper's discussion of
LDL^T).  Lowest-order Nedelec brick elements on an axis-aligned grid; element
integrals by tensor Gauss-Legendre quadrature (2 points per axis is exact for
the bilinear-by-linear integrands; the incident-field RHS uses 3x3 points per
face, a stated reading because the paper gives no quadrature).

Global edge numbering: x-edges, then y-edges, then z-edges; within each
family the start node (i, j, k) runs x-fastest over that family's box.  Every
edge points along +axis.

Pins (tests/test_oracle_fem.py): S G = 0 for the discrete gradient, M SPD,
1-D mass factors h/3, h/6, constant-field mass = eps * volume, A = A^T,
plane-wave convergence in a homogeneous box, reciprocity.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------- numbering


class Grid:
    """Axis-aligned brick grid [0,lx]x[0,ly]x[0,lz] with nx*ny*nz cells."""

    def __init__(self, nx, ny, nz, lx, ly, lz):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.ly, self.lz = float(lx), float(ly), float(lz)
        self.h = np.array([lx / nx, ly / ny, lz / nz])
        self.nex = nx * (ny + 1) * (nz + 1)
        self.ney = (nx + 1) * ny * (nz + 1)
        self.nez = (nx + 1) * (ny + 1) * nz
        self.n_edges = self.nex + self.ney + self.nez
        self.n_cells = nx * ny * nz

    @classmethod
    def of(cls, w):
        return cls(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)

    # edge ids from start-node indices (vectorised)
    def ex(self, i, j, k):
        return i + self.nx * (j + (self.ny + 1) * k)

    def ey(self, i, j, k):
        return self.nex + i + (self.nx + 1) * (j + self.ny * k)

    def ez(self, i, j, k):
        return self.nex + self.ney + i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def edge_info(self):
        """(direction 0/1/2, i, j, k) of every edge, as int arrays."""
        nx, ny, nz = self.nx, self.ny, self.nz
        out = []
        for d, (sx, sy, sz) in enumerate([(nx, ny + 1, nz + 1), (nx + 1, ny, nz + 1),
                                          (nx + 1, ny + 1, nz)]):
            kk, jj, ii = np.meshgrid(np.arange(sz), np.arange(sy), np.arange(sx), indexing="ij")
            out.append(np.stack([np.full(ii.size, d), ii.ravel(), jj.ravel(), kk.ravel()], 1))
        return np.concatenate(out, 0)

    def cell_ijk(self):
        kk, jj, ii = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                                 indexing="ij")
        return ii.ravel(), jj.ravel(), kk.ravel()

    def cell_edges(self, ci=None, cj=None, ck=None):
        """(ncells, 12) global edges of each cell in local order:
        x-edges (dy, dz) = (0,0),(1,0),(0,1),(1,1); y-edges (dx, dz) likewise;
        z-edges (dx, dy) likewise."""
        if ci is None:
            ci, cj, ck = self.cell_ijk()
        o = [(0, 0), (1, 0), (0, 1), (1, 1)]
        cols = [self.ex(ci, cj + a, ck + b) for a, b in o]
        cols += [self.ey(ci + a, cj, ck + b) for a, b in o]
        cols += [self.ez(ci + a, cj + b, ck) for a, b in o]
        return np.stack(cols, 1).astype(np.int64)


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
    S_e, M_e = element_matrices(g.h)
    cells = np.arange(g.n_cells) if cells is None else np.asarray(cells)
    ce = g.cell_edges()[cells]
    rows = np.repeat(ce, 12, axis=1).ravel()
    cols = np.tile(ce, (1, 12)).ravel()
    vals = (S_e.ravel()[None, :] - (k * k) * eps[cells][:, None] * M_e.ravel()[None, :]).ravel()
    R, C, V = [rows], [cols], [vals.astype(np.complex128)]
    for axis, side, cid, coeff in extra_faces:
        T = face_matrix(g.h, axis, side)
        ce = g.cell_edges()[cid]
        R.append(np.repeat(ce, 12, axis=1).ravel())
        C.append(np.tile(ce, (1, 12)).ravel())
        V.append(np.broadcast_to(coeff * T.ravel(), (len(cid), 144)).ravel().astype(np.complex128))
    return np.concatenate(R), np.concatenate(C), np.concatenate(V)


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
    g = Grid.of(w)
    r, c, v = assemble(g, w.eps, w.k, extra_faces=abc_faces(g, w.k))
    return sp.csr_matrix((v, (r, c)), shape=(g.n_edges, g.n_edges))


def free_edges(w):
    """Indices of edges that carry a dof (PEC edges removed)."""
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
    """f (n_edges, nrhs): f_v = -sum_faces int U . N_v dS, 3x3 Gauss-Legendre
    per outer-boundary face."""
    g = Grid.of(w)
    which = range(w.nrhs) if which is None else which
    which = list(which)
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


def edge_interpolant(w, khat, pol):
    """Line averages of E_inc along every edge (the exact dof of E_inc),
    computed by 4-point Gauss-Legendre along the edge."""
    g = Grid.of(w)
    info = g.edge_info()
    d = info[:, 0]
    start = info[:, 1:4] * g.h[None, :]
    q, wq = gauss01(4)
    out = np.zeros(g.n_edges, np.complex128)
    for t, wt in zip(q, wq):
        p = start.copy()
        p[np.arange(len(d)), d] += t * g.h[d]
        E, _ = incident(p, khat, pol, w.k)
        out += wt * E[np.arange(len(d)), d]
    return out


def discrete_gradient(g: Grid):
    """Edge-node incidence G (n_edges x n_nodes): (G phi)_e = phi(end) - phi(start)."""
    info = g.edge_info()
    d, i, j, k = info.T
    nid = lambda i, j, k: i + (g.nx + 1) * (j + (g.ny + 1) * k)
    start = nid(i, j, k)
    end = nid(i + (d == 0), j + (d == 1), k + (d == 2))
    n_nodes = (g.nx + 1) * (g.ny + 1) * (g.nz + 1)
    rows = np.concatenate([np.arange(g.n_edges)] * 2)
    return sp.csr_matrix((np.concatenate([-np.ones(g.n_edges), np.ones(g.n_edges)]),
                          (rows, np.concatenate([start, end]))), shape=(g.n_edges, n_nodes))


def solve_global(w, f=None):
    """Reference solution of the undecomposed system by sparse LU (SuperLU),
    PEC dofs fixed to zero.  Returns x (n_edges, nrhs)."""
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
    A = global_matrix(w)
    keep = free_edges(w)
    r = A[keep][:, keep] @ x[keep] - f[keep]
    return np.abs(r).max(axis=0) / np.abs(f[keep]).max(axis=0)
