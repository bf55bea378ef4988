"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Both the CPU oracle and the CUDA path draw their inputs from this module and
from nowhere else.  Units: free-space wavelength 1, so k = 2*pi.  The five
workloads mirror the paper's test geometries (Numerical Results: PEC plates and
dielectric spheres of growing electrical size) with brick meshes:

  1  unit cube 12^3, sphere r=0.25 eps=4, 2x2x1 equal subdomains, 1 plane wave
  2  3-wavelength cube 32^3, lossy sphere eps=4-0.1j (r = L/4), 4x4x2 jittered
     subdomains, 64 plane waves on a seeded 8x8 angle grid
  3  2-wavelength cube 20^3, per-cell eps ~ U[1,3], 2x2x2 equal subdomains,
     1 plane wave, 16 probe edges and 20 finite-difference cells
  4  4x4x2-wavelength box 48x48x24 with a centred 2x2-wavelength PEC plate
     (tangential edges removed), 4x4x2 jittered subdomains, 8 plane waves
  5  6-wavelength cube 64^3, sphere r = L/4 with per-cell eps' ~ U[2,6] and
     loss tangent 0.01, 4x4x4 jittered subdomains, 128 plane waves

Random draws, in this order, from numpy.random.default_rng(seed): interior
cut jitter (x cuts, then y, then z; integers in [-3, 3]), per-cell
permittivities, plane-wave angles and polarisations, probe edges, FD cells.

delaunay() makes an unstructured tetrahedral mesh of a box (general
connectivity: vertex positions and vertex ids per tetrahedron), as_mesh()
passes a lattice-tetrahedral workload in that general form.

tetrahedral(w) turns any of them into a tetrahedral mesh of the same cells
(the general FEM setting of the paper's Introduction): each cell is split into
six tetrahedra along its (0,0,0)-(1,1,1) diagonal, and the lattice vertices
are moved by a seeded uniform jitter of up to +-jitter*h per axis (vertices on
the outer boundary move only within their boundary planes).

Edge families (global numbering, family after family, each x-fastest over the
start nodes (i, j, k) of its own box): directions (1,0,0), (0,1,0), (0,0,1)
on brick meshes; tetrahedral meshes add the face diagonals (1,1,0), (1,0,1),
(0,1,1) and the cell diagonal (1,1,1).  Every edge points from its start node
to start + direction.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

K0 = 2.0 * math.pi  # free-space wavenumber for wavelength 1

EDGE_DIRS = {"brick": ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
             "tet": ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1))}


def family_sizes(nx, ny, nz, element="brick"):
    """Number of edges in each edge family of the mesh (see the module docstring)."""
    return [(nx + 1 - d[0]) * (ny + 1 - d[1]) * (nz + 1 - d[2]) for d in EDGE_DIRS[element]]


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    k: float
    eps: np.ndarray            # complex128, n_cells, x-fastest (i + nx*(j + ny*k))
    pec_edge: np.ndarray | None  # uint8 per global edge (1 = removed) or None
    cx: np.ndarray             # int32 cut cell indices, length px+1, 0..nx
    cy: np.ndarray
    cz: np.ndarray
    khat: np.ndarray           # (nrhs, 3) unit propagation directions
    pol: np.ndarray            # (nrhs, 3) complex polarisations, pol . khat = 0
    probes: np.ndarray | None = None    # int64 global edge ids (objective)
    fd_cells: np.ndarray | None = None  # int64 cell ids (finite differences)
    seed: int = 0
    alpha: complex | None = None  # interface loss/gain coefficient (None: jk)
    lm_weight: int = 0            # multiplier map D: 0 signed Boolean, 1 tangential-face-mass weighted
    element: str = "brick"        # "brick", "tet" (six tetrahedra per cell) or "mesh"
    vertices: np.ndarray | None = None  # (n_nodes, 3) float64 positions (x-fastest for "tet"); None: lattice
    tets: np.ndarray | None = None      # "mesh": (n_tets, 4) int64 vertex ids
    gcuts: tuple | None = None          # "mesh": subdomain cut coordinates per axis (px+1, py+1, pz+1)
    order: int = 1                      # "mesh": 1 Whitney; 2 also the edge gradient functions (2 dofs per edge);
                                        # 3 also two functions per face

    @property
    def n_cells(self) -> int:
        if self.element == "mesh":
            return len(self.tets)
        return self.nx * self.ny * self.nz

    @property
    def n_edges(self) -> int:
        if self.element == "mesh":
            ne = len(mesh_edge_pairs(self.tets))
            if self.order == 3:
                return 2 * ne + 2 * len(mesh_face_triples(self.tets))
            return self.order * ne
        return sum(family_sizes(self.nx, self.ny, self.nz, self.element))

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def nrhs(self) -> int:
        return self.khat.shape[0]

    @property
    def partition(self) -> tuple[int, int, int]:
        if self.element == "mesh":
            return tuple(len(g) - 1 for g in self.gcuts)
        return len(self.cx) - 1, len(self.cy) - 1, len(self.cz) - 1

    def khat_pol6(self) -> np.ndarray:
        """(nrhs, 9) float64 rows: 3 direction components, then the complex
        polarisation as (re x, im x, re y, im y, re z, im z)."""
        out = np.zeros((self.nrhs, 9))
        out[:, :3] = self.khat
        out[:, 3::2] = self.pol.real
        out[:, 4::2] = self.pol.imag
        return out


def cuts(n: int, p: int, rng: np.random.Generator | None, jit: int = 3) -> np.ndarray:
    """Cut cell indices round(i n / p) (+ jitter in [-jit, jit] when rng is given)."""
    c = [0]
    for i in range(1, p):
        v = int(round(i * n / p))
        if rng is not None:
            v += int(rng.integers(-jit, jit + 1))
        c.append(v)
    c.append(n)
    c = np.asarray(c, dtype=np.int32)
    if np.any(np.diff(c) < 1):
        raise ValueError(f"degenerate cuts {c}")
    return c


def _angles_to_waves(theta, phi, psi):
    st, ct, sp_, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    khat = np.stack([st * cp, st * sp_, ct], axis=1)
    th_hat = np.stack([ct * cp, ct * sp_, -st], axis=1)
    ph_hat = np.stack([-sp_, cp, np.zeros_like(phi)], axis=1)
    pol = np.cos(psi)[:, None] * th_hat + np.sin(psi)[:, None] * ph_hat
    return khat, pol.astype(np.complex128)


def _grid_waves(rng, nth, nph):
    u, v = rng.random(), rng.random()
    th = (np.arange(nth) + u) * math.pi / nth
    ph = (np.arange(nph) + v) * 2 * math.pi / nph
    theta = np.repeat(th, nph)
    phi = np.tile(ph, nth)
    psi = rng.random(nth * nph) * 2 * math.pi
    return _angles_to_waves(theta, phi, psi)


def _random_waves(rng, n):
    ct = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2 * math.pi, n)
    psi = rng.uniform(0.0, 2 * math.pi, n)
    return _angles_to_waves(np.arccos(ct), phi, psi)


def with_waves(w: Workload, n: int, seed: int = 0) -> Workload:
    """A copy of w with n seeded random plane waves as its right-hand sides."""
    khat, pol = _random_waves(np.random.default_rng(seed), n)
    return dataclasses.replace(w, khat=khat, pol=pol)


def _cell_centres(nx, ny, nz, lx, ly, lz):
    i = (np.arange(nx) + 0.5) * lx / nx
    j = (np.arange(ny) + 0.5) * ly / ny
    k = (np.arange(nz) + 0.5) * lz / nz
    kk, jj, ii = np.meshgrid(k, j, i, indexing="ij")
    return ii.ravel(), jj.ravel(), kk.ravel()   # x-fastest order


def _sphere_mask(nx, ny, nz, lx, ly, lz, r):
    x, y, z = _cell_centres(nx, ny, nz, lx, ly, lz)
    return (x - lx / 2) ** 2 + (y - ly / 2) ** 2 + (z - lz / 2) ** 2 <= r * r


def pec_plate_mask(nx, ny, nz, i0, i1, j0, j1, kp) -> np.ndarray:
    """Edge mask of a zero-thickness PEC plate in the plane of node layer kp,
    covering node range [i0, i1] x [j0, j1] (rim included): every x- and
    y-edge lying in it is marked.  Global edge numbering: x-edges, then
    y-edges, then z-edges, each x-fastest over its own (i, j, k) box."""
    nex = nx * (ny + 1) * (nz + 1)
    ney = (nx + 1) * ny * (nz + 1)
    nez = (nx + 1) * (ny + 1) * nz
    m = np.zeros(nex + ney + nez, dtype=np.uint8)
    for j in range(j0, j1 + 1):
        for i in range(i0, i1):
            m[i + nx * (j + (ny + 1) * kp)] = 1
    for j in range(j0, j1):
        for i in range(i0, i1 + 1):
            m[nex + i + (nx + 1) * (j + ny * kp)] = 1
    return m


def make(index: int, seed: int | None = None) -> Workload:
    """Workload 1..5 (see module docstring); seed defaults to the index."""
    seed = index if seed is None else seed
    rng = np.random.default_rng(seed)
    pec = None
    probes = fd = None
    if index == 1:
        n, L = 12, 1.0
        dims = (n, n, n, L, L, L)
        cx, cy, cz = cuts(n, 2, None), cuts(n, 2, None), cuts(n, 1, None)
        eps = np.ones(n ** 3, np.complex128)
        eps[_sphere_mask(*dims, 0.25)] = 4.0
        khat, pol = _random_waves(rng, 1)
    elif index == 2:
        n, L = 32, 3.0
        dims = (n, n, n, L, L, L)
        cx, cy, cz = cuts(n, 4, rng), cuts(n, 4, rng), cuts(n, 2, rng)
        eps = np.ones(n ** 3, np.complex128)
        eps[_sphere_mask(*dims, L / 4)] = 4.0 - 0.1j
        khat, pol = _grid_waves(rng, 8, 8)
    elif index == 3:
        n, L = 20, 2.0
        dims = (n, n, n, L, L, L)
        cx, cy, cz = cuts(n, 2, None), cuts(n, 2, None), cuts(n, 2, None)
        eps = rng.uniform(1.0, 3.0, n ** 3).astype(np.complex128)
        khat, pol = _random_waves(rng, 1)
    elif index == 4:
        dims = (48, 48, 24, 4.0, 4.0, 2.0)
        cx, cy, cz = cuts(48, 4, rng), cuts(48, 4, rng), cuts(24, 2, rng)
        eps = np.ones(48 * 48 * 24, np.complex128)
        pec = pec_plate_mask(48, 48, 24, 12, 36, 12, 36, 12)
        khat, pol = _grid_waves(rng, 2, 4)
    elif index == 5:
        n, L = 64, 6.0
        dims = (n, n, n, L, L, L)
        cx, cy, cz = cuts(n, 4, rng), cuts(n, 4, rng), cuts(n, 4, rng)
        eps = np.ones(n ** 3, np.complex128)
        m = _sphere_mask(*dims, L / 4)
        eps[m] = rng.uniform(2.0, 6.0, int(m.sum())) * (1.0 - 0.01j)
        khat, pol = _grid_waves(rng, 8, 16)
    else:
        raise ValueError(index)
    w = Workload(f"config{index}", *dims, K0, eps, pec, cx, cy, cz, khat, pol, seed=seed)
    if index == 3:
        w.probes = np.sort(rng.choice(w.n_edges, 16, replace=False)).astype(np.int64)
        w.fd_cells = np.sort(rng.choice(w.n_cells, 20, replace=False)).astype(np.int64)
    return w


def lattice_vertices(w: Workload) -> np.ndarray:
    """(n_nodes, 3) positions of the regular lattice, x-fastest."""
    kk, jj, ii = np.meshgrid(np.arange(w.nz + 1), np.arange(w.ny + 1), np.arange(w.nx + 1),
                             indexing="ij")
    return np.stack([ii.ravel() * (w.lx / w.nx), jj.ravel() * (w.ly / w.ny),
                     kk.ravel() * (w.lz / w.nz)], 1).astype(np.float64)


def tetrahedral(w: Workload, jitter: float = 0.1, seed: int | None = None) -> Workload:
    """A copy of w on six tetrahedra per cell, with seeded jittered vertices
    (uniform in [-jitter, jitter] * h per axis; none on an outer boundary
    plane's normal axis).  PEC masks of the brick numbering do not carry over."""
    if w.pec_edge is not None:
        raise ValueError("tetrahedral(): the brick PEC mask has no tetrahedral counterpart")
    rng = np.random.default_rng(w.seed if seed is None else seed)
    v = lattice_vertices(w)
    h = np.array([w.lx / w.nx, w.ly / w.ny, w.lz / w.nz])
    kk, jj, ii = np.meshgrid(np.arange(w.nz + 1), np.arange(w.ny + 1), np.arange(w.nx + 1),
                             indexing="ij")
    idx = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1)
    n = np.array([w.nx, w.ny, w.nz])
    movable = (idx > 0) & (idx < n[None, :])
    d = rng.uniform(-jitter, jitter, v.shape) * h[None, :]
    v = v + np.where(movable, d, 0.0)
    return dataclasses.replace(w, name=w.name + "-tet", element="tet", vertices=v, probes=None,
                               fd_cells=None)


def mesh_edge_pairs(tets) -> np.ndarray:
    """Distinct vertex pairs (i < j) of the tetrahedra, lexicographic: the
    global edge numbering of a general mesh (edge (i, j) points from i to j)."""
    t = np.asarray(tets, np.int64)
    p = np.concatenate([np.sort(t[:, [a, b]], axis=1) for a, b in
                        ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
    return np.unique(p, axis=0)


def mesh_face_triples(tets) -> np.ndarray:
    """Distinct vertex triples (i < j < k) of the tetrahedra, lexicographic."""
    t = np.asarray(tets, np.int64)
    f = np.concatenate([np.sort(t[:, list(q)], axis=1) for q in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))])
    return np.unique(f, axis=0)


def as_mesh(w: Workload) -> Workload:
    """A lattice-tetrahedral workload as a general mesh: the same vertices and
    tetrahedra (cell by cell, the six of a cell in the order of the axis
    permutations (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x)), the
    cell's eps on each of its six, cut planes at the lattice cut coordinates."""
    if w.element != "tet":
        raise ValueError("as_mesh(): needs a lattice-tetrahedral workload")
    v = lattice_vertices(w) if w.vertices is None else np.asarray(w.vertices, np.float64)
    nid = lambda i, j, k: i + (w.nx + 1) * (j + (w.ny + 1) * k)
    kk, jj, ii = np.meshgrid(np.arange(w.nz), np.arange(w.ny), np.arange(w.nx), indexing="ij")
    ci, cj, ck = ii.ravel(), jj.ravel(), kk.ravel()
    perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
    tets = np.zeros((len(ci), 6, 4), np.int64)
    for t, perm in enumerate(perms):
        o = np.zeros(3, np.int64)
        tets[:, t, 0] = nid(ci, cj, ck)
        for q, ax in enumerate(perm):
            o[ax] = 1
            tets[:, t, q + 1] = nid(ci + o[0], cj + o[1], ck + o[2])
    h = (w.lx / w.nx, w.ly / w.ny, w.lz / w.nz)
    gcuts = tuple(np.asarray(c, np.float64) * hh for c, hh in zip((w.cx, w.cy, w.cz), h))
    return dataclasses.replace(w, name=w.name + "-mesh", element="mesh", vertices=v,
                               tets=tets.reshape(-1, 4), eps=np.repeat(w.eps, 6), gcuts=gcuts)


def delaunay(nx, ny, nz, px, py, pz, seed=0, nrhs=1, h=0.1, jitter=0.3, lossy=True, order=1) -> Workload:
    """An unstructured tetrahedral mesh of the box [0, nx h] x [0, ny h] x
    [0, nz h]: the Delaunay tetrahedralisation (scipy.spatial.Delaunay) of
    the lattice points moved by a seeded uniform jitter of up to jitter*h per
    axis (boundary points only within their boundary planes, box edges along
    the edge, corners fixed); per-tetrahedron eps ~ U[1, 3] (lossy: times
    1 - 0.05j); px x py x pz subdomains cut at equal coordinates; random plane
    waves; order 2: two dofs per edge (Whitney and edge-gradient functions);
    order 3: also two per face (curl-complete second order).
    Draw order: jitter, eps, waves."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    idx = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1)
    n = np.array([nx, ny, nz])
    movable = (idx > 0) & (idx < n[None, :])
    pts = idx * h + np.where(movable, rng.uniform(-jitter, jitter, idx.shape) * h, 0.0)
    tets = Delaunay(pts).simplices.astype(np.int64)
    e = [pts[tets[:, q]] - pts[tets[:, 0]] for q in (1, 2, 3)]
    vol = np.abs(np.einsum("ij,ij->i", e[0], np.cross(e[1], e[2]))) / 6.0
    if vol.min() < 1e-6 * h ** 3:
        raise ValueError("delaunay(): degenerate tetrahedron")
    eps = rng.uniform(1.0, 3.0, len(tets)).astype(np.complex128)
    if lossy:
        eps = eps * (1.0 - 0.05j)
    khat, pol = _random_waves(rng, nrhs)
    L = (nx * h, ny * h, nz * h)
    gcuts = tuple(np.linspace(0.0, L[a], p + 1) for a, p in enumerate((px, py, pz)))
    empty = np.zeros(1, np.int32)
    return Workload(f"delaunay{nx}x{ny}x{nz}" + ("-o2" if order == 2 else ""), nx, ny, nz, *L, K0, eps, None,
                    empty, empty, empty, khat, pol, seed=seed, element="mesh", vertices=pts, tets=tets,
                    gcuts=gcuts, order=order)


def tiny(nx, ny, nz, px, py, pz, seed=0, lossy=True, nrhs=1, pec=None, jitter=False,
         h=0.1) -> Workload:
    """Small seeded mesh for unit tests: random per-cell eps (lossy if asked),
    equal or jittered (+-1 cell) cuts, random plane waves."""
    rng = np.random.default_rng(seed)
    cx = cuts(nx, px, rng if jitter else None, 1)
    cy = cuts(ny, py, rng if jitter else None, 1)
    cz = cuts(nz, pz, rng if jitter else None, 1)
    eps = rng.uniform(1.0, 3.0, nx * ny * nz).astype(np.complex128)
    if lossy:
        eps = eps * (1.0 - 0.05j)
    khat, pol = _random_waves(rng, nrhs)
    w = Workload(f"tiny{nx}x{ny}x{nz}", nx, ny, nz, nx * h, ny * h, nz * h, K0, eps, pec,
                 cx, cy, cz, khat, pol, seed=seed)
    return w
