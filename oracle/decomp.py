"""Decomposed BVP and its Lagrange-multiplier map -- oracle, test only.

Theory section / Eq. (1): Omega is cut by axis-aligned planes into a grid of
subdomains; edges on a cut plane are copied into every subdomain holding them.
Each subdomain matrix A_i is the FEM-ABC matrix of its cells plus the
interface loss/gain term sigma * alpha * T_f on each of its cut faces, with
alpha = jk, sigma = +1 when the neighbour across the face has the higher
subdomain index and -1 otherwise (reading of "loss or gain at the interfaces"
in the paper's discussion of Eq. (1); the two sides cancel when the copies
agree, which keeps the decomposition exact).  Subdomain index
s = ix + px*(iy + py*iz).

D (Eq. (1)) is read as a signed Boolean map: for a copied edge with copies in
subdomains s_1 < ... < s_m, every s_k (k >= 2) is tied to the smallest s_j
(j < k) sharing a face with it by one multiplier "x_{s_j} - x_{s_k} = 0"
(+1 on s_j, -1 on s_k).  A multiplier belongs to the interface block of the
pair (s_j, s_k); inside a block multipliers follow the global edge index.
RHS split: the owner (lowest-index copy) receives f_e, the other copies 0.

Parity pins: decomposed solution = global solution (tests/test_oracle_d3m.py),
sum over copies of A_i = A.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import fem


@dataclasses.dataclass
class Subdomain:
    index: int
    grid_pos: tuple
    cell_lo: tuple
    cell_hi: tuple
    edges: np.ndarray          # sorted global edge ids (free edges only)
    A: sp.csr_matrix | None = None


@dataclasses.dataclass
class Decomposition:
    grid: fem.Grid
    parts: tuple               # (px, py, pz)
    subs: list
    copies: dict               # global edge -> sorted list of subdomains
    lm_edge: np.ndarray        # per multiplier (block-local order, see blocks)
    lm_plus: np.ndarray        # subdomain with +1
    lm_minus: np.ndarray       # subdomain with -1
    blocks: list               # list of (a, b) pairs, block id = position
    block_lms: list            # block id -> array of multiplier ids
    lm_weight: int = 0         # 0: signed Boolean D; 1: D_bool T_lambda (see multiplier_mass)
    T_lambda: sp.csr_matrix | None = None


def sub_index(pos, parts):
    return pos[0] + parts[0] * (pos[1] + parts[1] * pos[2])


def sub_pos(s, parts):
    return (s % parts[0], (s // parts[0]) % parts[1], s // (parts[0] * parts[1]))


def face_adjacent(a, b, parts):
    pa, pb = sub_pos(a, parts), sub_pos(b, parts)
    d = [abs(x - y) for x, y in zip(pa, pb)]
    return sorted(d) == [0, 0, 1]


def box_edges(g: fem.Grid, lo, hi):
    """All edges of the cells in the box [lo, hi) (sorted): per edge family
    with direction d, the start nodes in [lo, hi - d] along each axis."""
    out = []
    r = lambda a, b: np.arange(a, b)
    for f, d in enumerate(g.dirs):
        i, j, k = np.meshgrid(r(lo[0], hi[0] + 1 - d[0]), r(lo[1], hi[1] + 1 - d[1]),
                              r(lo[2], hi[2] + 1 - d[2]), indexing="ij")
        out.append(g.edge_id(f, i, j, k).ravel())
    return np.sort(np.concatenate(out))


def decompose(w, with_matrices=True) -> Decomposition:
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        return tetmesh.decompose(w, with_matrices)
    g = fem.Grid.of(w)
    cuts = (np.asarray(w.cx), np.asarray(w.cy), np.asarray(w.cz))
    parts = tuple(len(c) - 1 for c in cuts)
    free = np.ones(g.n_edges, bool)
    if w.pec_edge is not None:
        free[w.pec_edge != 0] = False
    subs = []
    nsub = parts[0] * parts[1] * parts[2]
    for s in range(nsub):
        pos = sub_pos(s, parts)
        lo = tuple(int(cuts[a][pos[a]]) for a in range(3))
        hi = tuple(int(cuts[a][pos[a] + 1]) for a in range(3))
        e = box_edges(g, lo, hi)
        subs.append(Subdomain(s, pos, lo, hi, e[free[e]]))
    copies = {}
    for sd in subs:
        for e in sd.edges:
            copies.setdefault(int(e), []).append(sd.index)
    # multipliers, spanning-tree rule
    pairs = {}
    for e in sorted(copies):
        cs = copies[e]
        for kk in range(1, len(cs)):
            sk = cs[kk]
            sj = next(cs[j] for j in range(kk) if face_adjacent(cs[j], sk, parts))
            pairs.setdefault((sj, sk), []).append(e)
    from . import ordering
    block_order = ordering.block_nested_dissection(parts, set(pairs))
    lm_edge, lm_plus, lm_minus, block_lms = [], [], [], []
    for (a, b) in block_order:
        es = sorted(pairs[(a, b)])
        ids = np.arange(len(lm_edge), len(lm_edge) + len(es))
        block_lms.append(ids)
        lm_edge += es
        lm_plus += [a] * len(es)
        lm_minus += [b] * len(es)
    dec = Decomposition(g, parts, subs, copies, np.array(lm_edge, np.int64),
                        np.array(lm_plus, np.int64), np.array(lm_minus, np.int64),
                        list(block_order), block_lms, int(getattr(w, "lm_weight", 0) or 0))
    if dec.lm_weight:
        dec.T_lambda = multiplier_mass(dec)
    if with_matrices:
        for sd in subs:
            sd.A = subdomain_matrix(w, dec, sd)
    return dec


def interface_faces(dec: Decomposition, sd: Subdomain, alpha):
    """(axis, side, cells, +-alpha) for each cut face of subdomain sd."""
    g = dec.grid
    out = []
    for axis in range(3):
        for side in (0, 1):
            npos = list(sd.grid_pos)
            npos[axis] += -1 if side == 0 else 1
            if not 0 <= npos[axis] < dec.parts[axis]:
                continue
            nb = sub_index(npos, dec.parts)
            node = sd.cell_lo[axis] if side == 0 else sd.cell_hi[axis]
            for ax, sd_side, cid in fem.boundary_faces(g, sd.cell_lo, sd.cell_hi, {axis: (node,)}):
                if ax == axis and sd_side == side:
                    out.append((axis, side, cid, alpha if nb > sd.index else -alpha))
    return out


def subdomain_matrix(w, dec: Decomposition, sd: Subdomain):
    """A_i on the subdomain's local dofs (sorted global edge order); the interface coefficient
    is w.alpha when given, else jk (the decomposed solution does not depend on it)."""
    g = dec.grid
    ci, cj, ck = g.cell_ijk()
    lo, hi = sd.cell_lo, sd.cell_hi
    cells = np.flatnonzero((ci >= lo[0]) & (ci < hi[0]) & (cj >= lo[1]) & (cj < hi[1])
                           & (ck >= lo[2]) & (ck < hi[2]))
    alpha = 1j * w.k if getattr(w, "alpha", None) is None else complex(w.alpha)
    faces = fem.abc_faces(g, w.k, lo, hi) + interface_faces(dec, sd, alpha)
    r, c, v = fem.assemble(g, w.eps, w.k, cells=cells, extra_faces=faces)
    loc = -np.ones(g.n_edges, np.int64)
    loc[sd.edges] = np.arange(len(sd.edges))
    keep = (loc[r] >= 0) & (loc[c] >= 0)
    n = len(sd.edges)
    return sp.csr_matrix((v[keep], (loc[r[keep]], loc[c[keep]])), shape=(n, n))


def multiplier_mass(dec: Decomposition):
    """T_lambda (n_lambda x n_lambda): the Galerkin reading of the Theory
    section's multiplier lambda = j +- e.  With lambda expanded in the same
    tangential edge basis as the trace of E, the coupling of multipliers m and
    l of one interface block (a, b) is the tangential face mass
    int_f N_m . N_l dS over the cut face between subdomains a and b; there is
    no coupling across blocks.  D = D_bool T_lambda."""
    g = dec.grid
    lm_of = {(int(a), int(b), int(e)): l
             for l, (e, a, b) in enumerate(zip(dec.lm_edge, dec.lm_plus, dec.lm_minus))}
    ce_all = g.cell_edges()
    rows, cols, vals = [], [], []
    for (a, b) in dec.blocks:
        sd = dec.subs[a]
        for axis, side, cid, _ in interface_faces(dec, sd, 1.0):
            npos = list(sd.grid_pos)
            npos[axis] += -1 if side == 0 else 1
            if sub_index(npos, dec.parts) != b:
                continue
            Tc = fem.face_block(g, axis, side, cid)
            for c, T in zip(cid, Tc):
                ce = ce_all[c]
                for i in range(len(ce)):
                    m = lm_of.get((a, b, int(ce[i])))
                    if m is None:
                        continue
                    for j in range(len(ce)):
                        l = lm_of.get((a, b, int(ce[j])))
                        if l is None or T[i, j] == 0.0:
                            continue
                        rows.append(m)
                        cols.append(l)
                        vals.append(T[i, j])
    n = len(dec.lm_edge)
    return sp.csr_matrix((np.array(vals, float), (rows, cols)), shape=(n, n))


def D_matrix(dec: Decomposition, sd: Subdomain):
    """Sparse D_i (n_i x n_lambda): the signed Boolean map, or (lm_weight 1)
    the signed Boolean map times T_lambda."""
    Db = D_bool(dec, sd)
    return (Db @ dec.T_lambda).tocsr() if dec.lm_weight else Db


def D_bool(dec: Decomposition, sd: Subdomain):
    """Sparse signed Boolean D_i (n_i x n_lambda)."""
    loc = {int(e): i for i, e in enumerate(sd.edges)}
    rows, cols, vals = [], [], []
    for l, (e, a, b) in enumerate(zip(dec.lm_edge, dec.lm_plus, dec.lm_minus)):
        if a == sd.index:
            rows.append(loc[int(e)]); cols.append(l); vals.append(1.0)
        elif b == sd.index:
            rows.append(loc[int(e)]); cols.append(l); vals.append(-1.0)
    return sp.csr_matrix((np.array(vals), (rows, cols)), shape=(len(sd.edges), len(dec.lm_edge)))


def split_rhs(dec: Decomposition, sd: Subdomain, f):
    """Owner rule: f_e goes to the lowest-index copy of e."""
    owner = np.array([dec.copies[int(e)][0] == sd.index for e in sd.edges])
    fi = f[sd.edges].copy()
    fi[~owner] = 0
    return fi


def interface_dofs(dec: Decomposition, sd: Subdomain):
    """Local positions of the subdomain's edges that carry >= 1 multiplier."""
    lm_edges = set(int(e) for e, a, b in zip(dec.lm_edge, dec.lm_plus, dec.lm_minus)
                   if a == sd.index or b == sd.index)
    return np.array([i for i, e in enumerate(sd.edges) if int(e) in lm_edges], np.int64)
