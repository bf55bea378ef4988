"""Orderings and symbolic factorisation (main steps 3-4) -- oracle, test only.

The paper reorders the clique graph of K with METIS and symbolically factors
it (main steps 3-4, discussion of Algorithm 1).  METIS is not available, so the
reading used here is a deterministic geometric nested dissection:

* inside a subdomain, the dofs that carry no multiplier are ordered by
  recursive bisection of the cell box: a region whose unassigned edges number
  more than leaf_max is split at cell plane lo + (hi - lo) // 2 of its longest
  axis (ties x < y < z); the unassigned edges lying in that plane form the
  separator; order = left subtree, right subtree, separator; inside a node
  edges follow the global edge index;
* the interface dofs B_i (edges with >= 1 multiplier) come last, as one
  pivot block (the domain-matrix step, main step 1);
* the interface blocks of K are ordered by block nested dissection of the
  subdomain grid: split at the middle cut plane of the axis with most
  subdomains (ties x < y < z); the separator is the blocks crossing it,
  ordered by (a, b); order = left, right, separator.

Everything is one symmetric saddle matrix M = [[A, D], [D^T, 0]] (Eq. (1))
ordered as [subdomain 0: ND interior, B_0; subdomain 1: ...; multipliers in
block order].  Each ND node, each B_i and each interface block is a
supernode (a contiguous pivot range).  The supernodal structure is obtained by
the elimination game on packed bitsets: eliminating a supernode joins its
remaining neighbours into a clique; struct = those neighbours; parent = the
supernode holding min(struct).  These arrays are compared bit-exactly with the
library's own symbolic stage.
"""
from __future__ import annotations

import dataclasses

import numpy as np

LEAF_MAX = 64


def block_nested_dissection(parts, pairs):
    """Order of the interface blocks (pairs (a, b), a < b) by block ND: the
    separator of a box is every block of the box whose two subdomains lie on
    opposite sides of its middle cut (on lattice meshes these are the face
    neighbours across the cut; on general meshes a block may also join
    subdomains that touch only along an edge or at a point)."""
    px, py, pz = parts

    def pos(s):
        return (s % px, (s // px) % py, s // (px * py))

    def rec(lo, hi, P):
        ext = [hi[a] - lo[a] for a in range(3)]
        if max(ext) <= 1:
            return []
        axis = int(np.argmax(ext))       # first maximum: ties x < y < z
        mid = lo[axis] + ext[axis] // 2
        lhi = list(hi); lhi[axis] = mid
        rlo = list(lo); rlo[axis] = mid
        left = [p for p in P if pos(p[0])[axis] < mid and pos(p[1])[axis] < mid]
        right = [p for p in P if pos(p[0])[axis] >= mid and pos(p[1])[axis] >= mid]
        sep = [p for p in P if p not in left and p not in right]
        return rec(lo, lhi, left) + rec(rlo, hi, right) + sorted(sep)

    order = rec([0, 0, 0], [px, py, pz], sorted(pairs))
    assert sorted(order) == sorted(pairs)
    return order


def subdomain_nd(grid, sd, interface_edges, leaf_max=LEAF_MAX):
    """List of ND nodes (each a sorted array of global edges), post-order,
    for the non-interface dofs of subdomain sd."""
    info = grid.edge_info()
    avail = np.zeros(grid.n_edges, bool)
    avail[sd.edges] = True
    avail[np.asarray(list(interface_edges), dtype=np.int64)] = False
    nodes = []

    def region_edges(lo, hi):
        from .decomp import box_edges
        e = box_edges(grid, lo, hi)
        return e[avail[e]]

    def rec(lo, hi):
        E = region_edges(lo, hi)
        ext = [hi[a] - lo[a] for a in range(3)]
        if len(E) <= leaf_max or max(ext) < 2:
            if len(E):
                avail[E] = False
                nodes.append(E)
            return
        axis = int(np.argmax(ext))
        c = lo[axis] + ext[axis] // 2
        d = info[E, 0]
        coord = info[E, 1 + axis]
        sep = E[(grid.dirs[d, axis] == 0) & (coord == c)]
        avail[sep] = False
        lhi = list(hi); lhi[axis] = c
        rlo = list(lo); rlo[axis] = c
        rec(list(lo), lhi)
        rec(rlo, list(hi))
        if len(sep):
            nodes.append(np.sort(sep))

    rec(list(sd.cell_lo), list(sd.cell_hi))
    return nodes


@dataclasses.dataclass
class Plan:
    n: int                       # order of M
    sn_start: np.ndarray         # supernode ranges [start, end)
    sn_end: np.ndarray
    sn_kind: np.ndarray          # 0 = ND node, 1 = interface dofs B_i, 2 = block of K
    sn_owner: np.ndarray         # subdomain (kinds 0, 1) or block id (kind 2)
    parent: np.ndarray = None    # supernodal elimination tree (-1 = root)
    struct: list = None          # sorted update rows of each supernode
    # M index -> (subdomain, global edge) or multiplier id
    m_sub: np.ndarray = None     # -1 for multipliers
    m_edge: np.ndarray = None    # global edge (dofs) or multiplier id


def build_plan(dec, leaf_max=LEAF_MAX):
    """Ordering of M and supernode partition."""
    starts, ends, kinds, owners = [], [], [], []
    m_sub, m_edge = [], []
    pos = 0
    for sd in dec.subs:
        iface = set(int(e) for e, a, b in zip(dec.lm_edge, dec.lm_plus, dec.lm_minus)
                    if a == sd.index or b == sd.index)
        if getattr(dec.grid, "element", "brick") == "mesh":
            from .tetmesh import subdomain_nd as nd
        else:
            nd = subdomain_nd
        for node in nd(dec.grid, sd, iface, leaf_max):
            starts.append(pos); pos += len(node); ends.append(pos)
            kinds.append(0); owners.append(sd.index)
            m_sub += [sd.index] * len(node); m_edge += list(node)
        B = np.array(sorted(iface), np.int64)
        if len(B):
            starts.append(pos); pos += len(B); ends.append(pos)
            kinds.append(1); owners.append(sd.index)
            m_sub += [sd.index] * len(B); m_edge += list(B)
    for b, lms in enumerate(dec.block_lms):
        starts.append(pos); pos += len(lms); ends.append(pos)
        kinds.append(2); owners.append(b)
        m_sub += [-1] * len(lms); m_edge += list(lms)
    return Plan(pos, np.array(starts), np.array(ends), np.array(kinds), np.array(owners),
                m_sub=np.array(m_sub, np.int64), m_edge=np.array(m_edge, np.int64))


def saddle_pattern(dec, plan):
    """Lower+upper adjacency of M as (rows, cols) index arrays in M order."""
    where = {}
    for i, (s, e) in enumerate(zip(plan.m_sub, plan.m_edge)):
        where[(int(s), int(e))] = i
    R, C = [], []
    for sd in dec.subs:
        A = sd.A.tocoo()
        mi = np.array([where[(sd.index, int(e))] for e in sd.edges])
        R.append(mi[A.row]); C.append(mi[A.col])
    lm_pos = {int(l): i for i, (s, l) in enumerate(zip(plan.m_sub, plan.m_edge)) if s < 0}
    for l, (e, a, b) in enumerate(zip(dec.lm_edge, dec.lm_plus, dec.lm_minus)):
        for s in (a, b):
            i, j = where[(int(s), int(e))], lm_pos[l]
            R.append(np.array([i, j])); C.append(np.array([j, i]))
    return np.concatenate(R), np.concatenate(C)


def symbolic(plan, rows, cols):
    """Supernodal elimination game on packed bitsets; fills plan.parent and
    plan.struct."""
    n = plan.n
    nbytes = (n + 7) // 8
    bits = np.zeros((n, nbytes), np.uint8)
    off = rows != cols
    r, c = rows[off], cols[off]
    np.bitwise_or.at(bits, (r, c // 8), (1 << (c % 8)).astype(np.uint8))
    sn_of = np.repeat(np.arange(len(plan.sn_start)), plan.sn_end - plan.sn_start)
    parent = -np.ones(len(plan.sn_start), np.int64)
    structs = []
    for s, (a, b) in enumerate(zip(plan.sn_start, plan.sn_end)):
        nb = np.bitwise_or.reduce(bits[a:b], axis=0)
        mask = np.unpackbits(nb, bitorder="little")[:n].astype(bool)
        mask[:b] = False
        st = np.flatnonzero(mask)
        structs.append(st)
        if len(st):
            parent[s] = sn_of[st[0]]
            packed = np.packbits(mask, bitorder="little")
            bits[st] |= packed[None, :]
    plan.parent = parent
    plan.struct = structs
    return plan


def symbolic_merge(plan, rows, cols):
    """The same supernodal structure as symbolic(), for matrices too large
    for its n x n bitset: struct(s) = the neighbours of the rows of s in M,
    together with the structures of the children of s in the supernodal tree,
    keeping only indices past the last row of s; parent(s) = the supernode
    holding min struct(s).  (Eliminating a supernode makes its structure a
    clique; whatever of that clique lies past its parent is also in the
    parent's structure, so a supernode only has to merge its children's.)
    Pinned against the elimination game (tests/test_oracle_ordering.py)."""
    n = plan.n
    off = rows != cols
    r, c = np.asarray(rows)[off], np.asarray(cols)[off]
    o = np.argsort(r, kind="stable")
    r, c = r[o], c[o]
    ptr = np.searchsorted(r, np.arange(n + 1))
    sn_of = np.repeat(np.arange(len(plan.sn_start)), plan.sn_end - plan.sn_start)
    nsn = len(plan.sn_start)
    parent = -np.ones(nsn, np.int64)
    structs = [None] * nsn
    kids = [[] for _ in range(nsn)]
    for s, (a, b) in enumerate(zip(plan.sn_start, plan.sn_end)):
        u = np.unique(np.concatenate([c[ptr[a]:ptr[b]]] + [structs[k] for k in kids[s]]))
        st = u[u >= b].astype(np.int64)
        structs[s] = st
        if len(st):
            parent[s] = sn_of[st[0]]
            kids[parent[s]].append(s)
    plan.parent = parent
    plan.struct = structs
    return plan
