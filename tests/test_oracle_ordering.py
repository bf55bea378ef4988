"""Pins of the oracle's orderings and symbolic factorisation (main steps 3-4).

The block order of the interface blocks of K is fixed by the block nested
dissection rule (split the subdomain grid at the middle cut plane of the axis
with the most subdomains, ties x < y < z; left part, right part, then the
separator blocks sorted by (a, b)).  The expected orders below were derived by
hand from that rule for three subdomain grids and are written out literally,
so a wrong axis choice, split position, recursion order or separator sort
fails here even where the library (following the same rule) would agree.
"""
import numpy as np
import pytest

from oracle import decomp, ordering
from paper_2002_05018_gb300 import workloads as W


def _face_pairs(px, py, pz):
    sid = lambda x, y, z: x + px * (y + py * z)
    out = set()
    for z in range(pz):
        for y in range(py):
            for x in range(px):
                if x + 1 < px:
                    out.add((sid(x, y, z), sid(x + 1, y, z)))
                if y + 1 < py:
                    out.add((sid(x, y, z), sid(x, y + 1, z)))
                if z + 1 < pz:
                    out.add((sid(x, y, z), sid(x, y, z + 1)))
    return out


# 2x2x2: split x at 1 (separator (0,1),(2,3),(4,5),(6,7)); each half splits y,
# then z.
BND_222 = [(0, 4), (2, 6), (0, 2), (4, 6), (1, 5), (3, 7), (1, 3), (5, 7),
           (0, 1), (2, 3), (4, 5), (6, 7)]

# 3x2x1: split x at 1; the left column splits y; the right 2x2 block splits x
# at 2 (tie x < y), each of its columns splits y.
BND_321 = [(0, 3), (1, 4), (2, 5), (1, 2), (4, 5), (0, 1), (3, 4)]

# 4x4x2: split x at 2; each 2x4x2 half splits y at 2; each 2x2x2 quarter is
# the 2x2x2 pattern shifted by its first subdomain id.
_Q = [(0, 16), (4, 20), (0, 4), (16, 20), (1, 17), (5, 21), (1, 5), (17, 21),
      (0, 1), (4, 5), (16, 17), (20, 21)]


def _shift(lst, d):
    return [(a + d, b + d) for a, b in lst]


BND_442 = (_shift(_Q, 0) + _shift(_Q, 8) + [(4, 8), (5, 9), (20, 24), (21, 25)]
           + _shift(_Q, 2) + _shift(_Q, 10) + [(6, 10), (7, 11), (22, 26), (23, 27)]
           + [(1, 2), (5, 6), (9, 10), (13, 14), (17, 18), (21, 22), (25, 26), (29, 30)])


@pytest.mark.parametrize("parts,expected", [((2, 2, 2), BND_222), ((3, 2, 1), BND_321),
                                            ((4, 4, 2), BND_442)])
def test_block_nested_dissection_hand_orders(parts, expected):
    pairs = _face_pairs(*parts)
    assert len(expected) == len(pairs) == len(set(expected))
    assert ordering.block_nested_dissection(parts, pairs) == expected


def test_decomposition_uses_face_pairs_in_bnd_order():
    """The multiplier blocks of a 3x2x1 decomposition are exactly the face
    pairs, in the hand-derived block order."""
    w = W.tiny(6, 4, 3, 3, 2, 1, seed=2)
    dec = decomp.decompose(w, with_matrices=False)
    assert [tuple(b) for b in dec.blocks] == BND_321


def _elimination_game_dense(n, rows, cols, sn_start, sn_end):
    """Supernodal elimination on a dense boolean matrix (tiny n only)."""
    G = np.zeros((n, n), bool)
    G[rows, cols] = True
    np.fill_diagonal(G, False)
    structs = []
    for a, b in zip(sn_start, sn_end):
        nb = G[a:b].any(axis=0)
        nb[:b] = False
        st = np.flatnonzero(nb)
        structs.append(st)
        G[np.ix_(st, st)] = True
    return structs


@pytest.mark.parametrize("mk,leaf", [(lambda: W.tiny(4, 4, 4, 2, 2, 2, seed=1), 16),
                                     (lambda: W.tiny(9, 7, 5, 3, 2, 2, seed=4, jitter=True), 24),
                                     (lambda: W.tiny(6, 6, 6, 1, 1, 1, seed=2), 20)])
def test_symbolic_merge_equals_elimination_game(mk, leaf):
    """The children-merge form of the supernodal symbolic factorisation (used
    for the large workloads) equals the elimination game, both on packed
    bitsets and on a dense boolean matrix."""
    w = mk()
    dec = decomp.decompose(w, with_matrices=True)
    plan = ordering.build_plan(dec, leaf_max=leaf)
    r, c = ordering.saddle_pattern(dec, plan)
    ref = _elimination_game_dense(plan.n, r, c, plan.sn_start, plan.sn_end)
    ordering.symbolic(plan, r, c)
    game_parent = plan.parent.copy()
    for q, st in enumerate(ref):
        assert np.array_equal(plan.struct[q], st), q
    ordering.symbolic_merge(plan, r, c)
    assert np.array_equal(plan.parent, game_parent)
    for q, st in enumerate(ref):
        assert np.array_equal(plan.struct[q], st), q
