"""Adjoint gradient of a field objective -- oracle, test only.

Objective J = sum_{m in probes} |x_m|^2 with x = A(eps)^{-1} f and A =
S - k^2 sum_c eps_c M_c + jk T (Theory section discretisation).  With
dA/d(Re eps_c) = -k^2 M_c and A = A^T,
    dJ/d(Re eps_c) = 2 k^2 Re( u_c^T M_c x_c ),   u = A^{-1} (P conj(x)),
P the probe selector, u_c and x_c the local edge values of cell c (12 on
bricks, 19 on the six tetrahedra of a tetrahedral cell, 6 (12 at order 2)
per tetrahedron of a general mesh).  The
adjoint solve is a plain second sparse LU solve; no code is shared with the
library.  Pinned by central finite differences (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

from . import fem


def objective(x, probes):
    return float(np.sum(np.abs(x[probes]) ** 2))


def gradient(w, f, probes):
    """(J, dJ/d Re eps (n_cells,)) summed over the RHS columns of f."""
    g = None if getattr(w, "element", "brick") == "mesh" else fem.Grid.of(w)
    x = fem.solve_global(w, f)
    rhs = np.zeros_like(x)
    rhs[probes] = np.conj(x[probes])
    u = fem.solve_global(w, rhs)
    if getattr(w, "element", "brick") == "mesh":
        from . import tetmesh
        g = tetmesh.grid_of(w)
        _, M = tetmesh.tet_matrices(g, np.arange(g.n_cells))
        ce = g.tet_dofs
    elif g.element == "brick":
        _, M = fem.element_matrices(g.h)
        M = np.broadcast_to(M, (g.n_cells, 12, 12))
        ce = g.cell_edges()
    else:
        _, M = fem.tet_cell_matrices(g, np.arange(g.n_cells))
        ce = g.cell_edges()
    grad = np.zeros(len(ce))
    for col in range(x.shape[1]):
        xc = x[ce, col]          # (ncell, 12 or 19)
        uc = u[ce, col]
        grad += 2.0 * w.k ** 2 * np.real(np.einsum("ca,cab,cb->c", uc, M, xc))
    return objective(x, probes), grad
