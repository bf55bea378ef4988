"""Pins of the oracle's FEM layer against closed forms and invariants."""
import os

import numpy as np
import pytest

from oracle import fem
from paper_2002_05018_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "brick_unit_cube.txt")


def _golden():
    lines = open(GOLD).read().split("\n")
    out = {}
    for name in ("M", "S"):
        i = lines.index(name)
        out[name] = np.array([[float(v) for v in l.split()] for l in lines[i + 1:i + 13]]) / 36.0
    return out


def test_element_matrices_match_closed_form():
    g = _golden()
    S, M = fem.element_matrices(np.array([1.0, 1.0, 1.0]))
    assert np.abs(M - g["M"]).max() < 1e-14
    assert np.abs(S - g["S"]).max() < 1e-14


def test_element_scaling_and_nullspace():
    h = np.array([0.3, 0.2, 0.5])
    S, M = fem.element_matrices(h)
    ev = np.linalg.eigvalsh(S)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 7       # 8 nodes -> 7 gradients
    assert np.linalg.eigvalsh(M).min() > 0
    # 1-D mass factors: x-edges (0,0) and (1,0) share z and differ in y
    vol = h.prod()
    assert np.isclose(M[0, 0], vol / 9) and np.isclose(M[0, 1], vol / 18)
    assert np.isclose(M[0, 3], vol / 36)
    # constant field along x: x = 1 on all x-edges -> x^T M x = volume
    x = np.r_[np.ones(4), np.zeros(8)]
    assert np.isclose(x @ M @ x, vol)


def test_curl_grad_zero_and_symmetry():
    w = W.tiny(3, 4, 2, 1, 1, 1, seed=1)
    g = fem.Grid.of(w)
    G = fem.discrete_gradient(g)
    w0 = W.tiny(3, 4, 2, 1, 1, 1, seed=1)
    w0.k = 0.0
    S = fem.global_matrix(w0)
    assert np.abs((S @ G).toarray()).max() < 1e-12
    A = fem.global_matrix(w)
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()


def test_face_matrix():
    h = np.array([0.3, 0.2, 0.5])
    T = fem.face_matrix(h, 2, 0)       # face z = 0: x-edges (.,0) and y-edges (.,0)
    assert np.isclose(T[0, 0], h[0] * h[1] / 3) and np.isclose(T[0, 1], h[0] * h[1] / 6)
    assert np.abs(T[2]).max() == 0 and np.abs(T[8:]).max() == 0


def test_planewave_convergence_homogeneous_box():
    """In a homogeneous box the continuous solution is E_inc exactly (the ABC
    data is built from it), so the discrete solution converges to its edge
    interpolant; error must drop >= 2x per halving of h."""
    errs = []
    for n in (4, 8):
        w = W.tiny(n, n, n, 1, 1, 1, seed=3, lossy=False, h=1.0 / n)
        w.eps[:] = 1.0
        f = fem.rhs_planewave(w)
        x = fem.solve_global(w, f)[:, 0]
        xi = fem.edge_interpolant(w, w.khat[0], w.pol[0])
        errs.append(np.linalg.norm(x - xi) / np.linalg.norm(xi))
    assert errs[0] < 0.5 and errs[1] < errs[0] / 2.0


def test_reciprocity():
    w = W.tiny(4, 3, 3, 1, 1, 1, seed=2, nrhs=2)
    f = fem.rhs_planewave(w)
    x = fem.solve_global(w, f)
    assert abs(x[:, 0] @ f[:, 1] - x[:, 1] @ f[:, 0]) < 1e-10 * abs(x[:, 0] @ f[:, 1])


def test_pec_edges_removed():
    w = W.tiny(4, 4, 4, 1, 1, 1, seed=4)
    w.pec_edge = W.pec_plate_mask(4, 4, 4, 1, 3, 1, 3, 2)
    f = fem.rhs_planewave(w)
    x = fem.solve_global(w, f)
    assert np.all(x[w.pec_edge == 1] == 0)
    assert fem.rel_residual(w, x, f)[0] < 1e-12
