"""Pin of the oracle adjoint gradient against central finite differences."""
import numpy as np

from oracle import adjoint, fem
from paper_2002_05018_gb300 import workloads as W


def test_adjoint_matches_central_differences():
    w = W.tiny(4, 3, 3, 1, 1, 1, seed=21, nrhs=2)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(0)
    probes = np.sort(rng.choice(w.n_edges, 6, replace=False))
    J, g = adjoint.gradient(w, f, probes)
    h = 1e-6
    for c in rng.choice(w.n_cells, 6, replace=False):
        e0 = w.eps.copy()
        w.eps = e0.copy(); w.eps[c] += h
        Jp = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0.copy(); w.eps[c] -= h
        Jm = adjoint.objective(fem.solve_global(w, f), probes)
        w.eps = e0
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * max(abs(fd), 1e-3 * abs(g).max()), (c, fd, g[c])
