"""Adjoint gradient (row a8): torch.autograd through the library against the
oracle adjoint, central finite differences and torch.autograd.gradcheck."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint, fem  # noqa: E402
from paper_2002_05018_gb300 import autograd as ag, d3m, workloads as W  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _J(x, probes):
    return (x[probes].abs() ** 2).sum()


def test_config3_gradient_vs_oracle_and_fd():
    _need_gpu()
    w = W.make(3)
    f = fem.rhs_planewave(w)
    probes = torch.tensor(w.probes, device="cuda")
    eps = torch.tensor(w.eps.real.copy(), device="cuda", requires_grad=True)
    fd_t = torch.tensor(f.T.copy(), device="cuda").t()
    geom = ag.geom_of(w)
    x = ag.solve(eps, fd_t, geom)
    J = _J(x, probes)
    J.backward()
    g = eps.grad.cpu().numpy()
    # oracle adjoint (independent sparse-LU solves)
    Jo, go = adjoint.gradient(w, f, w.probes)
    assert abs(J.item() - Jo) < 1e-9 * Jo
    assert np.abs(g - go).max() < 1e-8 * np.abs(go).max()
    # central finite differences on the seeded cells, forward through the library
    h = 1e-6
    for c in w.fd_cells:
        vals = []
        for sgn in (1.0, -1.0):
            e = w.eps.real.copy()
            e[c] += sgn * h
            with torch.no_grad():
                xs = ag.solve(torch.tensor(e, device="cuda"), fd_t, geom)
            vals.append(_J(xs, probes).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        # 1e-5 relative, plus the noise floor of a 1e-6 central difference of a
        # solve accurate to ~1e-12 (relative to the largest gradient entry)
        assert abs(fd - g[c]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (int(c), fd, g[c])


@pytest.mark.parametrize("precision", [d3m.FP64, d3m.MIXED])
def test_adjoint_solve_is_conjugate_transpose(precision):
    """y = A^{-H} b: check <A^{-1} f, b> = <f, A^{-H} b> on a small mesh."""
    _need_gpu()
    w = W.tiny(4, 4, 3, 2, 2, 1, seed=3, nrhs=2)
    s = d3m.Solver.from_workload(w, precision=precision)
    s.factor()
    rng = np.random.default_rng(1)
    keep = fem.free_edges(w)
    f = np.zeros((w.n_edges, 2), complex)
    b = np.zeros((w.n_edges, 2), complex)
    f[keep] = rng.standard_normal((len(keep), 2)) + 1j * rng.standard_normal((len(keep), 2))
    b[keep] = rng.standard_normal((len(keep), 2)) + 1j * rng.standard_normal((len(keep), 2))
    x, _ = s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    y, _ = s.solve_adjoint(torch.tensor(b.T.copy(), device="cuda").t())
    x, y = x.cpu().numpy(), y.cpu().numpy()
    lhs = np.sum(np.conj(b) * x, axis=0)
    rhs = np.sum(np.conj(y) * f, axis=0)
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()


def test_gradcheck_tiny_mesh():
    _need_gpu()
    w = W.tiny(2, 2, 2, 2, 1, 1, seed=5, nrhs=1)
    geom = ag.geom_of(w)
    f = fem.rhs_planewave(w)
    eps = torch.tensor(w.eps.real.copy(), device="cuda", dtype=torch.float64, requires_grad=True)
    ft = torch.tensor(f.T.copy(), device="cuda").t().contiguous().requires_grad_(True)
    probes = torch.tensor([0, 3, 7, 11], device="cuda")

    def fn(e, ff):
        return _J(ag.solve(e, ff.t().contiguous().t(), geom), probes)

    assert torch.autograd.gradcheck(fn, (eps, ft), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)


def test_tetrahedral_gradient_vs_oracle():
    """d3m_grad_eps on six tetrahedra per cell (per-cell 19 x 19 masses)
    against the oracle adjoint gradient."""
    _need_gpu()
    w = W.tetrahedral(W.tiny(5, 4, 4, 2, 2, 1, seed=12, nrhs=2), 0.1)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(5)
    probes = np.sort(rng.choice(w.n_edges, 8, replace=False))
    eps = torch.tensor(w.eps.real.copy(), device="cuda", requires_grad=True)
    fd_t = torch.tensor(f.T.copy(), device="cuda").t()
    x = ag.solve(eps, fd_t, ag.geom_of(w))
    J = _J(x, torch.tensor(probes, device="cuda"))
    J.backward()
    g = eps.grad.cpu().numpy()
    Jo, go = adjoint.gradient(w, f, probes)
    assert abs(J.item() - Jo) < 1e-9 * Jo
    assert np.abs(g - go).max() < 1e-8 * np.abs(go).max()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_general_mesh_gradient_vs_oracle(order):
    """d3m_grad_eps on a Delaunay mesh (one entry per tetrahedron, orientation
    signs inside the per-tetrahedron masses; 6, 12 or 20 dofs per
    tetrahedron) against the oracle adjoint."""
    _need_gpu()
    w = W.delaunay(5, 4, 4, 2, 2, 1, seed=12, nrhs=2, order=order)
    f = fem.rhs_planewave(w)
    rng = np.random.default_rng(5)
    probes = np.sort(rng.choice(w.n_edges, 8, replace=False))
    eps = torch.tensor(w.eps.real.copy(), device="cuda", requires_grad=True)
    fd_t = torch.tensor(f.T.copy(), device="cuda").t()
    x = ag.solve(eps, fd_t, ag.geom_of(w))
    J = _J(x, torch.tensor(probes, device="cuda"))
    J.backward()
    g = eps.grad.cpu().numpy()
    Jo, go = adjoint.gradient(w, f, probes)
    assert g.shape == (w.n_cells,)
    assert abs(J.item() - Jo) < 1e-9 * Jo
    assert np.abs(g - go).max() < 1e-8 * np.abs(go).max()
