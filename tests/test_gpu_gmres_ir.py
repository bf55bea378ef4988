"""GMRES-based iterative refinement on the GPU (d3m_options.refine_method = 1)
against the oracle, and against plain refinement where that stalls.

The stalling case is a quasi-static one: a 6x6x6 brick mesh with 3e-4
wavelength cells (box 1.8e-3 wavelengths), lossless.  The curl-curl operator
dominates k^2 eps_r M by (kh)^-2, so the condition number is about 7e6; with
complex64 factors (unit roundoff 6e-8) plain refinement contracts too slowly
for 1e-10 in 10 steps, while flexible GMRES preconditioned by the same
factors reaches it (the same case behaves so with the oracle's complex64
sparse LU, tests/test_oracle_gmres_ir.py's reference implementation)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fem  # noqa: E402
from paper_2002_05018_gb300 import d3m, workloads as W  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solve(w, f, **kw):
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED, **kw)
    s.factor()
    rhs = torch.tensor(f.T.copy(), device="cuda").t()
    x = torch.zeros((f.shape[1], w.n_edges), dtype=torch.complex128, device="cuda").t()
    try:
        _, info = s.solve(rhs, x)
        code = d3m.D3M_OK
    except d3m.D3MError as e:
        info, code = None, e.code
    out = x.cpu().numpy()
    s.close()
    return out, info, code


def test_gmres_ir_where_plain_refinement_stalls():
    _need_gpu()
    w = W.tiny(6, 6, 6, 2, 2, 1, seed=3, lossy=False, h=3e-4)
    f = fem.rhs_planewave(w)
    xg = fem.solve_global(w, f)
    xp, ip, cp = _solve(w, f, max_refine=10)
    assert cp == d3m.D3M_ENOCONV or ip["iters"] >= 6
    xm, im, cm = _solve(w, f, max_refine=10, refine_method=1, gmres_tol=1e-6)
    assert cm == d3m.D3M_OK
    assert im["max_resid"] <= 1e-10 and im["iters"] <= 4 and im["inner_iters"] > 0
    assert fem.rel_residual(w, xm, f).max() <= 1e-10
    assert np.abs(xm - xg).max() <= 1e-8 * np.abs(xg).max()


@pytest.mark.parametrize("wk", [1, 3])
def test_gmres_ir_matches_oracle(wk):
    """On the ordinary workloads GMRES-IR reaches the criterion in no more
    outer steps than plain refinement and agrees with the oracle."""
    _need_gpu()
    w = W.make(wk)
    f = fem.rhs_planewave(w)
    xg = fem.solve_global(w, f)
    xp, ip, cp = _solve(w, f)
    xm, im, cm = _solve(w, f, refine_method=1)
    assert cp == d3m.D3M_OK and cm == d3m.D3M_OK
    assert im["iters"] <= ip["iters"] and im["max_resid"] <= 1e-10
    assert np.abs(xm - xg).max() <= 1e-8 * np.abs(xg).max()
