"""Failure paths reached from the host without faulting the GPU: a pivot column
that is exactly zero (D3M_ESINGULAR through the front kernel) and refinement
that cannot reach its tolerance (D3M_ENOCONV, the last iterate left in x)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fem  # noqa: E402
from paper_2002_05018_gb300 import d3m, workloads as W  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("kernel", [0, 1])
def test_dense_front_zero_pivot_column(kernel):
    """Row and column 5 of the pivot block are zero: eliminating the other
    pivots never fills them, so when that column is reached its candidates
    and diagonal are all zero.  info = 1 + its pivot position, and perm puts
    original index 5 there; the other fronts of the batch are unaffected."""
    _need_gpu()
    rng = np.random.default_rng(3)
    m, p = 48, 20
    mats = []
    for b in range(2):
        F = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        F = F + F.T
        if b == 0:
            F[5, :p] = 0
            F[:p, 5] = 0
        mats.append(F)
    A = torch.tensor(np.ascontiguousarray(np.stack([M.T for M in mats])), device="cuda")
    A, perm, dinv, info = d3m.dense_ldlt(A, p, panel_kernel=kernel)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    perm = perm.cpu().numpy()
    assert info[0] >= 1 and perm[0, info[0] - 1] == 5
    assert info[1] == 0


def test_refinement_cap_reports_noconv_and_keeps_last_iterate():
    """A tolerance below the fp64 residual floor (1e-15) with max_refine = 2
    on workload 1 in mixed precision: the solve returns D3M_ENOCONV after two
    corrections and x holds the last iterate (far better than the factor
    precision alone)."""
    _need_gpu()
    w = W.make(1)
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED, max_refine=2, refine_tol=1e-15)
    s.factor()
    f = fem.rhs_planewave(w)
    rhs = torch.tensor(f.T.copy(), device="cuda").t()
    x = torch.zeros((f.shape[1], w.n_edges), dtype=torch.complex128, device="cuda").t()
    with pytest.raises(d3m.D3MError) as e:
        s.solve(rhs, x)
    assert e.value.code == d3m.D3M_ENOCONV
    assert "refinement stopped" in str(e.value)
    res = fem.rel_residual(w, x.cpu().numpy(), f).max()
    assert 0 < res < 1e-8
    s.close()


# Host-side fault injection (environment D3M_FAULT, read by d3m_setup): the
# failure is made on the host -- a refused allocation, a poisoned copy of the
# operator's entries, or a zero bound on the tensor-core kernel's first
# mbarrier waits -- and the library must report it through its status codes
# while the GPU context stays usable.

def _factor_with_fault(monkeypatch, fault, **kw):
    monkeypatch.setenv("D3M_FAULT", fault)
    w = W.make(1)
    s = d3m.Solver.from_workload(w, **kw)
    monkeypatch.delenv("D3M_FAULT")
    with pytest.raises(d3m.D3MError) as e:
        s.factor()
    s.close()
    return e.value


def _still_usable():
    w = W.tiny(4, 4, 4, 2, 1, 1, seed=1)
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED)
    s.factor()
    f = fem.rhs_planewave(w)
    x, info = s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    s.close()
    assert info["max_resid"] < 1e-10


def test_fault_alloc_reports_enomem(monkeypatch):
    _need_gpu()
    e = _factor_with_fault(monkeypatch, "alloc")
    assert e.code == d3m.D3M_ENOMEM and "D3M_FAULT" in str(e)
    _still_usable()


@pytest.mark.parametrize("prec", [d3m.FP64, d3m.MIXED])
def test_fault_zero_pivot_reports_singular(monkeypatch, prec):
    _need_gpu()
    e = _factor_with_fault(monkeypatch, "pivot", precision=prec)
    assert e.code == d3m.D3M_ESINGULAR and "zero pivot column" in str(e) and "front 0" in str(e)
    _still_usable()


def test_fault_nan_reports_non_finite_pivot(monkeypatch):
    _need_gpu()
    e = _factor_with_fault(monkeypatch, "nan", precision=d3m.MIXED)
    assert e.code == d3m.D3M_ESINGULAR and "not finite" in str(e)
    _still_usable()


def test_fault_expired_wait_reports_timeout(monkeypatch):
    """Every first mbarrier wait of the tensor-core product kernel is bounded
    by zero polls: each tile raises the error flag, waits (bounded) for its own
    loads and MMAs, frees its TMEM and returns; d3m_factor reports
    D3M_ETIMEOUT and the next context factors and solves normally."""
    _need_gpu()
    e = _factor_with_fault(monkeypatch, "timeout", precision=d3m.MIXED, update_kernel=2)
    assert e.code == d3m.D3M_ETIMEOUT
    _still_usable()


def test_fault_expired_wait_in_solve_reports_timeout(monkeypatch):
    """The same bound on the tensor-core substitution products: the factor
    completes, d3m_solve reports D3M_ETIMEOUT (every tile gave up and wrote
    nothing), and the next context factors and solves normally."""
    _need_gpu()
    monkeypatch.setenv("D3M_FAULT", "solve_timeout")
    w = W.make(1)
    s = d3m.Solver.from_workload(w, precision=d3m.MIXED)
    monkeypatch.delenv("D3M_FAULT")
    s.factor()
    f = fem.rhs_planewave(w)
    with pytest.raises(d3m.D3MError) as e:
        s.solve(torch.tensor(f.T.copy(), device="cuda").t())
    assert e.value.code == d3m.D3M_ETIMEOUT and "substitution" in str(e.value)
    s.close()
    _still_usable()
