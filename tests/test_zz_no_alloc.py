"""The allocation-free front factorisation (d3m_dense_ldlt_noalloc) against the
regular entry point.

Some callers cannot allocate device memory (stream-ordered regions that must
not synchronise, allocator hooks, fixed memory budgets); for them the library
keeps the scratch of this one entry point in a fixed device array.  This test
calls it through the C ABI twice in a row -- the second call reuses the array
left over from the first -- and compares every output with d3m_dense_ldlt on
the same input.  It lives in its own file, collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2002_05018_gb300 import d3m  # noqa: E402


def _case(m, batch, seed, diag_scale):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(batch):
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        X = X + X.T
        X[np.diag_indices(m)] *= diag_scale
        mats.append(X)
    return np.ascontiguousarray(np.stack([M.T for M in mats]))


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for call, (m, p, batch, seed, scale) in enumerate([(200, 120, 3, 11, 0.3), (257, 257, 2, 12, 0.0)]):
        host = _case(m, batch, seed, scale)
        A_ref = torch.tensor(host, device="cuda")
        A_ref, perm_ref, dinv_ref, info_ref = d3m.dense_ldlt(A_ref, p)
        A_na = torch.tensor(host, device="cuda")
        A_na, perm_na, dinv_na, info_na = d3m.dense_ldlt_noalloc(A_na, p)
        torch.cuda.synchronize()
        assert torch.equal(info_na, info_ref) and int(info_na.abs().sum()) == 0, call
        assert torch.equal(perm_na, perm_ref), call
        scale_ref = A_ref.abs().max().item()
        assert (A_na - A_ref).abs().max().item() <= 1e-12 * scale_ref, call
        assert (dinv_na[:, :p] - dinv_ref[:, :p]).abs().max().item() <= 1e-12 * max(
            1.0, dinv_ref[:, :p].abs().max().item()), call


def test_noalloc_rejects_oversized_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    lib = d3m.load()
    # 16*32*m*batch bytes of workspace alone exceed the fixed scratch here; the
    # size check rejects the call before any buffer is touched
    m, batch = 4096, 8
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    rc = lib.d3m_dense_ldlt_noalloc(m, m, batch, ptr, ptr, ptr, ptr, None)
    assert rc == d3m.D3M_EINVAL
    assert torch.count_nonzero(buf).item() == 0
