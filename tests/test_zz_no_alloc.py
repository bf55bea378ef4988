"""The allocation-free front factorisation (d3m_dense_ldlt_noalloc) against the
regular entry point.

Some callers cannot allocate device memory (stream-ordered regions that must
not synchronise, allocator hooks, fixed memory budgets); for them the library
keeps the scratch of this one entry point in a fixed device array.  These
tests call it through the C ABI -- twice in a row, so the second call reuses
the array left over from the first -- and compare every output with
d3m_dense_ldlt on the same input; they check that a call leaves the device's
free memory unchanged, the empty pivot block (p = 0), a batch whose scratch
just fits the array and the rejection of one that does not.  The file is
collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2002_05018_gb300 import d3m  # noqa: E402

SCRATCH = 8 << 20   # D3M_NOALLOC_SCRATCH_BYTES
NB = 32


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(m, batch, seed, diag_scale):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(batch):
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        X = X + X.T
        X[np.diag_indices(m)] *= diag_scale
        mats.append(X)
    return np.ascontiguousarray(np.stack([M.T for M in mats]))


def _scratch_bytes(m, p, batch):
    """The documented scratch need: every table rounded up to 256 bytes."""
    r = lambda n: (n + 255) // 256 * 256
    b, pp = batch, max(p, 1)
    return (4 * r(4 * b) + 4 * r(8 * b) + r(16 * b * m * NB) + r(4 * b * pp) + 2 * r(16 * b * pp)
            + 2 * r(4 * b) + r(8 * b) + r(b * pp) + r(8 * b * 2 * NB) + r(8 * b))


def _outputs(m, p, b):
    perm = torch.empty((b, m), dtype=torch.int32, device="cuda")
    dinv = torch.empty((b, max(p, 1), 6), dtype=torch.float64, device="cuda")
    info = torch.empty((b,), dtype=torch.int32, device="cuda")
    return perm, dinv, info


def _call_noalloc(lib, A, p, perm, dinv, info):
    b, m, _ = A.shape
    v = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.d3m_dense_ldlt_noalloc(m, p, b, v(A), v(perm), v(dinv), v(info), None)


def _compare(host, p, A_na, perm_na, dinv_na, info_na, tag):
    A_ref = torch.tensor(host, device="cuda")
    A_ref, perm_ref, dinv_ref, info_ref = d3m.dense_ldlt(A_ref, p)
    torch.cuda.synchronize()
    assert torch.equal(info_na, info_ref) and int(info_na.abs().sum()) == 0, tag
    assert torch.equal(perm_na, perm_ref), tag
    scale_ref = A_ref.abs().max().item()
    assert (A_na - A_ref).abs().max().item() <= 1e-12 * scale_ref, tag
    if p > 0:
        assert (dinv_na[:, :p] - dinv_ref[:, :p]).abs().max().item() <= 1e-12 * max(
            1.0, dinv_ref[:, :p].abs().max().item()), tag


def test_noalloc_matches_allocating_entry_point_twice():
    _need_gpu()
    lib = d3m.load()
    for call, (m, p, batch, seed, scale) in enumerate([(200, 120, 3, 11, 0.3), (257, 257, 2, 12, 0.0)]):
        host = _case(m, batch, seed, scale)
        A_na = torch.tensor(host, device="cuda")
        perm, dinv, info = _outputs(m, p, batch)
        assert _call_noalloc(lib, A_na, p, perm, dinv, info) == d3m.D3M_OK
        torch.cuda.synchronize()   # the call only enqueues its work
        _compare(host, p, A_na, perm, dinv, info, call)


def test_noalloc_leaves_free_memory_unchanged():
    """After a first call (which looks the array up), a second call changes
    the device's free memory by nothing: it allocates nothing."""
    _need_gpu()
    lib = d3m.load()
    m, p, b = 160, 100, 4
    host = _case(m, b, 21, 0.5)
    A1, A2 = torch.tensor(host, device="cuda"), torch.tensor(host, device="cuda")
    o1, o2 = _outputs(m, p, b), _outputs(m, p, b)
    assert _call_noalloc(lib, A1, p, *o1) == d3m.D3M_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call_noalloc(lib, A2, p, *o2) == d3m.D3M_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(A1, A2) and all(torch.equal(x, y) for x, y in zip(o1, o2))


def test_noalloc_empty_pivot_block():
    """p = 0: nothing is eliminated; A is unchanged, perm is the identity."""
    _need_gpu()
    lib = d3m.load()
    m, b = 50, 2
    host = _case(m, b, 31, 1.0)
    A = torch.tensor(host, device="cuda")
    perm, dinv, info = _outputs(m, 0, b)
    assert _call_noalloc(lib, A, 0, perm, dinv, info) == d3m.D3M_OK
    torch.cuda.synchronize()
    assert torch.equal(A, torch.tensor(host, device="cuda"))
    assert torch.equal(perm.cpu(), torch.arange(m, dtype=torch.int32).repeat(b, 1))
    assert int(info.abs().sum()) == 0


def test_noalloc_batch_at_the_scratch_limit():
    """The largest batch of 64 x 64 fronts whose scratch fits the array is
    factored like d3m_dense_ldlt; one more matrix is refused with EINVAL
    before any device work (the outputs stay untouched)."""
    _need_gpu()
    lib = d3m.load()
    m = p = 64
    b = 1
    while _scratch_bytes(m, p, b + 1) <= SCRATCH:
        b += 1
    assert SCRATCH - _scratch_bytes(m, p, b) < _scratch_bytes(m, p, 1)
    host = _case(m, b + 1, 41, 0.2)
    A = torch.tensor(host[:b].copy(), device="cuda")
    perm, dinv, info = _outputs(m, p, b)
    assert _call_noalloc(lib, A, p, perm, dinv, info) == d3m.D3M_OK
    torch.cuda.synchronize()
    _compare(host[:b].copy(), p, A, perm, dinv, info, "limit")
    A2 = torch.tensor(host, device="cuda")
    perm2, dinv2, info2 = _outputs(m, p, b + 1)
    info2.fill_(-7)
    assert _call_noalloc(lib, A2, p, perm2, dinv2, info2) == d3m.D3M_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(A2, torch.tensor(host, device="cuda"))
    assert bool((info2 == -7).all())


def test_noalloc_rejects_oversized_request():
    _need_gpu()
    lib = d3m.load()
    # 16*32*m*batch bytes of workspace alone exceed the fixed scratch here; the
    # size check rejects the call before any buffer is touched
    m, batch = 4096, 8
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    rc = lib.d3m_dense_ldlt_noalloc(m, m, batch, ptr, ptr, ptr, ptr, None)
    assert rc == d3m.D3M_EINVAL
    assert torch.count_nonzero(buf).item() == 0
