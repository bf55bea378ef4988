"""Python binding of the D^3M C ABI (include/d3m.h): argument marshalling only.

Every numeric step runs in libd3m.so (host set-up in C++, factorisation and
substitution in CUDA kernels).  There is no CPU fallback: if the library is
missing, importing raises; if no GPU is present, d3m_factor / d3m_solve fail
with D3M_ECUDA.  PyTorch supplies device memory and the stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libd3m.so")

D3M_OK, D3M_EINVAL, D3M_ENOMEM, D3M_ESINGULAR, D3M_ENOCONV, D3M_ETIMEOUT, D3M_ECUDA, D3M_ESTATE = range(8)
FP64, MIXED = 0, 1
SN_RANGE, SN_PARENT, SN_KIND, SN_STRUCT, M_MAP, LM, BLOCKS, LAMBDA, STATS, M_ENTRIES, LEVELS = range(11)

_SYMBOLS = ["d3m_setup", "d3m_factor", "d3m_solve", "d3m_solve_host", "d3m_rhs_planewave",
            "d3m_structure", "d3m_dense_ldlt", "d3m_dense_ldlt_noalloc", "d3m_export_front", "d3m_stats_get",
            "d3m_last_error", "d3m_free", "d3m_solve_adjoint", "d3m_grad_eps", "d3m_set_profile"]


BRICK, TET, TET_MESH = 0, 1, 2


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("element", ctypes.c_int32), ("vertices", ctypes.POINTER(ctypes.c_double)),
                ("n_vertices", ctypes.c_int64), ("n_tets", ctypes.c_int64),
                ("tets", ctypes.POINTER(ctypes.c_int64)), ("order", ctypes.c_int32)]


class Materials(ctypes.Structure):
    _fields_ = [("eps_r", ctypes.POINTER(ctypes.c_double)), ("pec_edge", ctypes.POINTER(ctypes.c_uint8))]


class Partition(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int32), ("py", ctypes.c_int32), ("pz", ctypes.c_int32),
                ("cx", ctypes.POINTER(ctypes.c_int32)), ("cy", ctypes.POINTER(ctypes.c_int32)),
                ("cz", ctypes.POINTER(ctypes.c_int32)), ("gx", ctypes.POINTER(ctypes.c_double)),
                ("gy", ctypes.POINTER(ctypes.c_double)), ("gz", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("leaf_max", ctypes.c_int32),
                ("refine_tol", ctypes.c_double), ("max_refine", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("profile", ctypes.c_int32), ("panel_kernel", ctypes.c_int32),
                ("update_kernel", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("autotune_cache", ctypes.c_char_p), ("lookahead", ctypes.c_int32),
                ("refine_method", ctypes.c_int32), ("gmres_restart", ctypes.c_int32), ("gmres_tol", ctypes.c_double),
                ("alpha_re", ctypes.c_double), ("alpha_im", ctypes.c_double), ("solve_kernel", ctypes.c_int32),
                ("lm_weight", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("resid", ctypes.POINTER(ctypes.c_double)), ("iters", ctypes.c_int32),
                ("max_resid", ctypes.c_double), ("inner_iters", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_edges", "n_free", "n_lm", "n_blocks", "n_subdomains", "n_m",
                                               "n_fronts", "n_levels", "max_front", "arena_bytes")] + \
               [(n, ctypes.c_double) for n in ("flops_interior", "flops_domain", "flops_k")] + \
               [("n_2x2", ctypes.c_int64), ("min_pivot_ratio", ctypes.c_double),
                ("launches_factor", ctypes.c_int64), ("launches_solve", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in ("flops_update", "flops_panel", "ms_assemble", "ms_panel",
                                               "ms_update", "ms_fwd", "ms_bwd", "ms_residual", "solve_flops",
                                               "ms_inverse")] + \
               [("tuned_levels_tc", ctypes.c_int64), ("tuned_levels_cs2", ctypes.c_int64),
                ("ms_tuning", ctypes.c_double), ("ms_tc", ctypes.c_double), ("flops_tc", ctypes.c_double)]

    def asdict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class D3MError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"D3M error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libd3m.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.d3m_setup.argtypes = [ctypes.POINTER(Mesh), ctypes.POINTER(Materials), ctypes.c_double,
                              ctypes.POINTER(Partition), ctypes.POINTER(Options), ctypes.POINTER(P)]
    lib.d3m_factor.argtypes = [P]
    lib.d3m_solve.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(SolveInfo)]
    lib.d3m_solve_host.argtypes = lib.d3m_solve.argtypes
    lib.d3m_solve_adjoint.argtypes = lib.d3m_solve.argtypes
    lib.d3m_grad_eps.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int32, P]
    lib.d3m_rhs_planewave.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int64]
    lib.d3m_structure.argtypes = [P, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.d3m_dense_ldlt.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, ctypes.c_int32]
    lib.d3m_dense_ldlt_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P]
    lib.d3m_stats_get.argtypes = [P, ctypes.POINTER(Stats)]
    lib.d3m_set_profile.argtypes = [P, ctypes.c_int32]
    lib.d3m_export_front.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), P, P, P]
    lib.d3m_last_error.argtypes = [P]
    lib.d3m_last_error.restype = ctypes.c_char_p
    lib.d3m_free.argtypes = [P]
    lib.d3m_free.restype = None
    _lib = lib
    return lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _colmajor(t, n):
    """(tensor, ld): t as an n x r column-major block (copy only if needed)."""
    if t.dim() == 1:
        t = t[:, None]
    r = t.shape[1]
    if t.stride(0) == 1 and (r == 1 or t.stride(1) >= n):
        return t, max(n, t.stride(1) if r > 1 else n)
    t = t.t().contiguous().t()
    return t, n


class Solver:
    """One D^3M problem: set-up on construction (host), factor() and solve()
    on the GPU.  Names follow the paper: K, K_D, D, lambda."""

    def __init__(self, nx, ny, nz, lx, ly, lz, eps, k, cx, cy, cz, pec=None, precision=FP64,
                 leaf_max=64, refine_tol=1e-10, max_refine=10, stream=None, profile=False, panel_kernel=0,
                 update_kernel=0, autotune=0, autotune_cache=None, lookahead=0, refine_method=0,
                 gmres_restart=0, gmres_tol=0.0, alpha=None, solve_kernel=0, lm_weight=0, element=BRICK,
                 vertices=None, tets=None, gcuts=None, order=1):
        """Lattice meshes: nx..lz, cuts cx, cy, cz (cell indices).  General
        tetrahedral meshes (element=TET_MESH): vertices (n, 3), tets (m, 4)
        and gcuts = (gx, gy, gz) coordinate cuts, order 1 (Whitney), 2 (two
        dofs per edge) or 3 (also two per face); nx..lz and cx..cz unused."""
        self.lib = load()
        self._eps = np.ascontiguousarray(np.asarray(eps, np.complex128).view(np.float64))
        self._vert = None if vertices is None else np.ascontiguousarray(np.asarray(vertices, np.float64))
        self._tets = None if tets is None else np.ascontiguousarray(np.asarray(tets, np.int64))
        self.n_cells = len(self._tets) if element == TET_MESH else nx * ny * nz
        self._gcuts = None if gcuts is None else [np.ascontiguousarray(np.asarray(g, np.float64)) for g in gcuts]
        self._cuts = [np.ascontiguousarray(np.asarray(c, np.int32)) for c in (cx, cy, cz)]
        self._pec = None if pec is None else np.ascontiguousarray(np.asarray(pec, np.uint8))
        mesh = Mesh(nx, ny, nz, lx, ly, lz, int(element),
                    None if self._vert is None else _ptr(self._vert, ctypes.c_double),
                    0 if self._vert is None else len(self._vert), 0 if self._tets is None else len(self._tets),
                    None if self._tets is None else _ptr(self._tets, ctypes.c_int64), int(order))
        mat = Materials(_ptr(self._eps, ctypes.c_double),
                        None if self._pec is None else _ptr(self._pec, ctypes.c_uint8))
        if self._gcuts is not None:
            part = Partition(*[len(g) - 1 for g in self._gcuts], *[_ptr(c, ctypes.c_int32) for c in self._cuts],
                             *[_ptr(g, ctypes.c_double) for g in self._gcuts])
        else:
            part = Partition(len(cx) - 1, len(cy) - 1, len(cz) - 1, *[_ptr(c, ctypes.c_int32) for c in self._cuts])
        self.precision = precision
        self.stream = stream
        self._cache = None if autotune_cache is None else str(autotune_cache).encode()
        opt = Options(precision, leaf_max, refine_tol, max_refine, _stream_handle(stream), int(profile),
                      int(panel_kernel), int(update_kernel), int(autotune), self._cache, int(lookahead),
                      int(refine_method), int(gmres_restart), float(gmres_tol),
                      0.0 if alpha is None else complex(alpha).real, 0.0 if alpha is None else complex(alpha).imag,
                      int(solve_kernel), int(lm_weight))
        h = ctypes.c_void_p()
        rc = self.lib.d3m_setup(ctypes.byref(mesh), ctypes.byref(mat), float(k), ctypes.byref(part),
                                ctypes.byref(opt), ctypes.byref(h))
        self.h = h
        self._check(rc)
        self.n_edges = int(self.stats()["n_edges"])

    @classmethod
    def from_workload(cls, w, precision=FP64, **kw):
        kw.setdefault("alpha", getattr(w, "alpha", None))
        kw.setdefault("lm_weight", getattr(w, "lm_weight", 0))
        kw.setdefault("element", {"tet": TET, "mesh": TET_MESH}.get(getattr(w, "element", "brick"), BRICK))
        kw.setdefault("vertices", getattr(w, "vertices", None))
        kw.setdefault("tets", getattr(w, "tets", None))
        kw.setdefault("gcuts", getattr(w, "gcuts", None))
        kw.setdefault("order", getattr(w, "order", 1))
        return cls(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.eps, w.k, w.cx, w.cy, w.cz, pec=w.pec_edge,
                   precision=precision, **kw)

    def _check(self, rc):
        if rc != D3M_OK:
            msg = self.lib.d3m_last_error(self.h) if self.h else b""
            raise D3MError(rc, (msg or b"").decode())

    def factor(self):
        self._check(self.lib.d3m_factor(self.h))

    def solve(self, rhs, x=None, resid=True):
        """rhs: torch complex128 CUDA tensor (n_edges, nrhs) with column-major
        layout (e.g. a .t() view of an (nrhs, n_edges) tensor) or any tensor
        (copied to that layout).  Returns (x, info dict)."""
        import torch
        rhs, ldb = _colmajor(rhs, self.n_edges)
        r = rhs.shape[1]
        if x is None:
            x = torch.empty((r, self.n_edges), dtype=torch.complex128, device=rhs.device).t()
        res = np.zeros(r)
        info = SolveInfo(_ptr(res, ctypes.c_double), 0, 0.0, 0)
        ldx = x.stride(1) if r > 1 else self.n_edges
        rc = self.lib.d3m_solve(self.h, ctypes.c_void_p(rhs.data_ptr()), ldb,
                                ctypes.c_void_p(x.data_ptr()), ldx, r, ctypes.byref(info))
        self._check(rc)
        return x, dict(resid=res, iters=info.iters, max_resid=info.max_resid, inner_iters=info.inner_iters)

    def solve_adjoint(self, rhs, y=None):
        """y = A^{-H} rhs with the same factors (device tensors, layout as solve)."""
        import torch
        rhs, ldb = _colmajor(rhs, self.n_edges)
        r = rhs.shape[1]
        if y is None:
            y = torch.empty((r, self.n_edges), dtype=torch.complex128, device=rhs.device).t()
        res = np.zeros(r)
        info = SolveInfo(_ptr(res, ctypes.c_double), 0, 0.0, 0)
        ldy = y.stride(1) if r > 1 else self.n_edges
        rc = self.lib.d3m_solve_adjoint(self.h, ctypes.c_void_p(rhs.data_ptr()), ldb,
                                        ctypes.c_void_p(y.data_ptr()), ldy, r, ctypes.byref(info))
        self._check(rc)
        return y, dict(resid=res, iters=info.iters, max_resid=info.max_resid, inner_iters=info.inner_iters)

    def grad_eps(self, x, y):
        """grad[c] = k^2 Re(sum_r conj(y)_c^T M_c x_c) on the device (float64, n_cells)."""
        import torch
        x, ldx = _colmajor(x, self.n_edges)
        y, ldy = _colmajor(y, self.n_edges)
        g = torch.empty(self.n_cells, dtype=torch.float64, device=x.device)
        rc = self.lib.d3m_grad_eps(self.h, ctypes.c_void_p(x.data_ptr()), ldx, ctypes.c_void_p(y.data_ptr()),
                                   ldy, x.shape[1], ctypes.c_void_p(g.data_ptr()))
        self._check(rc)
        return g

    def solve_host(self, rhs, x):
        """Host (ideally pinned) column-major complex128 arrays/tensors."""
        r = rhs.shape[1]
        res = np.zeros(r)
        info = SolveInfo(_ptr(res, ctypes.c_double), 0, 0.0, 0)
        rp = rhs.data_ptr() if hasattr(rhs, "data_ptr") else rhs.ctypes.data
        xp = x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        ld_r = rhs.stride(1) if hasattr(rhs, "data_ptr") else rhs.strides[1] // 16
        ld_x = x.stride(1) if hasattr(x, "data_ptr") else x.strides[1] // 16
        rc = self.lib.d3m_solve_host(self.h, ctypes.c_void_p(rp), ld_r, ctypes.c_void_p(xp), ld_x, r,
                                     ctypes.byref(info))
        self._check(rc)
        return dict(resid=res, iters=info.iters, max_resid=info.max_resid, inner_iters=info.inner_iters)

    def rhs_planewave(self, khat_pol6):
        kp = np.ascontiguousarray(np.asarray(khat_pol6, np.float64))
        r = kp.shape[0]
        out = np.zeros((self.n_edges, r), np.complex128, order="F")
        self._check(self.lib.d3m_rhs_planewave(self.h, kp.ctypes.data, r, out.ctypes.data, self.n_edges))
        return out

    def structure(self, which):
        n = ctypes.c_size_t(0)
        self._check(self.lib.d3m_structure(self.h, which, None, ctypes.byref(n)))
        dt = np.float64 if which in (LAMBDA, M_ENTRIES, LEVELS) else np.int64
        buf = np.zeros(max(n.value // 8, 1), dt)
        self._check(self.lib.d3m_structure(self.h, which, buf.ctypes.data, ctypes.byref(n)))
        buf = buf[: n.value // 8]
        if which in (SN_RANGE, SN_KIND, M_MAP):
            return buf.reshape(-1, 2)
        if which in (LM, BLOCKS):
            return buf.reshape(-1, 3)
        if which == LAMBDA:
            return buf.view(np.complex128)
        if which == M_ENTRIES:
            return buf.reshape(-1, 4)
        if which == LEVELS:
            return buf.reshape(-1, 10)
        return buf

    def lam(self, nrhs):
        v = self.structure(LAMBDA)
        return v.reshape(nrhs, -1).T

    def export_front(self, q):
        """(F (m, m) row-major view of the factored front, perm, dinv (p, 6))."""
        m, p = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.d3m_export_front(self.h, q, ctypes.byref(m), ctypes.byref(p), None, None, None))
        F = np.zeros((m.value, m.value), np.complex128)
        perm = np.zeros(max(p.value, 1), np.int32)
        dinv = np.zeros((max(p.value, 1), 6))
        self._check(self.lib.d3m_export_front(self.h, q, None, None, F.ctypes.data, perm.ctypes.data,
                                              dinv.ctypes.data))
        return F.T.copy(), perm[: p.value], dinv[: p.value]

    def set_profile(self, on):
        """Per-kernel-class event timing on/off for the following calls."""
        self._check(self.lib.d3m_set_profile(self.h, int(bool(on))))

    def stats(self):
        s = Stats()
        self._check(self.lib.d3m_stats_get(self.h, ctypes.byref(s)))
        return s.asdict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.d3m_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dense_ldlt(A, p, stream=None, panel_kernel=0):
    """Restricted Bunch-Kaufman partial LDL^T of a batch of complex-symmetric
    matrices (torch complex128 CUDA tensor (batch, m, m), lower triangle of
    each column-major matrix read: pass A.transpose(1, 2) layout, i.e. element
    (i, j) at A[b, j, i]).  Returns (A in place, perm, dinv, info)."""
    import torch
    lib = load()
    if A.dim() != 3 or A.dtype != torch.complex128 or not A.is_cuda or not A.is_contiguous():
        raise ValueError("dense_ldlt wants a contiguous complex128 CUDA tensor (batch, m, m)")
    b, m, _ = A.shape
    perm = torch.empty((b, m), dtype=torch.int32, device=A.device)
    dinv = torch.empty((b, max(p, 1), 6), dtype=torch.float64, device=A.device)
    info = torch.empty((b,), dtype=torch.int32, device=A.device)
    rc = lib.d3m_dense_ldlt(m, p, b, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                            ctypes.c_void_p(dinv.data_ptr()), ctypes.c_void_p(info.data_ptr()),
                            _stream_handle(stream), int(panel_kernel))
    if rc != D3M_OK:
        raise D3MError(rc, "d3m_dense_ldlt failed")
    return A, perm, dinv, info


def dense_ldlt_noalloc(A, p, stream=None):
    """As dense_ldlt through d3m_dense_ldlt_noalloc: for callers that cannot
    allocate (all scratch lives in the library's fixed device array).  The
    output tensors are the caller's; nothing is allocated by the library."""
    import torch
    lib = load()
    if A.dim() != 3 or A.dtype != torch.complex128 or not A.is_cuda or not A.is_contiguous():
        raise ValueError("dense_ldlt_noalloc wants a contiguous complex128 CUDA tensor (batch, m, m)")
    b, m, _ = A.shape
    perm = torch.empty((b, m), dtype=torch.int32, device=A.device)
    dinv = torch.empty((b, max(p, 1), 6), dtype=torch.float64, device=A.device)
    info = torch.empty((b,), dtype=torch.int32, device=A.device)
    rc = lib.d3m_dense_ldlt_noalloc(m, p, b, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                    ctypes.c_void_p(dinv.data_ptr()), ctypes.c_void_p(info.data_ptr()),
                                    _stream_handle(stream))
    if rc != D3M_OK:
        raise D3MError(rc, "d3m_dense_ldlt_noalloc failed")
    return A, perm, dinv, info
