"""torch.autograd.Function over the D^3M solve (adjoint gradient, row a8).

Forward: x = A(eps)^{-1} f with A = S - k^2 sum_c eps_c M_c + jk T, factored by
the library for the given per-cell eps (d3m_setup + d3m_factor) and solved with
d3m_solve.  Backward, for an upstream gradient g = dJ/dx (PyTorch's complex
convention): A is complex symmetric, so the adjoint solve reuses the same LDL^T
factors -- y = A^{-H} g (d3m_solve_adjoint) -- and
    grad_f = y,   grad_eps_c = k^2 Re( conj(y)_c^T M_c x_c )   (d3m_grad_eps),
the derivative with respect to the real part of eps_c (dA/deps_c = -k^2 M_c).
"""
from __future__ import annotations

import numpy as np
import torch

from . import d3m


class D3MSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_re, f, geom):
        """eps_re: real float64 tensor (n_cells), the real part of eps_r (the
        imaginary part comes from geom['eps_im']); f: complex128 CUDA tensor
        (n_edges, nrhs); geom: dict(nx, ny, nz, lx, ly, lz, k, cx, cy, cz,
        eps_im, pec, precision[, element, vertices, tets, gcuts, order])."""
        eps = eps_re.detach().cpu().numpy() + 1j * np.asarray(geom.get("eps_im", 0.0))
        s = d3m.Solver(geom["nx"], geom["ny"], geom["nz"], geom["lx"], geom["ly"], geom["lz"], eps, geom["k"],
                       geom["cx"], geom["cy"], geom["cz"], pec=geom.get("pec"),
                       precision=geom.get("precision", d3m.FP64), element=geom.get("element", d3m.BRICK),
                       vertices=geom.get("vertices"), tets=geom.get("tets"), gcuts=geom.get("gcuts"),
                       order=geom.get("order", 1))
        s.factor()
        x, _ = s.solve(f)
        x = x.clone()
        ctx.solver = s
        ctx.save_for_backward(x)
        ctx.eps_device = eps_re.device
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        s = ctx.solver
        y, _ = s.solve_adjoint(grad_x)
        grad_eps = s.grad_eps(x, y).to(ctx.eps_device)
        # the factors live as long as the graph (backward may run more than
        # once with retain_graph); the solver is freed with the context
        return grad_eps, y, None


def solve(eps_re, f, geom):
    return D3MSolve.apply(eps_re, f, geom)


def geom_of(w, precision=d3m.FP64):
    return dict(nx=w.nx, ny=w.ny, nz=w.nz, lx=w.lx, ly=w.ly, lz=w.lz, k=w.k, cx=w.cx, cy=w.cy, cz=w.cz,
                eps_im=np.asarray(w.eps).imag.copy(), pec=w.pec_edge, precision=precision,
                element={"tet": d3m.TET, "mesh": d3m.TET_MESH}.get(getattr(w, "element", "brick"), d3m.BRICK),
                vertices=getattr(w, "vertices", None), tets=getattr(w, "tets", None),
                gcuts=getattr(w, "gcuts", None), order=getattr(w, "order", 1))
