"""torch.autograd.Function front ends of the solver's adjoint (dw_cg_backward).

Tensors are CUDA complex128 in the canonical layout (U[V, 4, 3, 3],
psi[V, 4, 3], site = x + Lx*(y + Ly*(z + Lz*t))).  Gradients follow
PyTorch's convention for complex numbers: for a real loss L,
grad z = dL/dRe z + i dL/dIm z.

  CGSolve.apply(U, b, lattice, params)        x = (D^dag D)^{-1} b
  PseudofermionAction.apply(U, phi, lattice, params)
                                              S = phi^dag (D^dag D)^{-1} phi
                                                = |D (D^dag D)^{-1} phi|^2
Every solve and the link force run in the library's kernels; this module
moves tensors in and out of fields.
"""
from __future__ import annotations

import ctypes

import torch

from . import dw


def _field_from(t, lat, kind):
    f = dw.Field(lat, kind, dw.DW_F64)
    f.import_(t.contiguous())
    return f


def _stats():
    return (dw.dw_solver_stats * 2)()


class CGSolve(torch.autograd.Function):
    """x = (D^dag D)^{-1} b; backward gives grad_b = (D^dag D)^{-1} grad_x
    (a second solve) and grad_U = F(D x, grad_b) + F(D grad_b, x)."""

    @staticmethod
    def forward(ctx, U, b, lat, params=None, su3_project=False):
        p = params or dw.params(tol=1e-10, inner="f32")
        Uf = _field_from(U, lat, dw.DW_GAUGE)
        bf = _field_from(b, lat, dw.DW_SPINOR_FULL)
        xf = dw.Field(lat, dw.DW_SPINOR_FULL)
        dw.cg_solve_normal(Uf, bf, xf, p)
        x = xf.export()
        ctx.save_for_backward(U, b, x if not p.recompute_fwd else torch.empty(0))
        ctx.lat, ctx.p, ctx.su3 = lat, p, su3_project
        return x

    @staticmethod
    def backward(ctx, grad_x):
        U, b, x = ctx.saved_tensors
        lat, p = ctx.lat, ctx.p
        Uf = _field_from(U, lat, dw.DW_GAUGE)
        bf = _field_from(b, lat, dw.DW_SPINOR_FULL)
        gxf = _field_from(grad_x, lat, dw.DW_SPINOR_FULL)
        xf = _field_from(x, lat, dw.DW_SPINOR_FULL) if x.numel() else None
        gbf = dw.Field(lat, dw.DW_SPINOR_FULL)
        gUf = dw.Field(lat, dw.DW_GAUGE)
        dw.check(dw.dw_cg_backward(Uf.handle, bf.handle, gxf.handle, xf.handle if xf else None, gbf.handle,
                                   gUf.handle, 1 if ctx.su3 else 0, ctypes.byref(p), _stats(), dw.current_stream()))
        gU = gUf.export() if ctx.needs_input_grad[0] else None
        gb = gbf.export() if ctx.needs_input_grad[1] else None
        return gU, gb, None, None, None


class PseudofermionAction(torch.autograd.Function):
    """S = phi^dag (D^dag D)^{-1} phi (real); backward gives
    grad_phi = 2 X and grad_U = 2 F(D X, X), X = (D^dag D)^{-1} phi."""

    @staticmethod
    def forward(ctx, U, phi, lat, params=None, su3_project=False):
        p = params or dw.params(tol=1e-10, inner="f32")
        Uf = _field_from(U, lat, dw.DW_GAUGE)
        pf = _field_from(phi, lat, dw.DW_SPINOR_FULL)
        xf = dw.Field(lat, dw.DW_SPINOR_FULL)
        dw.cg_solve_normal(Uf, pf, xf, p)
        X = xf.export()
        # S = phi^dag X = X^dag D^dag D X = |D X|^2, from the library's FP64
        # grid reduction fused into the launch that applies D to X
        yf = dw.Field(lat, dw.DW_SPINOR_FULL)
        S = torch.tensor(float(dw.apply_norm(Uf, xf, yf)[0]), dtype=torch.float64, device=phi.device)
        ctx.save_for_backward(U, phi, X if not p.recompute_fwd else torch.empty(0))
        ctx.lat, ctx.p, ctx.su3 = lat, p, su3_project
        return S

    @staticmethod
    def backward(ctx, gS):
        U, phi, X = ctx.saved_tensors
        lat, p = ctx.lat, ctx.p
        Uf = _field_from(U, lat, dw.DW_GAUGE)
        pf = _field_from(phi, lat, dw.DW_SPINOR_FULL)
        xf = _field_from(X, lat, dw.DW_SPINOR_FULL) if X.numel() else None
        gpf = dw.Field(lat, dw.DW_SPINOR_FULL)
        gUf = dw.Field(lat, dw.DW_GAUGE)
        dw.check(dw.dw_cg_backward(Uf.handle, pf.handle, None, xf.handle if xf else None, gpf.handle, gUf.handle,
                                   1 if ctx.su3 else 0, ctypes.byref(p), _stats(), dw.current_stream()))
        g = gS.to(torch.float64)
        gU = gUf.export() * g if ctx.needs_input_grad[0] else None
        gphi = gpf.export() * g if ctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None
