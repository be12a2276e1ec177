"""Torch-facing helpers over the C ABI: tensor allocation in the canonical layouts and
a torch.autograd.Function for sgn(H_W) b.

Every computation runs in the CUDA library (``lib``); this module only allocates
tensors, passes pointers and wires the adjoint into autograd.
"""
from __future__ import annotations

import torch

from . import lib


def spinor_shape(dims, nrhs=None):
    lx, ly, lz, lt = dims
    shp = (lt, lz, ly, lx, 4, 3)
    return shp if nrhs is None else (nrhs,) + shp


def force_shape(dims):
    lx, ly, lz, lt = dims
    return (4, lt, lz, ly, lx, 8)


def sgn_apply(ctx: "lib.Context", b: torch.Tensor, opts=None) -> torch.Tensor:
    """S_N b for a complex128 CUDA tensor of shape (..., Lt, Lz, Ly, Lx, 4, 3)."""
    b = b.contiguous()
    out = torch.empty_like(b)
    nrhs = b.numel() // (12 * ctx.V)
    ctx.sgn(b, out, nrhs, opts)
    return out


def overlap_apply(ctx: "lib.Context", m_q: float, b: torch.Tensor, opts=None) -> torch.Tensor:
    """D_ov(m_q) b (Eq. 1) for a complex128 CUDA tensor."""
    b = b.contiguous()
    out = torch.empty_like(b)
    nrhs = b.numel() // (12 * ctx.V)
    ctx.overlap(m_q, b, out, nrhs, opts)
    return out


class SignFunction(torch.autograd.Function):
    """out = S_N b on one source, differentiable in b and in the gauge links.

    ``omega`` is a real tensor of shape (4, Lt, Lz, Ly, Lx, 8): the su(3) coordinates of
    a left perturbation U_mu(x) -> exp(i omega_a lambda_a / 2) U_mu(x) about the links
    loaded in ``ctx``.  Its value must be zero (the forward uses the loaded links); its
    gradient is the link force.  For a real loss L, backward returns dL/db* (torch's
    convention: S_N^dag applied to the incoming gradient) and dL/d omega from the fused
    force kernel (ov_sgn_vjp).
    """

    @staticmethod
    def forward(fctx, b, omega, ctx, opts=None):
        if torch.count_nonzero(omega).item() != 0:
            raise ValueError("omega must be zero: it only carries the link gradient")
        out = sgn_apply(ctx, b, opts)
        fctx.ov = ctx
        fctx.opts = opts
        fctx.save_for_backward(b)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        (b,) = fctx.saved_tensors
        ctx = fctx.ov
        g = grad_out.contiguous()
        grad_b = torch.empty_like(b) if fctx.needs_input_grad[0] else None
        force = (torch.empty(force_shape(ctx.dims), dtype=torch.float64, device=b.device)
                 if fctx.needs_input_grad[1] else None)
        if grad_b is not None or force is not None:
            ctx.sgn_vjp(g, b.contiguous(), grad_b, force, fctx.opts)
        return grad_b, force, None, None


def sgn(ctx, b, omega=None, opts=None):
    """Differentiable S_N b (see SignFunction); omega defaults to a zero force carrier."""
    if omega is None:
        omega = torch.zeros(force_shape(ctx.dims), dtype=torch.float64, device=b.device)
    return SignFunction.apply(b, omega, ctx, opts)
