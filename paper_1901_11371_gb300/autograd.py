"""Differentiable H-IDBF-LU solve and far-field loss (adjoint form).

`hb_solve(f, b)` returns x = A^{-1} b (GMRES of libhb) and back-propagates by the
adjoint solve  A^H lambda = g  (hb_gmres with HB_OP_H, i.e. the conjugate-
transposed factors in reverse stage order and the preconditioner
L~^{-H} U~^{-H}).  `far_field(f, x, phi)` is the far zone of the scattered field
with backward F^H (hb_far_field_adjoint).

Complex gradients follow PyTorch's convention: for a real loss L(z) the
gradient is dL/d(Re z) + i dL/d(Im z).  For x = A^{-1} b this gives
grad_b = A^{-H} grad_x, and for E = F x, grad_x = F^H grad_E.
"""
from __future__ import annotations

import torch

import paper_1901_11371_gb300 as hb


class HBSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, f, rtol, restart, maxit):
        x, info = hb.hb_gmres(f, b.detach().contiguous(), rtol=rtol, restart=restart, maxit=maxit)
        ctx.f, ctx.rtol, ctx.restart, ctx.maxit = f, rtol, restart, maxit
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, g):
        lam, _ = hb.hb_gmres(ctx.f, g.contiguous(), op=hb.HB_OP_H, rtol=ctx.rtol, restart=ctx.restart,
                             maxit=ctx.maxit)
        return lam, None, None, None, None


class FarField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, phi_obs):
        ctx.f, ctx.phi = f, phi_obs
        return hb.hb_far_field(f, x.detach().contiguous(), phi_obs)

    @staticmethod
    def backward(ctx, g):
        return hb.hb_far_field_adjoint(ctx.f, g.contiguous(), ctx.phi), None, None


def hb_solve(f, b, rtol=1e-6, restart=30, maxit=1000):
    """x = A^{-1} b for b of shape (R, N) complex128 (physical excitation), differentiable in b."""
    return HBSolve.apply(b, f, rtol, restart, maxit)


def far_field(f, x, phi_obs_deg):
    """E(phi_q) for x of shape (R, N); output (R, nobs), differentiable in x."""
    return FarField.apply(x, f, phi_obs_deg)


def far_field_loss(f, b, target, phi_obs_deg, rtol=1e-6, restart=30, maxit=1000):
    """L(b) = sum_q |E_far(phi_q) - t_q|^2 with E_far the far field of x = A^{-1} b."""
    x = hb_solve(f, b, rtol, restart, maxit)
    e = far_field(f, x, phi_obs_deg)
    return torch.sum(torch.abs(e - target) ** 2)
