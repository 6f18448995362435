"""torch.autograd wrappers over the C ABI.

FreeformTrace maps control heights P^z to the irradiance on the extended grid
(fr_trace_forward); its backward is the recompute adjoint (fr_trace_adjoint).
LossL2 is the squared-L2 loss against an interior target (fr_loss_l2);
LossFrobenius the paper's normalised Frobenius loss (fr_loss_frobenius).
TanhReparam maps unconstrained variables to control heights in (z_min, z_max)
plus an offset (fr_reparam_tanh / fr_reparam_tanh_adjoint).
"""
import torch

from . import api


class FreeformTrace(torch.autograd.Function):
    """E = trace(P^z); dL/dP^z by the adjoint kernel."""

    @staticmethod
    def forward(ctx, ctrl_z, problem, options=None):
        problem.set_ctrl(ctrl_z.detach())
        E = problem.forward(options)
        ctx.problem = problem
        ctx.options = options
        ctx.save_for_backward(ctrl_z)
        return E

    @staticmethod
    def backward(ctx, dLdE):
        (ctrl_z,) = ctx.saved_tensors
        ctx.problem.set_ctrl(ctrl_z.detach())
        g = ctx.problem.adjoint(dLdE.contiguous(), ctx.options)
        return g, None, None


class LossL2(torch.autograd.Function):
    """L = sum over interior pixels of (E - E_ref)^2 (float64 scalar)."""

    @staticmethod
    def forward(ctx, E, E_ref, problem):
        loss = torch.empty((), dtype=torch.float64, device=E.device)
        dLdE = torch.empty_like(E)
        api.fr_loss_l2(api.default_handle(), E.contiguous(), E_ref.contiguous(), problem.nx, problem.ny,
                       problem.nu_x, problem.nu_y, loss, dLdE)
        ctx.save_for_backward(dLdE)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dLdE,) = ctx.saved_tensors
        return dLdE * g.to(dLdE.dtype), None, None


class LossFrobenius(torch.autograd.Function):
    """L = ||E/sum E - E_ref/sum E_ref||_F / sqrt(nx ny) over the interior (float64 scalar)."""

    @staticmethod
    def forward(ctx, E, E_ref, problem):
        loss = torch.empty((), dtype=torch.float64, device=E.device)
        dLdE = torch.empty_like(E)
        api.fr_loss_frobenius(api.default_handle(), E.contiguous(), E_ref.contiguous(), problem.nx, problem.ny,
                              problem.nu_x, problem.nu_y, loss, dLdE)
        ctx.save_for_backward(dLdE)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dLdE,) = ctx.saved_tensors
        return dLdE * g.to(dLdE.dtype), None, None


class TanhReparam(torch.autograd.Function):
    """P = offset + z_min + (tanh(theta) + 1)(z_max - z_min)/2 (offset not differentiated)."""

    @staticmethod
    def forward(ctx, theta, z_min, z_max, offset=None):
        theta = theta.contiguous()
        P = torch.empty_like(theta)
        off = None if offset is None else offset.contiguous()
        api.fr_reparam_tanh(api.default_handle(), theta, off, theta.numel(), z_min, z_max, P)
        ctx.save_for_backward(theta)
        ctx.z = (z_min, z_max)
        return P

    @staticmethod
    def backward(ctx, dLdP):
        (theta,) = ctx.saved_tensors
        out = torch.empty_like(theta)
        api.fr_reparam_tanh_adjoint(api.default_handle(), theta, dLdP.contiguous(), theta.numel(), ctx.z[0],
                                    ctx.z[1], out)
        return out, None, None, None


def trace(ctrl_z, problem, options=None):
    return FreeformTrace.apply(ctrl_z, problem, options)


def loss_l2(E, E_ref, problem):
    return LossL2.apply(E, E_ref, problem)


def loss_frobenius(E, E_ref, problem):
    return LossFrobenius.apply(E, E_ref, problem)


def reparam_tanh(theta, z_min, z_max, offset=None):
    return TanhReparam.apply(theta, z_min, z_max, offset)
