"""torch.autograd wrappers over the C ABI.

FreeformTrace maps control heights P^z to the irradiance on the extended grid
(fr_trace_forward); its backward is the recompute adjoint (fr_trace_adjoint).
LossL2 is the squared-L2 loss against an interior target (fr_loss_l2).
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


def trace(ctrl_z, problem, options=None):
    return FreeformTrace.apply(ctrl_z, problem, options)


def loss_l2(E, E_ref, problem):
    return LossL2.apply(E, E_ref, problem)
