"""torch.autograd.Function faces of the discrete adjoint (argument marshalling only).

``SdcRun`` maps an initial state to the state after ``nsteps`` dSDC steps; its
backward calls the library's checkpointed adjoint (sdc_run_adjoint).
``SdcHeightLoss`` maps an initial state to the height-misfit loss
0.5 sum (h(T) - h_target)^2 and returns the gradient the library computed
together with the loss (sdc_adjoint_run).  Gradients of complex states follow
torch's convention (real part d/dRe, imaginary part d/dIm), which is the
library's.
"""
from __future__ import annotations

import torch


class SdcRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, nsteps: int, nsnapshots: int = 8):
        ctx.solver = solver
        ctx.nsteps = int(nsteps)
        ctx.nsnapshots = int(nsnapshots)
        ctx.save_for_backward(u0.detach())
        u = u0.detach().clone().contiguous()
        solver.run(u, ctx.nsteps)
        return u

    @staticmethod
    def backward(ctx, grad_out):
        (u0,) = ctx.saved_tensors
        g, _ = ctx.solver.run_adjoint(u0, ctx.nsteps, grad_out.contiguous(), ctx.nsnapshots)
        return g, None, None, None


class SdcHeightLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, nsteps: int, h_target, nsnapshots: int = 8):
        loss, grad = solver.adjoint_run(u0.detach().contiguous(), int(nsteps), h_target, int(nsnapshots))
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gl):
        (grad,) = ctx.saved_tensors
        return grad * gl, None, None, None, None


def sdc_run(u0, solver, nsteps: int, nsnapshots: int = 8):
    return SdcRun.apply(u0, solver, nsteps, nsnapshots)


def height_loss(u0, solver, nsteps: int, h_target, nsnapshots: int = 8):
    return SdcHeightLoss.apply(u0, solver, nsteps, h_target, nsnapshots)
