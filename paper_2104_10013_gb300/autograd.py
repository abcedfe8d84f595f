"""PyTorch autograd front end of the cPINN / XPINN objective.

`xpinn_loss(theta, solver)` returns the scalar J(theta) = sum over subdomains
q of J(Theta_q) (Eqs. cPINNLoss / XPINNLoss, each term weighted by its
subdomain's loss weights), computed by the CUDA library (xpinn_objective),
and its backward returns the gradient the library's hand-written jet reverse
pass produced in the same call.  As in Algorithm 1, the gradient with
respect to Theta_q is that of J(Theta_q) alone, with the neighbours'
interface values held constant: it is the training direction of the method,
block by block, not the total derivative of the sum (which would also
differentiate the neighbours' losses through the shared interfaces).

theta must be a float32 CUDA tensor in the packed parameter layout; this
module only wraps the call: the library computes, torch holds the memory.
"""
from __future__ import annotations

import torch


class XpinnLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, solver):
        if not (theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()):
            raise ValueError("theta must be a contiguous float32 CUDA tensor")
        solver.set_params(theta)
        J = torch.empty(1, dtype=torch.float32, device=theta.device)
        J_sub = torch.empty(solver.n_sub, dtype=torch.float32, device=theta.device)
        losses = torch.empty((solver.n_sub, 5), dtype=torch.float32, device=theta.device)
        grads = torch.empty_like(theta)
        solver.objective(J=J, J_sub=J_sub, losses=losses, grads=grads)
        ctx.save_for_backward(grads)
        ctx.J_sub, ctx.losses = J_sub, losses
        return J.reshape(())

    @staticmethod
    def backward(ctx, g_out):
        (grads,) = ctx.saved_tensors
        return g_out * grads, None


def xpinn_loss(theta: torch.Tensor, solver) -> torch.Tensor:
    """Differentiable J(theta) through the CUDA library."""
    return XpinnLoss.apply(theta, solver)
