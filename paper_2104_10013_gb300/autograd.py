"""PyTorch autograd front end of the cPINN / XPINN loss.

`XpinnLoss.apply(theta, solver)` returns the scalar J(theta) = sum over
subdomains q of J(Theta_q) (Eqs. cPINNLoss / XPINNLoss) computed by the CUDA
library, and its backward returns the gradient the library's hand-written
jet reverse pass produced in the same call.  As in Algorithm 1, the gradient
with respect to Theta_q is that of J(Theta_q) alone, with the neighbours'
interface values held constant: it is the training direction of the method,
block by block, not the total derivative of the sum (which would also
differentiate the neighbours' losses through the shared interfaces).

theta must be a float32 CUDA tensor in the packed parameter layout; the
library computes in its own kernels and torch only holds the memory.
"""
from __future__ import annotations

import numpy as np
import torch

from . import problems as P


class XpinnLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, solver, weights: torch.Tensor):
        if not (theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()):
            raise ValueError("theta must be a contiguous float32 CUDA tensor")
        solver.set_params(theta)
        losses = torch.empty((solver.n_sub, P.N_TERMS), dtype=torch.float32, device=theta.device)
        grads = torch.empty_like(theta)
        solver.grad(losses=losses, grads=grads)
        ctx.save_for_backward(grads)
        ctx.losses = losses
        return (losses * weights).sum()

    @staticmethod
    def backward(ctx, g_out):
        (grads,) = ctx.saved_tensors
        return g_out * grads, None, None


def loss_weights(problem: P.Problem, device) -> torch.Tensor:
    """[n_sub, 5] weights (W_u of each net, W_F, W_I, W_flux | W_IF) as float32."""
    W = np.zeros((problem.n_sub, P.N_TERMS), np.float32)
    for q, s in enumerate(problem.subs):
        for n, w in enumerate(s.w_data):
            W[q, n] = w
        W[q, 2:] = (s.w_res, s.w_avg, s.w_iface)
    return torch.from_numpy(W).to(device)


def xpinn_loss(theta: torch.Tensor, solver, weights: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable J(theta) through the CUDA library."""
    if weights is None:
        weights = loss_weights(solver.pb, theta.device)
    return XpinnLoss.apply(theta, solver, weights)
