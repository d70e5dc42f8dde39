"""torch.autograd entry points over the adjoint kernels.

``QaoaExpectation.apply(gamma, beta, sim)`` returns <C>(gamma, beta) of a
``Simulator`` as a float64 tensor. When either angle tensor requires a
gradient, the forward call runs ``qaoa_grad_angles`` (forward pass, <C>, and
the adjoint sweep back through the inverse layers with lambda = C psi), so
backward only scales the stored d<C>/d(gamma_k, beta_k) by the incoming
gradient. ``lr_expectation`` builds the linear-ramp angles
gamma_k = (k+1)/p dgamma, beta_k = (1 - k/p) dbeta (Sec. II-B) with torch ops,
so autograd applies the chain rule to (dgamma, dbeta).
"""
from __future__ import annotations

import torch


class QaoaExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma, beta, sim):
        g = gamma.detach().to(torch.float64).cpu().numpy()
        b = beta.detach().to(torch.float64).cpu().numpy()
        if gamma.requires_grad or beta.requires_grad:
            r = sim.grad_angles(g, b)
            ctx.save_for_backward(torch.as_tensor(r["g_gamma"], dtype=torch.float64),
                                  torch.as_tensor(r["g_beta"], dtype=torch.float64))
            val = r["exp_c"]
        else:
            sim.run_angles(g, b)
            val = sim.expect()["exp_c"]
        return torch.tensor(val, dtype=torch.float64, device=gamma.device)

    @staticmethod
    def backward(ctx, grad_out):
        gg, gb = ctx.saved_tensors
        go = grad_out.detach().to(torch.float64).cpu()
        return (go * gg).to(grad_out.device), (go * gb).to(grad_out.device), None


def expectation(sim, gamma: torch.Tensor, beta: torch.Tensor) -> torch.Tensor:
    """<C> of ``sim`` after the layers (gamma_k, beta_k), differentiable in both."""
    return QaoaExpectation.apply(gamma, beta, sim)


def lr_expectation(sim, p: int, dgamma: torch.Tensor, dbeta: torch.Tensor) -> torch.Tensor:
    """<C> under the LR schedule, differentiable in (dgamma, dbeta)."""
    k = torch.arange(p, dtype=torch.float64, device=dgamma.device)
    gamma = (k + 1) / p * dgamma
    beta = (1 - k / p) * dbeta
    return QaoaExpectation.apply(gamma, beta, sim)
