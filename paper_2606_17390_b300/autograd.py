"""Differentiable displacement misfit: a torch.autograd.Function around hfe_adjoint.

``misfit(theta, solver, t, u_target, w)`` returns J(theta) = w sum_n ||u^n(theta) - u_target^n||^2
(paper Sec. 2.3) as a 0-d tensor; ``J.backward()`` gives dJ/dtheta, computed by the library's
discrete adjoint (Eq. dR_u, Eq. main_grad, Algorithm adjoint_ad) in the same call as J.
theta has the layout of hfe_material.theta: (11,) for a uniform material or (n_el, 11) per
element.  Argument marshalling only: every computation runs in libhfe.so.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["HfeMisfit", "misfit"]


class HfeMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver, t, u_target, w):
        th = theta.detach().to(torch.float64).cpu().numpy()
        solver.set_material(th, solver_theta_axes(solver))
        J, grad, stats = solver.adjoint(np.asarray(t, dtype=np.float64), u_target, w)
        ctx.save_for_backward(torch.as_tensor(grad.reshape(th.shape), dtype=theta.dtype, device=theta.device))
        ctx.stats = stats
        return torch.as_tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad, None, None, None, None


def solver_theta_axes(solver):
    return getattr(solver, "Theta_axes", None)


def misfit(theta: torch.Tensor, solver, t, u_target, w: float = 1.0) -> torch.Tensor:
    """J(theta) with an adjoint backward; ``u_target`` is [n_steps, n_dof] (host or device)."""
    return HfeMisfit.apply(theta, solver, t, u_target, float(w))
