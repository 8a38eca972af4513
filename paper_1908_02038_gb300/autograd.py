"""torch.autograd bindings of the differentiable form (RGL, FP64).

``RGLEnergy``: E(x, theta) with the hand-written backward of the library
(dE/dx = -F, dE/dtheta).  ``RGLRelax``: x*(theta), the FIRE 2.0 minimum
reached from x0, whose backward is the implicit gradient (Hessian-vector
products + conjugate gradients in the library).  Argument marshalling only:
every value comes from the CUDA library through the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (FireHandle, fire_minimize_dev, fire_rgl_energy_grad_dev,
               fire_rgl_implicit_grad_dev, fire_set_rgl_params)


def _theta_list(theta: torch.Tensor):
    return [float(v) for v in theta.detach().cpu().reshape(4)]


class RGLEnergy(torch.autograd.Function):
    """E = RGLEnergy.apply(pos, theta, handle, box); pos: CUDA float64 (N, 3),
    theta: float64 (4,) = (A, xi, p, q)."""

    @staticmethod
    def forward(ctx, pos, theta, handle: FireHandle, box):
        pos_c = pos.detach().contiguous()
        forces = torch.empty_like(pos_c)
        e, de = fire_rgl_energy_grad_dev(handle.h, pos_c, box, _theta_list(theta), forces)
        ctx.save_for_backward(forces, torch.tensor(de, dtype=theta.dtype, device=theta.device))
        return torch.tensor(e, dtype=pos.dtype, device=pos.device)

    @staticmethod
    def backward(ctx, grad_e):
        forces, de = ctx.saved_tensors
        g = grad_e.to(forces.device)
        return -forces * g, de * grad_e.to(de.device), None, None


class RGLRelax(torch.autograd.Function):
    """x* = RGLRelax.apply(x0, theta, handle, box, ftol, maxiter, cg_tol):
    FIRE 2.0 relaxation of x0 with parameters theta; the backward returns
    dL/dtheta = lambda . dF/dtheta with H lambda = dL/dx* (and no gradient
    for x0, whose small changes do not move the minimum)."""

    @staticmethod
    def forward(ctx, x0, theta, handle: FireHandle, box, ftol=1e-10, maxiter=200000,
                cg_tol=1e-10):
        th = _theta_list(theta)
        fire_set_rgl_params(handle.h, th)
        x = x0.detach().contiguous().clone()
        res = fire_minimize_dev(handle.h, x, box, ftol, maxiter)
        ctx.handle, ctx.box, ctx.theta, ctx.cg_tol = handle, box, th, cg_tol
        ctx.result = res
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        g = grad_x.detach().contiguous().to(torch.float64)
        dl, _ = fire_rgl_implicit_grad_dev(ctx.handle.h, x, ctx.box, ctx.theta, g, ctx.cg_tol)
        return None, torch.tensor(dl, dtype=torch.float64), None, None, None, None, None


def theta_tensor(params: dict, requires_grad: bool = True) -> torch.Tensor:
    return torch.tensor([params["A"], params["xi"], params["p"], params["q"]],
                        dtype=torch.float64, requires_grad=requires_grad)


__all__ = ["RGLEnergy", "RGLRelax", "theta_tensor", "np"]
