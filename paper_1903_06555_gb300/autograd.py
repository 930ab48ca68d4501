"""Differentiable measurement operator.

PhiDegrid: y = Phi x (phi_degrid) as a torch.autograd.Function whose
backward is the hand-written adjoint gridding, grad_x = Re(Phi^H grad_y)
(phi_grid).  PhiGrid: x = Re(Phi^H y) whose backward is degridding.

PyTorch passes a complex gradient g = dL/dRe(y) + i dL/dIm(y) for a real
loss L, so dL = Re<g, dy> = Re<g, Phi dx> = <Re(Phi^H g), dx> for a real
image x: the real-linear adjoint phi_grid computes exactly that, fold
included (Sec. 3.1 adjoint, Sec. 3.3 fold).
"""
from __future__ import annotations

import torch


class PhiDegrid(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.degrid(x.contiguous())

    @staticmethod
    def backward(ctx, grad_y):
        plan = ctx.plan
        return plan.grid(grad_y.to(plan.complex_dtype).contiguous()), None


class PhiGrid(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, plan):
        ctx.plan = plan
        return plan.grid(y.contiguous())

    @staticmethod
    def backward(ctx, grad_x):
        plan = ctx.plan
        return plan.degrid(grad_x.to(plan.real_dtype).contiguous()), None


def degrid(x, plan):
    """y = Phi x, differentiable with respect to x."""
    return PhiDegrid.apply(x, plan)


def grid(y, plan):
    """x = Re(Phi^H y), differentiable with respect to y."""
    return PhiGrid.apply(y, plan)
