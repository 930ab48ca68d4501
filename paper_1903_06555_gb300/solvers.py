"""Consumers of the operator: the power-method normalisation of Phi
(Sec. 3.1: "the full operator Phi is normalized using the power method")
and a least-squares gradient descent on 1/2 ||Phi x - y||^2, standing in
for the paper's ADMM (Sec. 3.4; its wavelet prior is out of scope).

Every operator application is a phi_degrid / phi_grid call; the vector
updates are plain device tensor operations.
"""
from __future__ import annotations

import torch


def power_method(plan, iters: int = 20, seed: int = 0, x0=None):
    """Largest eigenvalue of Phi^H Phi (= ||Phi||^2) after `iters` steps of
    x <- Re(Phi^H Phi x) / ||.||.  Returns (estimate, history)."""
    n = plan.image_n
    if x0 is None:
        g = torch.Generator(device=plan.device).manual_seed(seed)
        x = torch.randn((n, n), generator=g, device=plan.device, dtype=plan.real_dtype)
    else:
        x = x0.to(plan.device, plan.real_dtype).clone()
    x /= torch.linalg.vector_norm(x)
    hist = []
    lam = 0.0
    for _ in range(iters):
        z = plan.grid(plan.degrid(x))
        lam = float(torch.linalg.vector_norm(z.double()))
        hist.append(lam)
        x = z / lam
    return lam, hist


def least_squares(plan, y, steps: int = 20, step: float | None = None, x0=None,
                  power_iters: int = 20):
    """Gradient descent x <- x - step Re(Phi^H (Phi x - y)) from x0 (zeros),
    step = 1 / ||Phi||^2 by default.  Returns (x, losses) with
    losses[k] = 1/2 ||Phi x_k - y||^2 before step k and after the last."""
    if step is None:
        lam, _ = power_method(plan, power_iters)
        step = 1.0 / lam
    n = plan.image_n
    x = torch.zeros((n, n), device=plan.device, dtype=plan.real_dtype) if x0 is None \
        else x0.to(plan.device, plan.real_dtype).clone()
    losses = []
    for _ in range(steps):
        r = plan.degrid(x) - y
        losses.append(0.5 * float(torch.sum(torch.abs(r.to(torch.complex128)) ** 2)))
        x = x - step * plan.grid(r)
    r = plan.degrid(x) - y
    losses.append(0.5 * float(torch.sum(torch.abs(r.to(torch.complex128)) ** 2)))
    return x, losses
