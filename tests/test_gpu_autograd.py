"""Differentiation (autograd with the hand-written adjoint as backward) and
the operator's consumers (power method, least squares), on the GPU."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
from paper_1903_06555_gb300 import autograd as PA
from paper_1903_06555_gb300 import solvers
import workloads as W

pytestmark = pytest.mark.gpu


def small(precision="f64", n=16, m=40, k=2, fold=True):
    geo = O.Geometry(n, 2.0, 0.3, 4.0, tol_rel=1e-13, tol_abs=1e-13)
    uvw = W.uvw_disk(m, 20.0, 10.0, 8)
    tol = 1e-12 if precision == "f64" else 1e-6
    plan = phi.Plan(torch.from_numpy(uvw), image_n=n, fov_rad=0.3, n_stacks=k, conj_fold=int(fold),
                    precision=precision, quad_rel_tol=tol, quad_abs_tol=tol)
    return geo, uvw, plan


def test_gradcheck_degrid_and_grid():
    geo, uvw, plan = small()
    x = torch.randn(16, 16, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: PA.degrid(t, plan), (x,), eps=1e-6, atol=1e-7)
    y = torch.randn(40, dtype=torch.complex128, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: PA.grid(t, plan), (y,), eps=1e-6, atol=1e-7)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_backward_matches_oracle_adjoint(precision):
    """grad of 1/2 ||Phi x - y||^2 is Re(Phi^H (Phi x - y)), against the oracle."""
    geo, uvw, plan = small(precision, n=32, m=200, k=3)
    op = O.make_plan(uvw, geo, 3, True)
    x_np = W.random_image(32, 11)
    y_np = W.random_vis(200, 12)
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    x = torch.from_numpy(x_np).to("cuda", rd).requires_grad_(True)
    y = torch.from_numpy(y_np).to("cuda", cd)
    loss = 0.5 * torch.sum(torch.abs(PA.degrid(x, plan) - y) ** 2)
    loss.backward()
    ref = O.grid(op, O.degrid(op, x_np) - y_np)
    err = O.rel_l2(x.grad.double().cpu().numpy(), ref)
    assert err < (1e-10 if precision == "f64" else 1e-5), err


@pytest.fixture(scope="module")
def diff_workload():
    wl = W.differentiable()
    uvw = W.uvw_for(wl)
    plan = phi.Plan(torch.from_numpy(uvw), image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg),
                    n_stacks=wl.n_stacks, conj_fold=int(wl.conj_fold), max_support=192)
    x_true = torch.from_numpy(W.point_sources(wl.image_n, wl.n_sources, wl.seed)).cuda().float()
    y = plan.degrid(x_true)
    return wl, plan, x_true, y


def test_differentiable_config_finite_differences(diff_workload):
    """4096^2 image, 10M visibilities, 16 stacks: the gradient of
    L = 1/2 ||Phi x - y||^2 along a direction supported on 64 random pixels
    equals the central difference (exact for a quadratic, up to rounding)."""
    wl, plan, x_true, y = diff_workload
    n = wl.image_n
    rng = np.random.default_rng(3)
    pix = rng.choice(n * n, 64, replace=False)
    v = torch.zeros(n * n, device="cuda")
    v[torch.from_numpy(pix).cuda()] = torch.from_numpy(rng.standard_normal(64)).cuda().float()
    v = v.view(n, n)
    x = (0.5 * x_true).requires_grad_(True)
    loss = 0.5 * torch.sum(torch.abs(PA.degrid(x, plan) - y).double() ** 2)
    loss.backward()
    g_dir = float(torch.sum(x.grad.double() * v.double()))

    def L(t):
        r = plan.degrid(t) - y
        return 0.5 * float(torch.sum(torch.abs(r.to(torch.complex128)) ** 2))

    eps = 1e-2 * float(x_true.abs().max())
    fd = (L(x.detach() + eps * v) - L(x.detach() - eps * v)) / (2 * eps)
    assert abs(fd - g_dir) <= 2e-3 * abs(g_dir), (fd, g_dir)


def test_differentiable_config_power_method_and_descent(diff_workload):
    """20 power iterations for ||Phi||^2 (Sec. 3.1), then 20 steps of
    gradient descent with step 1/||Phi||^2: the loss decreases monotonically."""
    wl, plan, x_true, y = diff_workload
    lam, hist = solvers.power_method(plan, 20)
    assert lam > 0 and abs(hist[-1] - hist[-2]) < 1e-2 * hist[-1]
    x, losses = solvers.least_squares(plan, y, steps=20, step=1.0 / lam)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.5 * losses[0]
