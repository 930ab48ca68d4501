"""Direction-dependent effects (Sec. 5.2) on the GPU: per-visibility separable
DDE kernels convolved with the w-kernel (phi_degrid_dde / phi_grid_dde)
against the oracle's degrid_dde / grid_dde, with the quadrature path's gates
(1e-5 FP32, 1e-10 FP64), plus the identities that pin the oracle: a delta
is the plain operator, a shifted delta moves the visibility."""

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W
from test_gpu_parity import TOL32, TOL64, gpu_plan, oracle_geo, to_t

pytestmark = pytest.mark.gpu


def dtypes(precision):
    if precision == "f64":
        return torch.float64, torch.complex128, TOL64
    return torch.float32, torch.complex64, TOL32


@pytest.fixture(scope="module")
def case():
    geo = oracle_geo(128)
    uvw = W.uvw_disk(600, 60.0, 40.0, 71)
    h = geo.Npad / 2 * geo.du
    uvw[:2, 0] = [h - 0.4 * geo.du, -h + 0.3 * geo.du]   # combined boxes across the edge
    wts = np.linspace(0.5, 1.5, len(uvw))
    op = O.make_plan(uvw, geo, 3, False, weights=wts)
    a, b = W.dde_kernels(len(uvw), 5, 72)
    x = W.point_sources(128, 20, 73)
    yr = W.random_vis(len(uvw), 74)
    return dict(geo=geo, uvw=uvw, w=wts, op=op, a=a, b=b, x=x, yr=yr,
                y_ref=O.degrid_dde(op, x, a, b), x_ref=O.grid_dde(op, yr, a, b))


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_dde_matches_oracle(case, precision):
    plan = gpu_plan(case["uvw"], case["geo"], 3, False, precision, case["w"])
    rd, cd, tol = dtypes(precision)
    y = plan.degrid_dde(to_t(case["x"], rd), case["a"], case["b"]).cpu().numpy()
    assert O.rel_l2(y, case["y_ref"]) < tol
    x = plan.grid_dde(to_t(case["yr"], cd), case["a"], case["b"]).cpu().numpy()
    assert O.rel_l2(x, case["x_ref"]) < tol
    bad, taps = plan.stats()
    assert bad == 0 and taps > 0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_dde_adjoint_dot_product(case, precision):
    plan = gpu_plan(case["uvw"], case["geo"], 3, False, precision, case["w"])
    rd, cd, _ = dtypes(precision)
    x = to_t(W.random_image(128, 75), rd)
    y = to_t(W.random_vis(len(case["uvw"]), 76), cd)
    yd = plan.degrid_dde(x, case["a"], case["b"]).to(torch.complex128)
    lhs = torch.real(torch.vdot(y.to(torch.complex128), yd)).item()
    rhs = torch.sum(x.double() * plan.grid_dde(y, case["a"], case["b"]).double()).item()
    if precision == "f64":
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    else:
        # the DDE phases make <y, Phi x> cancel strongly; FP32 rounding is
        # bounded on the Cauchy-Schwarz scale |y| |Phi x|
        scale = (torch.linalg.vector_norm(y.to(torch.complex128)) * torch.linalg.vector_norm(yd)).item()
        assert abs(lhs - rhs) <= 1e-6 * scale


def test_dde_delta_and_shifted_delta(case):
    """D = delta is phi_degrid; D = delta at offset s is phi_degrid of the
    visibilities moved by -s pixels."""
    geo, uvw = case["geo"], case["uvw"]
    n = len(uvw)
    plan = gpu_plan(uvw, geo, 3, False, "f32")
    x = to_t(case["x"], torch.float32)
    one = np.ones((n, 1), np.complex64)
    assert O.rel_l2(plan.degrid_dde(x, one, one).cpu().numpy(), plan.degrid(x).cpu().numpy()) < 1e-6
    su, sv, h = -1, 2, 2
    a = np.zeros((n, 5), np.complex64)
    b = np.zeros((n, 5), np.complex64)
    a[:, su + h] = 1.0
    b[:, sv + h] = 1.0
    moved = uvw.copy()
    moved[:, 0] -= su * geo.du
    moved[:, 1] -= sv * geo.du
    inside = np.all(np.abs(moved[:, :2] / geo.du) < geo.Npad / 2 - 1, axis=1) & \
        np.all(np.abs(uvw[:, :2] / geo.du) < geo.Npad / 2 - 1, axis=1)
    plan_m = gpu_plan(moved, geo, 3, False, "f32")
    y_d = plan.degrid_dde(x, a, b).cpu().numpy()
    y_m = plan_m.degrid(x).cpu().numpy()
    assert O.rel_l2(y_d[inside], y_m[inside]) < 1e-6


def test_dde_in_a_radial_mode_plan(case):
    """In a radial-mode plan the w-kernel box comes from the visibility's
    Chebyshev series: the same operator within the quadrature tolerance."""
    plan = gpu_plan(case["uvw"], case["geo"], 3, False, "f32", case["w"], kernel_mode="radial")
    y = plan.degrid_dde(to_t(case["x"], torch.float32), case["a"], case["b"]).cpu().numpy()
    assert O.rel_l2(y, case["y_ref"]) < TOL32


def test_dde_refused_on_folded_plans(case):
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, "f32")
    with pytest.raises(phi.PhiError) as e:
        plan.degrid_dde(to_t(case["x"], torch.float32), case["a"], case["b"])
    assert e.value.status == phi.PHI_ERR_ARG


def test_dde_mwa_snapshot_unfolded_at_full_size():
    """The DDE bench workload: 2048^2, 1.95M visibilities, no fold, 16 stacks,
    J_D = 5: eight visibilities of two stacks against the oracle one by one,
    and the full-size dot test."""
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    geo = O.geometry_from(wl, tol_rel=1e-12, tol_abs=1e-12)
    a, b = W.dde_kernels(len(uvw), 5, 77)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    plan = gpu_plan(uvw, geo, 16, False, "f32")
    y = plan.degrid_dde(to_t(x, torch.float32), a, b).cpu().numpy()
    op = O.make_plan(uvw, geo, 16, False)
    assert np.allclose(plan.info()["wbar"], op.wbar, rtol=1e-11, atol=1e-11)
    sel = np.concatenate([np.nonzero((op.stack == k) & ~op.dropped)[0][:4] for k in (4, 11)])
    y_ref = O.degrid_dde(op, x, a, b, subset=sel)
    assert O.rel_l2(y[sel], y_ref) < TOL32
    assert plan.stats()[0] == 0
    xr = to_t(W.random_image(wl.image_n, 78), torch.float32)
    yv = to_t(W.random_vis(len(uvw), 79), torch.complex64)
    lhs = torch.real(torch.vdot(yv.to(torch.complex128),
                                plan.degrid_dde(xr, a, b).to(torch.complex128))).item()
    rhs = torch.sum(xr.double() * plan.grid_dde(yv, a, b).double()).item()
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


@pytest.fixture(scope="module")
def wide():
    """Supports of 38 taps (w up to 60 wavelengths in one stack): a whole
    w-kernel box per warp in shared memory would leave fewer than 24 warps
    per SM, so these plans take the two-pass path (boxes through a transient
    global buffer, then the separable convolution)."""
    geo = oracle_geo(128)
    uvw = W.uvw_disk(120, 60.0, 60.0, 81)
    wts = np.linspace(0.5, 1.5, len(uvw))
    op = O.make_plan(uvw, geo, 1, False, weights=wts)
    a, b = W.dde_kernels(len(uvw), 5, 82)
    x = W.point_sources(128, 20, 83)
    yr = W.random_vis(len(uvw), 84)
    return dict(geo=geo, uvw=uvw, w=wts, op=op, a=a, b=b, x=x, yr=yr,
                y_ref=O.degrid_dde(op, x, a, b), x_ref=O.grid_dde(op, yr, a, b))


@pytest.mark.parametrize("mode", ["quadrature", "radial"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_dde_two_pass_matches_oracle(wide, precision, mode):
    """Boxes by the per-tap quadrature or (radial) from the series, through
    the two-pass path, against the oracle at the quadrature path's gates."""
    plan = gpu_plan(wide["uvw"], wide["geo"], 1, False, precision, wide["w"], kernel_mode=mode)
    jw = plan.info()["max_jw"]
    assert jw >= 30
    rd, cd, tol = dtypes(precision)
    y = plan.degrid_dde(to_t(wide["x"], rd), wide["a"], wide["b"]).cpu().numpy()
    assert O.rel_l2(y, wide["y_ref"]) < tol
    x = plan.grid_dde(to_t(wide["yr"], cd), wide["a"], wide["b"]).cpu().numpy()
    assert O.rel_l2(x, wide["x_ref"]) < tol
    bad, taps = plan.stats()
    kept = int((~wide["op"].dropped).sum())
    assert bad == 0 and taps == 2 * kept * (jw + 4) ** 2


def test_dde_two_pass_delta_is_the_plain_operator(wide):
    """J_D = 1 with a = b = 1 through the two-pass path is phi_degrid /
    phi_grid (the boxes' taps are the plain kernel's, in another order of
    summation)."""
    plan = gpu_plan(wide["uvw"], wide["geo"], 1, False, "f32")
    n = len(wide["uvw"])
    one = np.ones((n, 1), np.complex64)
    x = to_t(wide["x"], torch.float32)
    assert O.rel_l2(plan.degrid_dde(x, one, one).cpu().numpy(), plan.degrid(x).cpu().numpy()) < 1e-6
    y = to_t(wide["yr"], torch.complex64)
    assert O.rel_l2(plan.grid_dde(y, one, one).cpu().numpy(), plan.grid(y).cpu().numpy()) < 1e-6
