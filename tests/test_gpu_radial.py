"""Radial interpolation mode (PHI_KERNEL_RADIAL): per visibility the w-kernel
is integrated by the same adaptive quadrature at the Chebyshev points of
pieces of [0, rho_max], and every tap is evaluated from its piece's series in
rho.  It computes the same operator as the per-tap quadrature within the
quadrature tolerance, so the gates are the quadrature path's: the oracle's
per-tap operator to 1e-5 (FP32) and 1e-10 (FP64)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W
from test_gpu_parity import CASES, TOL32, TOL64, gpu_plan, oracle_geo, to_t

pytestmark = pytest.mark.gpu


def radial_plan(uvw, geo, k=1, fold=False, precision="f32", weights=None, **kw):
    return gpu_plan(uvw, geo, k, fold, precision, weights, kernel_mode="radial", **kw)


def dtypes(precision):
    if precision == "f64":
        return torch.float64, torch.complex128, TOL64
    return torch.float32, torch.complex64, TOL32


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    n, k, fold, rule, weighted = CASES[request.param]
    geo = oracle_geo(128)
    uvw = W.uvw_disk(n, 60.0, 40.0, 21)
    h = geo.Npad / 2 * geo.du
    uvw[:4, 0] = [h - 0.3 * geo.du, -h + 0.2 * geo.du, 1.05 * h, 0.1]
    uvw[:4, 1] = [0.4, h - 1.1 * geo.du, 0.0, -1.2 * h]
    wts = np.linspace(0.25, 2.0, n) if weighted else None
    x = W.point_sources(128, 20, 21)
    rule_o = O.SUPPORT_VIS if rule == "vis" else O.SUPPORT_STACK
    op = O.make_plan(uvw, geo, k, fold, weights=wts, support_rule=rule_o)
    yr = W.random_vis(n, 22)
    return dict(geo=geo, uvw=uvw, w=wts, x=x, k=k, fold=fold, rule=rule, op=op, yr=yr,
                y_ref=O.degrid(op, x), x_ref=O.grid(op, yr))


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_radial_degrid_and_grid_match_oracle(case, precision):
    plan = radial_plan(case["uvw"], case["geo"], case["k"], case["fold"], precision, case["w"],
                       support_rule=case["rule"])
    assert plan.info()["kernel_mode"] == phi.PHI_KERNEL_RADIAL
    rd, cd, tol = dtypes(precision)
    y = plan.degrid(to_t(case["x"], rd)).cpu().numpy()
    assert O.rel_l2(y, case["y_ref"]) < tol
    assert np.all(y[case["op"].dropped] == 0)
    x = plan.grid(to_t(case["yr"], cd)).cpu().numpy()
    assert O.rel_l2(x, case["x_ref"]) < tol
    bad, taps = plan.stats()
    assert bad == 0 and taps > 0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_radial_adjoint_dot_product(case, precision):
    plan = radial_plan(case["uvw"], case["geo"], case["k"], case["fold"], precision, case["w"],
                       support_rule=case["rule"])
    rd, cd, _ = dtypes(precision)
    x = to_t(W.random_image(128, 3), rd)
    y = to_t(W.random_vis(len(case["uvw"]), 4), cd)
    lhs = torch.real(torch.vdot(y.to(torch.complex128), plan.degrid(x).to(torch.complex128))).item()
    rhs = torch.sum(x.double() * plan.grid(y).double()).item()
    assert abs(lhs - rhs) <= (1e-12 if precision == "f64" else 2e-5) * abs(lhs)


def test_radial_is_deterministic(case):
    p1 = radial_plan(case["uvw"], case["geo"], case["k"], case["fold"], "f32", case["w"],
                     support_rule=case["rule"])
    p2 = radial_plan(case["uvw"], case["geo"], case["k"], case["fold"], "f32", case["w"],
                     support_rule=case["rule"])
    x = to_t(case["x"], torch.float32)
    assert torch.equal(p1.degrid(x), p2.degrid(x))


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_radial_on_grid_points_matches_oracle(precision):
    """Visibilities on grid points and one ulp either side: a tap at rho = 0
    (the first Chebyshev piece's left end) and the exact box."""
    geo = oracle_geo(128)
    uvw = W.uvw_disk(500, 60.0, 40.0, 81)
    k = np.round(uvw[:300, :2] / geo.du)
    uvw[:100, :2] = k[:100] * geo.du
    uvw[100:200, :2] = np.nextafter(k[100:200], -np.inf) * geo.du
    uvw[200:300, :2] = np.nextafter(k[200:300], np.inf) * geo.du
    op = O.make_plan(uvw, geo, 3, True)
    x = W.point_sources(128, 20, 82)
    yr = W.random_vis(len(uvw), 83)
    plan = radial_plan(uvw, geo, 3, True, precision)
    rd, cd, tol = dtypes(precision)
    y = plan.degrid(to_t(x, rd)).cpu().numpy()
    y_ref = O.degrid(op, x)
    assert O.rel_l2(y, y_ref) < tol and O.rel_l2(y[:300], y_ref[:300]) < tol
    assert O.rel_l2(plan.grid(to_t(yr, cd)).cpu().numpy(), O.grid(op, yr)) < tol


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_radial_maximum_support_matches_oracle(precision):
    """J_w = 64: rho_max ~45 pixels, 12 pieces of 4 pixels per visibility."""
    geo = oracle_geo(128)
    rng = np.random.default_rng(91)
    n = 20
    r = 40.0 * np.sqrt(rng.random(n))
    t = rng.uniform(0, 2 * np.pi, n)
    wm = 29.5 / geo.c_support
    w = np.concatenate([np.linspace(-wm, wm, n // 2), -np.linspace(-wm, wm, n // 2)])
    uvw = np.column_stack([r * np.cos(t), r * np.sin(t), w])
    op = O.make_plan(uvw, geo, 1, False)
    assert op.jw.max() == 64
    plan = radial_plan(uvw, geo, 1, False, precision)
    rd, cd, tol = dtypes(precision)
    x = W.point_sources(128, 20, 92)
    yr = W.random_vis(n, 93)
    assert O.rel_l2(plan.degrid(to_t(x, rd)).cpu().numpy(), O.degrid(op, x)) < tol
    assert O.rel_l2(plan.grid(to_t(yr, cd)).cpu().numpy(), O.grid(op, yr)) < tol
    assert plan.stats()[0] == 0


def test_radial_mwa_snapshot_at_full_size():
    """The bench workload (2048^2, 1.95M visibilities, 8 stacks, fold on): 300
    sampled visibilities against the oracle, the whole degrid against the
    quadrature path, the full-size dot test, no unconverged pieces."""
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    geo = O.geometry_from(wl, tol_rel=1e-12, tol_abs=1e-12)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    plan = radial_plan(uvw, geo, wl.n_stacks, wl.conj_fold, "f32")
    y = plan.degrid(to_t(x, torch.float32)).cpu().numpy().astype(np.complex128)
    op = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    sel = W.subsample(len(uvw), 300, 1)
    assert O.rel_l2(y[sel], O.degrid(op, x, subset=sel)) < TOL32
    assert plan.stats()[0] == 0
    quad = gpu_plan(uvw, geo, wl.n_stacks, wl.conj_fold, "f32")
    yq = quad.degrid(to_t(x, torch.float32)).cpu().numpy().astype(np.complex128)
    assert O.rel_l2(y, yq) < TOL32
    xr = to_t(W.random_image(wl.image_n, 5), torch.float32)
    yv = to_t(W.random_vis(len(uvw), 6), torch.complex64)
    lhs = torch.real(torch.vdot(yv.to(torch.complex128), plan.degrid(xr).to(torch.complex128))).item()
    rhs = torch.sum(xr.double() * plan.grid(yv).double()).item()
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_radial_series_storage_limit():
    """FP64, window alpha = 1.5 (pieces of 2.7 pixels) and J_w = 256: the
    per-warp series storage would exceed a thread block's shared memory, so
    the plan is refused with PHI_ERR_SUPPORT instead of launching."""
    geo = O.Geometry(128, 2.0, math.radians(20.0), 4.0, alpha=1.5)
    wm = 125.5 / geo.c_support
    uvw = np.array([[10.0, 5.0, -wm], [3.0, -7.0, wm]])
    with pytest.raises(phi.PhiError) as e:
        phi.Plan(torch.from_numpy(uvw), image_n=128, fov_rad=geo.fov, n_stacks=1,
                 alpha=1.5, precision="f64", max_support=256, kernel_mode="radial")
    assert e.value.status == phi.PHI_ERR_SUPPORT
