"""Pre-sampled 1-D w-planes with bilinear interpolation (Sec. 5.1.1) on the
GPU against the oracle's own table path: same sample grid (spacing from
the same error-bound rule), independent quadrature and interpolation.
Tolerances as for the quadrature path: 1e-5 (FP32) and 1e-10 (FP64)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W

pytestmark = pytest.mark.gpu

TABLE_TOL = 1e-3


@pytest.fixture(scope="module")
def case():
    geo = O.Geometry(128, 2.0, math.radians(20.0), 4.0, tol_rel=1e-13, tol_abs=1e-13)
    uvw = W.uvw_disk(1200, 60.0, 40.0, 51)
    h = geo.Npad / 2 * geo.du
    uvw[:3, 0] = [h - 0.3 * geo.du, -h + 0.2 * geo.du, 1.05 * h]
    op = O.make_plan(uvw, geo, 3, True)
    tab = O.make_table(op, TABLE_TOL)
    x = W.point_sources(128, 20, 51)
    yr = W.random_vis(len(uvw), 52)
    return dict(geo=geo, uvw=uvw, op=op, tab=tab, x=x, yr=yr,
                y_ref=O.degrid_table(op, x, tab), x_ref=O.grid_table(op, yr, tab))


def plan_for(c, precision, staging=0):
    tol = 1e-12 if precision == "f64" else 1e-6
    return phi.Plan(torch.from_numpy(c["uvw"]), image_n=128, fov_rad=c["geo"].fov, n_stacks=3,
                    conj_fold=1, precision=precision, quad_rel_tol=tol, quad_abs_tol=tol,
                    kernel_mode="table", table_tol=TABLE_TOL, grid_staging=staging)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_table_geometry_matches_oracle(case, precision):
    info = plan_for(case, precision).info()
    tab = case["tab"]
    assert info["kernel_mode"] == phi.PHI_KERNEL_TABLE
    assert info["table_n_rho"] == tab.nr and info["table_n_w"] == tab.nw
    assert abs(info["table_h_rho"] - tab.hr) < 1e-15 and abs(info["table_h_w"] - tab.hw) < 1e-15


@pytest.mark.parametrize("staging", [0, 1, 2])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_table_degrid_and_grid_match_oracle(case, precision, staging):
    plan = plan_for(case, precision, staging)
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    tol = 1e-10 if precision == "f64" else 1e-5
    y = plan.degrid(torch.from_numpy(case["x"]).to("cuda", rd)).cpu().numpy()
    assert O.rel_l2(y, case["y_ref"]) < tol
    x = plan.grid(torch.from_numpy(case["yr"]).to("cuda", cd)).cpu().numpy()
    assert O.rel_l2(x, case["x_ref"]) < tol


def test_table_adjoint_and_closeness_to_quadrature(case):
    plan = plan_for(case, "f32")
    quad = phi.Plan(torch.from_numpy(case["uvw"]), image_n=128, fov_rad=case["geo"].fov,
                    n_stacks=3, conj_fold=1)
    x = torch.from_numpy(W.random_image(128, 5)).cuda().float()
    y = torch.from_numpy(W.random_vis(len(case["uvw"]), 6)).cuda().to(torch.complex64)
    lhs = torch.real(torch.vdot(y.to(torch.complex128), plan.degrid(x).to(torch.complex128))).item()
    rhs = torch.sum(x.double() * plan.grid(y).double()).item()
    assert abs(lhs - rhs) <= 2e-5 * abs(lhs)
    xs = torch.from_numpy(case["x"]).cuda().float()
    yq = quad.degrid(xs)
    yt = plan.degrid(xs)
    assert (torch.linalg.vector_norm(yt - yq) / torch.linalg.vector_norm(yq)).item() < 2e-3


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_table_on_grid_points_matches_oracle(precision):
    """Visibilities exactly on grid points (and a hair off them): their
    central taps sit at table position s ~ 0, the first interval's left end."""
    geo = O.Geometry(128, 2.0, math.radians(20.0), 4.0, tol_rel=1e-13, tol_abs=1e-13)
    uvw = W.uvw_disk(600, 60.0, 40.0, 71)
    k = np.round(uvw[:300, :2] / geo.du)
    uvw[:200, :2] = k[:200] * geo.du
    uvw[200:300, :2] = (k[200:300] + 1e-4) * geo.du
    op = O.make_plan(uvw, geo, 3, True)
    tab = O.make_table(op, TABLE_TOL)
    x = W.point_sources(128, 20, 72)
    yr = W.random_vis(len(uvw), 73)
    tol = 1e-12 if precision == "f64" else 1e-6
    plan = phi.Plan(torch.from_numpy(uvw), image_n=128, fov_rad=geo.fov, n_stacks=3,
                    conj_fold=1, precision=precision, quad_rel_tol=tol, quad_abs_tol=tol,
                    kernel_mode="table", table_tol=TABLE_TOL)
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    ptol = 1e-10 if precision == "f64" else 1e-5
    y = plan.degrid(torch.from_numpy(x).to("cuda", rd)).cpu().numpy()
    y_ref = O.degrid_table(op, x, tab)
    assert O.rel_l2(y, y_ref) < ptol
    assert O.rel_l2(y[:300], y_ref[:300]) < ptol
    xg = plan.grid(torch.from_numpy(yr).to("cuda", cd)).cpu().numpy()
    assert O.rel_l2(xg, O.grid_table(op, yr, tab)) < ptol


def test_table_close_to_quadrature_at_full_size():
    """The bench workload (2048^2 image, 1.95M visibilities, 8 stacks, fold on)
    at table_tol 1e-4: bilinear interpolation bounds each kernel sample's
    error by table_tol times the kernel's scale, so the visibilities differ
    from the quadrature path by less than table_tol, in L2 and per
    visibility relative to the largest."""
    wl = W.mwa_snapshot()
    uvw = torch.from_numpy(W.uvw_for(wl))
    geo = O.geometry_from(wl)
    common = dict(image_n=wl.image_n, fov_rad=geo.fov, n_stacks=wl.n_stacks,
                  conj_fold=int(wl.conj_fold))
    x = torch.from_numpy(W.point_sources(wl.image_n, wl.n_sources, wl.seed)).cuda().float()
    ys = {}
    for mode, staging in (("quadrature", 0), ("table", 0), ("table", 2)):
        p = phi.Plan(uvw, kernel_mode=mode, table_tol=1e-4, grid_staging=staging, **common)
        ys[(mode, staging)] = p.degrid(x).to(torch.complex128)
        p.close()
    # the w-row-staged kernel: the same taps, order and arithmetic
    assert torch.equal(ys[("table", 2)], ys[("table", 0)])
    ys = {"table": ys[("table", 0)], "quadrature": ys[("quadrature", 0)]}
    d = ys["table"] - ys["quadrature"]
    scale = torch.abs(ys["quadrature"]).max()
    assert (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(ys["quadrature"])).item() < 1e-4
    assert (torch.abs(d).max() / scale).item() < 1e-4


def test_table_at_maximum_support_matches_oracle():
    """J_w = 64 (the default cap), radii up to ~45 pixels: the far end of the
    planes and the last interval.  FP32 against the oracle's table path at the
    same sample points (table_tol 1e-2 keeps the oracle's table small; the
    oracle samples at tol 1e-9, below the FP32 gate)."""
    geo = O.Geometry(128, 2.0, math.radians(20.0), 4.0, tol_rel=1e-9, tol_abs=1e-9)
    rng = np.random.default_rng(91)
    n = 20
    r = 40.0 * np.sqrt(rng.random(n))
    t = rng.uniform(0, 2 * np.pi, n)
    wm = 29.5 / geo.c_support
    w = np.concatenate([np.linspace(-wm, wm, n // 2), -np.linspace(-wm, wm, n // 2)])
    uvw = np.column_stack([r * np.cos(t), r * np.sin(t), w])
    op = O.make_plan(uvw, geo, 1, False)
    assert op.jw.max() == 64
    tab = O.make_table(op, 1e-2)
    plan = phi.Plan(torch.from_numpy(uvw), image_n=128, fov_rad=geo.fov, n_stacks=1,
                    kernel_mode="table", table_tol=1e-2)
    info = plan.info()
    assert info["jw"] == [64] and info["table_n_rho"] == tab.nr and info["table_n_w"] == tab.nw
    x = W.point_sources(128, 20, 92)
    yr = W.random_vis(n, 93)
    y = plan.degrid(torch.from_numpy(x).cuda().float()).cpu().numpy()
    assert O.rel_l2(y, O.degrid_table(op, x, tab)) < 1e-5
    xg = plan.grid(torch.from_numpy(yr).cuda().to(torch.complex64)).cpu().numpy()
    assert O.rel_l2(xg, O.grid_table(op, yr, tab)) < 1e-5


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_row_staging_equals_the_unstaged_kernel(case, precision):
    """grid_staging 2 (one w-row of the table staged in shared memory for all
    visibilities on it) evaluates the same taps in the same order and
    arithmetic as the unstaged kernel: degrid is bitwise equal; grid differs
    only by the order of the FP atomics."""
    p0, p2 = plan_for(case, precision, 0), plan_for(case, precision, 2)
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    x = torch.from_numpy(case["x"]).to("cuda", rd)
    assert torch.equal(p0.degrid(x), p2.degrid(x))
    y = torch.from_numpy(case["yr"]).to("cuda", cd)
    g0, g2 = p0.grid(y), p2.grid(y)
    assert (torch.linalg.vector_norm(g2 - g0) / torch.linalg.vector_norm(g0)).item() < (
        1e-12 if precision == "f64" else 1e-6)
    assert p2.stats()[1] == p0.stats()[1]
