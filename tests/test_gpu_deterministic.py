"""Deterministic gridding (plan field grid_deterministic = 1): every gridding
contribution is rounded to a 64-bit fixed-point integer and added with
integer atomics, so phi_grid returns the same bits on every call.

Checked on the GPU: the oracle's gates (1e-5 FP32, 1e-10 FP64) for the
quadrature and radial modes, the table path (against the oracle's own table
path) and the DDE convolution; identical bits on repeated calls and across
plans; agreement with the FP-atomic gridder; degridding untouched by the
flag; the exponent chosen from the data (visibilities scaled by 1e-20 and
1e20, 1e-150 and 1e150 in FP64, grid to the scaled image); a non-finite
visibility gives a NaN image rather than wrapped integers."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_parity import TOL32, TOL64, gpu_plan, oracle_geo, to_t

pytestmark = pytest.mark.gpu

TABLE_TOL = 1e-3


def ctype(precision):
    return torch.complex128 if precision == "f64" else torch.complex64


def rtype(precision):
    return torch.float64 if precision == "f64" else torch.float32


def gate(precision):
    return TOL64 if precision == "f64" else TOL32


@pytest.fixture(scope="module")
def case():
    geo = oracle_geo(128)
    uvw = W.uvw_disk(1500, 60.0, 40.0, 91)
    h = geo.Npad / 2 * geo.du
    uvw[:3, 0] = [h - 0.3 * geo.du, -h + 0.2 * geo.du, 1.05 * h]   # edge wrap, one dropped
    wts = np.linspace(0.25, 2.0, len(uvw))
    op = O.make_plan(uvw, geo, 3, True, weights=wts)
    yr = W.random_vis(len(uvw), 92)
    return dict(geo=geo, uvw=uvw, w=wts, op=op, yr=yr, x_ref=O.grid(op, yr))


@pytest.mark.parametrize("mode", ["quadrature", "radial"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_deterministic_grid_matches_oracle_bit_for_bit_repeatable(case, precision, mode):
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"], kernel_mode=mode,
                    grid_deterministic=1)
    y = to_t(case["yr"], ctype(precision))
    x1 = plan.grid(y)
    assert O.rel_l2(x1.cpu().numpy(), case["x_ref"]) < gate(precision)
    x2 = plan.grid(y)
    assert torch.equal(x1, x2)
    other = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"], kernel_mode=mode,
                     grid_deterministic=1)
    assert torch.equal(other.grid(y), x1)
    # the FP-atomic gridder computes the same operator
    plain = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"], kernel_mode=mode)
    xp = plain.grid(y)
    assert O.rel_l2(x1.cpu().numpy(), xp.cpu().numpy()) < gate(precision)
    bad, taps = plan.stats()
    assert bad == 0 and taps > 0


@pytest.mark.parametrize("staging", [0, 2])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_deterministic_table_grid(case, precision, staging):
    """Table path (Sec. 5.1.1) against the oracle's table path."""
    op = O.make_plan(case["uvw"], case["geo"], 3, True)
    tab = O.make_table(op, TABLE_TOL)
    x_ref = O.grid_table(op, case["yr"], tab)
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, precision, kernel_mode="table",
                    table_tol=TABLE_TOL, grid_staging=staging, grid_deterministic=1)
    y = to_t(case["yr"], ctype(precision))
    x1 = plan.grid(y)
    assert O.rel_l2(x1.cpu().numpy(), x_ref) < gate(precision)
    assert torch.equal(plan.grid(y), x1)


@pytest.mark.parametrize("mode", ["quadrature", "radial"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_deterministic_dde_grid(precision, mode):
    """DDE convolution (Sec. 5.2): the term bound includes the DDE kernels'
    sums; both the whole-box (quadrature) and the banded (radial) kernel."""
    geo = oracle_geo(128)
    uvw = W.uvw_disk(600, 60.0, 40.0, 93)
    wts = np.linspace(0.5, 1.5, len(uvw))
    op = O.make_plan(uvw, geo, 3, False, weights=wts)
    a, b = W.dde_kernels(len(uvw), 5, 94)
    yr = W.random_vis(len(uvw), 95)
    x_ref = O.grid_dde(op, yr, a, b)
    plan = gpu_plan(uvw, geo, 3, False, precision, wts, kernel_mode=mode, grid_deterministic=1)
    y = to_t(yr, ctype(precision))
    x1 = plan.grid_dde(y, a, b)
    assert O.rel_l2(x1.cpu().numpy(), x_ref) < gate(precision)
    assert torch.equal(plan.grid_dde(y, a, b), x1)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_deterministic_grid_one_stack_per_group(case, precision):
    """max_grid_mib = 1 leaves room for one grid and its fixed-point sums at a
    time: every stack group sets its own exponent and converts its own sums,
    and the result still matches the oracle and repeats bit for bit."""
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"], max_grid_mib=1,
                    grid_deterministic=1)
    assert plan.info()["group"] == 1
    y = to_t(case["yr"], ctype(precision))
    x1 = plan.grid(y)
    assert O.rel_l2(x1.cpu().numpy(), case["x_ref"]) < gate(precision)
    assert torch.equal(plan.grid(y), x1)


def test_degrid_is_unchanged_by_the_flag(case):
    x = to_t(W.point_sources(128, 20, 96), torch.float32)
    det = gpu_plan(case["uvw"], case["geo"], 3, True, "f32", case["w"], grid_deterministic=1)
    plain = gpu_plan(case["uvw"], case["geo"], 3, True, "f32", case["w"])
    assert torch.equal(det.degrid(x), plain.degrid(x))


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_deterministic_adjoint_dot_product(case, precision):
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"],
                    grid_deterministic=1)
    x = to_t(W.random_image(128, 97), rtype(precision))
    y = to_t(W.random_vis(len(case["uvw"]), 98), ctype(precision))
    lhs = torch.real(torch.vdot(y.to(torch.complex128), plan.degrid(x).to(torch.complex128))).item()
    rhs = torch.sum(x.double() * plan.grid(y).double()).item()
    assert abs(lhs - rhs) <= (1e-12 if precision == "f64" else 2e-5) * abs(lhs)


@pytest.mark.parametrize("precision,scale", [("f32", 1e-20), ("f32", 1e20), ("f64", 1e-150),
                                             ("f64", 1e150)])
def test_exponent_follows_the_data(case, precision, scale):
    """Linearity across 40 (FP32) and 300 (FP64) decades: the fixed-point
    exponent is chosen per call from the largest term, so scaled visibilities
    grid to the scaled image within the gate."""
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, precision, case["w"],
                    grid_deterministic=1)
    y = to_t(case["yr"], ctype(precision))
    x = plan.grid(y).double()
    xs = plan.grid(y * scale).double() / scale
    assert torch.isfinite(xs).all()
    assert (torch.linalg.norm(xs - x) / torch.linalg.norm(x)).item() < gate(precision)


def test_non_finite_visibility_gives_nan_image(case):
    plan = gpu_plan(case["uvw"], case["geo"], 3, True, "f32", case["w"], grid_deterministic=1)
    y = to_t(case["yr"], torch.complex64)
    y[7] = complex(math.inf, 0.0)
    assert torch.isnan(plan.grid(y)).all()
    # the next call with finite data is unaffected
    y[7] = 0.5
    assert torch.isfinite(plan.grid(y)).all()


def test_deterministic_plan_holds_its_fixed_point_grids(case):
    det = gpu_plan(case["uvw"], case["geo"], 3, True, "f32", case["w"], grid_deterministic=1)
    plain = gpu_plan(case["uvw"], case["geo"], 3, True, "f32", case["w"])
    i_det, i_plain = det.info(), plain.info()
    npad = i_det["npad"]
    assert i_det["device_bytes"] - i_plain["device_bytes"] >= 16 * npad * npad * i_det["group"]
