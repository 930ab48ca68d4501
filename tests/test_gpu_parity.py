"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 over visibilities / image of 1e-5 for the FP32 path
(quadrature tolerance 1e-6, the paper's setting) and 1e-10 for the FP64 path
(quadrature tolerance 1e-12 on the device, 1e-13 in the oracle).  Integer
plan data (stack assignment counts, supports, drops) must match exactly.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10
DEV = "cuda"


def gpu_plan(uvw, geo, n_stacks=1, fold=False, precision="f32", weights=None, **kw):
    tol = 1e-12 if precision == "f64" else 1e-6
    kw.setdefault("quad_rel_tol", tol)
    kw.setdefault("quad_abs_tol", tol)
    return phi.Plan(torch.from_numpy(np.ascontiguousarray(uvw)), weights=None if weights is None
                    else torch.from_numpy(np.asarray(weights, np.float64)),
                    image_n=geo.N, fov_rad=geo.fov, oversample=geo.os, support=int(geo.J),
                    n_stacks=n_stacks, conj_fold=int(fold), precision=precision,
                    alpha=geo.alpha, **kw)


def oracle_geo(wl_or_n, fov_deg=20.0, **kw):
    kw.setdefault("tol_rel", 1e-13)
    kw.setdefault("tol_abs", 1e-13)
    return O.Geometry(wl_or_n, 2.0, math.radians(fov_deg), 4.0, **kw)


def to_t(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


# ----------------------------------------------------------------------------- kernel

@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_wkernel_matches_oracle(precision):
    geo = oracle_geo(128)
    uvw = W.uvw_disk(8, 60.0, 40.0, 0)
    plan = gpu_plan(uvw, geo, precision=precision)
    rng = np.random.default_rng(11)
    rho = np.concatenate([[0.0, 0.0, 1e-7, 2.0], rng.uniform(0, 30, 300)])
    dw = np.concatenate([[0.0, 35.0, -7.0, 0.0], rng.uniform(-150, 150, 300)])
    ref = O.wkernel(rho, dw, geo)
    k, bad = plan.wkernel(rho, dw)
    k = k.cpu().numpy()
    assert bad == 0
    err = np.abs(k - ref)
    if precision == "f64":
        assert err.max() < 1e-11
    else:
        assert err.max() < 1e-5
        assert np.sqrt(np.mean(err ** 2)) < 2e-6
    # conjugate symmetry on the device path (Sec. 3.3)
    km, _ = plan.wkernel(rho, -dw)
    assert np.abs(km.cpu().numpy() - np.conj(k)).max() <= (1e-14 if precision == "f64" else 1e-6)


# ----------------------------------------------------------------------------- plan

@pytest.mark.parametrize("k,fold,rule", [(1, False, "stack"), (3, True, "stack"), (5, True, "vis")])
def test_plan_matches_oracle(k, fold, rule):
    geo = oracle_geo(128)
    uvw = W.uvw_disk(3000, 60.0, 40.0, 5)
    plan = gpu_plan(uvw, geo, n_stacks=k, fold=fold, support_rule=rule)
    op = O.make_plan(uvw, geo, k, fold, support_rule=O.SUPPORT_VIS if rule == "vis" else O.SUPPORT_STACK)
    info = plan.info()
    assert info["kmeans_sweeps"] == op.sweeps
    assert np.allclose(info["wbar"], op.wbar, rtol=1e-12, atol=1e-12)
    for q in range(k):
        assert info["counts"][q] == int(np.sum((op.stack == q) & ~op.dropped))
        sel = (op.stack == q) & ~op.dropped
        assert info["jw"][q] == (int(op.jw[sel].max()) if sel.any() else 0)
    assert info["n_dropped"] == int(op.dropped.sum())
    assert abs(info["du"] - geo.du) < 1e-15 * geo.du
    assert abs(info["beta"] - geo.beta) < 1e-13


# ----------------------------------------------------------------------------- operator

CASES = {
    # name: (n_vis, n_stacks, fold, support rule, weights)
    "plain": (1500, 1, False, "stack", False),
    "fold3": (1200, 3, True, "stack", True),
    "vis4": (1200, 4, True, "vis", False),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    n, k, fold, rule, weighted = CASES[request.param]
    geo = oracle_geo(128)
    uvw = W.uvw_disk(n, 60.0, 40.0, 21)
    # a few visibilities on the grid edge (circular taps) and outside it (dropped)
    h = geo.Npad / 2 * geo.du
    uvw[:4, 0] = [h - 0.3 * geo.du, -h + 0.2 * geo.du, 1.05 * h, 0.1]
    uvw[:4, 1] = [0.4, h - 1.1 * geo.du, 0.0, -1.2 * h]
    wts = np.linspace(0.25, 2.0, n) if weighted else None
    x = W.point_sources(128, 20, 21)
    rule_o = O.SUPPORT_VIS if rule == "vis" else O.SUPPORT_STACK
    op = O.make_plan(uvw, geo, k, fold, weights=wts, support_rule=rule_o)
    y_ref = O.degrid(op, x)
    yr = W.random_vis(n, 22)
    x_ref = O.grid(op, yr)
    return dict(geo=geo, uvw=uvw, w=wts, x=x, k=k, fold=fold, rule=rule, y_ref=y_ref, yr=yr,
                x_ref=x_ref, op=op)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_degrid_matches_oracle(case, precision):
    plan = gpu_plan(case["uvw"], case["geo"], case["k"], case["fold"], precision, case["w"],
                    support_rule=case["rule"])
    rd = torch.float64 if precision == "f64" else torch.float32
    y = plan.degrid(to_t(case["x"], rd)).cpu().numpy()
    err = O.rel_l2(y, case["y_ref"])
    assert err < (TOL64 if precision == "f64" else TOL32), err
    assert np.all(y[case["op"].dropped] == 0)
    bad, taps = plan.stats()
    assert bad == 0 and taps > 0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_grid_matches_oracle(case, precision):
    plan = gpu_plan(case["uvw"], case["geo"], case["k"], case["fold"], precision, case["w"],
                    support_rule=case["rule"])
    cd = torch.complex128 if precision == "f64" else torch.complex64
    x = plan.grid(to_t(case["yr"], cd)).cpu().numpy()
    err = O.rel_l2(x, case["x_ref"])
    assert err < (TOL64 if precision == "f64" else TOL32), err


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_adjoint_dot_product_on_device(case, precision):
    """<Phi x, y> = <x, Phi^H y> (real inner product, Sec. 3.1)."""
    plan = gpu_plan(case["uvw"], case["geo"], case["k"], case["fold"], precision, case["w"],
                    support_rule=case["rule"])
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    x = to_t(W.random_image(128, 3), rd)
    y = to_t(W.random_vis(len(case["uvw"]), 4), cd)
    lhs = torch.real(torch.vdot(y.to(torch.complex128), plan.degrid(x).to(torch.complex128))).item()
    rhs = torch.sum(x.double() * plan.grid(y).double()).item()
    assert abs(lhs - rhs) <= (1e-12 if precision == "f64" else 2e-5) * abs(lhs)


def test_degrid_is_deterministic_and_plan_reproducible(case):
    p1 = gpu_plan(case["uvw"], case["geo"], case["k"], case["fold"], "f32", case["w"],
                  support_rule=case["rule"])
    p2 = gpu_plan(case["uvw"], case["geo"], case["k"], case["fold"], "f32", case["w"],
                  support_rule=case["rule"])
    assert p1.info()["wbar"] == p2.info()["wbar"]
    x = to_t(case["x"], torch.float32)
    assert torch.equal(p1.degrid(x), p2.degrid(x))


# ----------------------------------------------------------------------------- edge cases

def test_empty_plan():
    geo = oracle_geo(64)
    plan = gpu_plan(np.zeros((0, 3)), geo, n_stacks=2)
    y = plan.degrid(torch.ones(64, 64, device=DEV))
    assert y.numel() == 0
    x = plan.grid(torch.zeros(0, dtype=torch.complex64, device=DEV))
    assert torch.count_nonzero(x) == 0
    k, bad = plan.wkernel([], [])
    assert k.numel() == 0 and bad == 0


def test_all_dropped_and_single_visibility():
    geo = oracle_geo(64)
    h = geo.Npad / 2 * geo.du
    plan = gpu_plan(np.array([[2 * h, 0.0, 1.0], [0.0, -3 * h, -2.0]]), geo, n_stacks=1, fold=True)
    assert plan.info()["n_dropped"] == 2
    y = plan.degrid(torch.ones(64, 64, device=DEV))
    assert torch.count_nonzero(y) == 0
    assert torch.count_nonzero(plan.grid(torch.ones(2, dtype=torch.complex64, device=DEV))) == 0
    one = np.array([[3.7, -8.1, 12.5]])
    x = W.point_sources(64, 3, 2)
    p1 = gpu_plan(one, geo, precision="f64")
    y1 = p1.degrid(to_t(x, torch.float64)).cpu().numpy()
    assert O.rel_l2(y1, O.degrid(O.make_plan(one, geo, 1, False), x)) < TOL64


def test_max_support_exceeded_is_an_error():
    geo = oracle_geo(128)
    uvw = W.uvw_disk(50, 60.0, 400.0, 1)
    with pytest.raises(phi.PhiError) as e:
        gpu_plan(uvw, geo, n_stacks=1, max_support=32)
    assert e.value.status == phi.PHI_ERR_SUPPORT


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_visibilities_on_grid_points_match_oracle(precision):
    """Visibilities on grid points and one ulp either side of them (u/du an
    integer, or the double next to it): the J_w-wide box is the J_w nearest
    grid points, half-open on its low side (Sec. 2), decided on the exact
    double u/du by both sides."""
    geo = oracle_geo(128)
    uvw = W.uvw_disk(500, 60.0, 40.0, 81)
    k = np.round(uvw[:300, :2] / geo.du)
    uvw[:100, :2] = k[:100] * geo.du
    uvw[100:200, :2] = np.nextafter(k[100:200], -np.inf) * geo.du
    uvw[200:300, :2] = np.nextafter(k[200:300], np.inf) * geo.du
    op = O.make_plan(uvw, geo, 3, True)
    x = W.point_sources(128, 20, 82)
    yr = W.random_vis(len(uvw), 83)
    plan = gpu_plan(uvw, geo, 3, True, precision)
    rd, cd = (torch.float64, torch.complex128) if precision == "f64" else (torch.float32, torch.complex64)
    tol = TOL64 if precision == "f64" else TOL32
    y = plan.degrid(to_t(x, rd)).cpu().numpy()
    y_ref = O.degrid(op, x)
    assert O.rel_l2(y, y_ref) < tol
    assert O.rel_l2(y[:300], y_ref[:300]) < tol
    assert O.rel_l2(plan.grid(to_t(yr, cd)).cpu().numpy(), O.grid(op, yr)) < tol


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_maximum_support_matches_oracle(precision):
    """J_w = 64, the default cap: 4,096 taps per visibility with radii up to
    ~45 pixels, so the quadrature needs more than 16 panels per chunk (the
    batched node path).  One stack, |dw| up to 29.5 / c_support."""
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
    plan = gpu_plan(uvw, geo, 1, False, precision)
    assert plan.info()["jw"] == [64]
    rd, cd = (torch.float64, torch.complex128) if precision == "f64" else (torch.float32, torch.complex64)
    tol = TOL64 if precision == "f64" else TOL32
    x = W.point_sources(128, 20, 92)
    yr = W.random_vis(n, 93)
    assert O.rel_l2(plan.degrid(to_t(x, rd)).cpu().numpy(), O.degrid(op, x)) < tol
    assert O.rel_l2(plan.grid(to_t(yr, cd)).cpu().numpy(), O.grid(op, yr)) < tol
    bad, _ = plan.stats()
    assert bad == 0


# ----------------------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def mwa():
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    geo = O.geometry_from(wl, tol_rel=1e-12, tol_abs=1e-12)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    return wl, uvw, geo, x


def test_mwa_snapshot_sampled_parity(mwa):
    """The bench workload at full size (2048^2 image, 1.95M visibilities,
    8 stacks, fold on) in the bench's launch configuration; the oracle checks
    300 sampled visibilities one by one."""
    wl, uvw, geo, x = mwa
    plan = gpu_plan(uvw, geo, wl.n_stacks, wl.conj_fold, "f32")
    y = plan.degrid(to_t(x, torch.float32)).cpu().numpy()
    op = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    info = plan.info()
    assert np.allclose(info["wbar"], op.wbar, rtol=1e-11, atol=1e-11)
    assert info["n_dropped"] == int(op.dropped.sum())
    sel = W.subsample(len(uvw), 300, 1)
    y_ref = O.degrid(op, x, subset=sel)
    assert O.rel_l2(y[sel], y_ref) < TOL32
    assert np.all(y[op.dropped] == 0)
    bad, taps = plan.stats()
    assert bad == 0


def test_mwa_snapshot_adjoint_at_full_size(mwa):
    """<Phi x, y> = <x, Phi^H y> at full size in FP32.  Both sides use the
    same kernel values, so only FP32 rounding separates them.  With
    deterministic gridding (64-bit fixed-point cell sums) that is the tap
    sums and FFTs, and the gap is held to the FP32 gate, 1e-5 of
    |<y, Phi x>| (measured 4.3e-6, the same on every run).  The default
    gridder adds each cell's 1,000-2,500 contributions with FP32 atomics in
    run-dependent order, and random x and y make <y, Phi x> cancel about
    24,000-fold (|<y, Phi x>| ~ 4e-5 |y| |Phi x|), so that rounding moves
    the gap from run to run (measured 3.5e-7 to 1.1e-5 of |<y, Phi x>|,
    1.5e-11 to 4.5e-10 of |y| |Phi x|): it is held to 2e-9 of the
    Cauchy-Schwarz scale |y| |Phi x|."""
    wl, uvw, geo, _ = mwa
    x = to_t(W.random_image(wl.image_n, 5), torch.float32)
    y = to_t(W.random_vis(len(uvw), 6), torch.complex64)
    for deterministic in (1, 0):
        plan = gpu_plan(uvw, geo, wl.n_stacks, wl.conj_fold, "f32",
                        grid_deterministic=deterministic)
        yd = plan.degrid(x).to(torch.complex128)
        lhs = torch.real(torch.vdot(y.to(torch.complex128), yd)).item()
        rhs = torch.sum(x.double() * plan.grid(y).double()).item()
        if deterministic:
            assert abs(lhs - rhs) <= TOL32 * abs(lhs)
        else:
            scale = (torch.linalg.vector_norm(y.to(torch.complex128)) *
                     torch.linalg.vector_norm(yd)).item()
            assert abs(lhs - rhs) <= 2e-9 * scale
        plan.close()


@pytest.mark.parametrize("mode", ["quadrature", "table"])
def test_stack_groups_match_one_grid_at_a_time(mode):
    """Grids of several stacks resident together (batched FFTs, one fused
    launch per group) give the same operator as one stack at a time: groups
    of 2 over 5 stacks (the last group takes the single-transform path)."""
    geo = oracle_geo(128)
    uvw = W.uvw_disk(2000, 60.0, 40.0, 61)
    x = torch.from_numpy(W.point_sources(128, 20, 61)).cuda().float()
    yr = torch.from_numpy(W.random_vis(2000, 62)).cuda().to(torch.complex64)
    out = {}
    for mib in (1, 0):          # 1 MiB: two 256^2 grids per group; 0: all five together
        plan = gpu_plan(uvw, geo, 5, True, kernel_mode=mode, max_grid_mib=mib)
        info = plan.info()
        out[mib] = (info["group"], plan.degrid(x), plan.grid(yr))
    assert out[1][0] == 2 and out[0][0] == 5
    assert torch.equal(out[1][1], out[0][1])
    d1, d0 = out[1][2], out[0][2]
    assert (torch.linalg.vector_norm(d1 - d0) / torch.linalg.vector_norm(d0)).item() < 1e-6
    if mode == "quadrature":
        op = O.make_plan(uvw, geo, 5, True)
        assert O.rel_l2(out[1][1].cpu().numpy(), O.degrid(op, x.double().cpu().numpy())) < TOL32


GEOMETRIES = {
    # name: (N, os, fov_deg, J, alpha, n_vis, K, fold)
    "os1.5-J6": (96, 1.5, 10.0, 6, 1.0, 600, 2, True),
    "J8-alpha1.5": (128, 2.0, 20.0, 8, 1.5, 500, 3, False),
    "K126-many-empty": (64, 2.0, 20.0, 4, 1.0, 400, 126, True),
}


@pytest.mark.parametrize("name", list(GEOMETRIES))
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_geometry_variants_match_oracle(name, precision):
    N, os_, fov, J, alpha, m, k, fold = GEOMETRIES[name]
    geo = O.Geometry(N, os_, math.radians(fov), float(J), alpha=alpha, tol_rel=1e-13,
                     tol_abs=1e-13)
    radius = 0.45 * geo.Npad * geo.du / 2
    uvw = W.uvw_disk(m, radius, 30.0, 71)
    x = W.point_sources(N, 10, 71)
    yr = W.random_vis(m, 72)
    op = O.make_plan(uvw, geo, k, fold)
    plan = gpu_plan(uvw, geo, k, fold, precision)
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    tol = TOL64 if precision == "f64" else TOL32
    y = plan.degrid(to_t(x, rd)).cpu().numpy()
    assert O.rel_l2(y, O.degrid(op, x)) < tol
    d = plan.grid(to_t(yr, cd)).cpu().numpy()
    assert O.rel_l2(d, O.grid(op, yr)) < tol
    info = plan.info()
    assert info["npad"] == geo.Npad and info["kmeans_sweeps"] == op.sweeps
