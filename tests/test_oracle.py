"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the paper passage the checked function follows and what pins
it: a closed form, a library routine, an independent quadrature, brute force
on a tiny input, or an identity the mathematics fixes.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_geo(**kw):
    return O.Geometry(128, 2.0, math.radians(20.0), 4.0, **kw)


# ---------------------------------------------------------------- quadrature rule

def test_gauss_kronrod_rule_exactness():
    """The adaptive quadrature (Sec. 3.1, Sec. 4) uses a Gauss-Kronrod 7/15
    pair.  Pin: the 15-point rule integrates x^k exactly up to k = 22 and not
    at 24; the 7-point subset up to 13 and not at 14; nodes inside (-1, 1)."""
    x, wk, wg = O.gauss_kronrod_15()
    for k in range(0, 23, 2):
        assert abs((wk * x ** k).sum() - 2.0 / (k + 1)) < 1e-14
    for k in range(0, 14, 2):
        assert abs((wg * x ** k).sum() - 2.0 / (k + 1)) < 1e-14
    assert abs((wk * x ** 24).sum() - 2.0 / 25) > 1e-10
    assert abs((wg * x ** 14).sum() - 2.0 / 15) > 1e-6
    assert np.all(np.abs(x) < 1) and np.all(wk > 0)
    assert np.count_nonzero(wg) == 7
    xg, _ = np.polynomial.legendre.leggauss(7)
    assert np.allclose(np.sort(x[wg != 0]), np.sort(xg), atol=1e-15)


# ---------------------------------------------------------------- special functions

@pytest.mark.parametrize("x", [0.0, 0.3, 2.9, 3.1, 7.7, 25.0, 141.0])
def test_bessel_against_scipy(x):
    L = O.lib()
    assert abs(L.orc_bessel_j0(x) - sp.j0(x)) < 1e-14
    assert abs(L.orc_bessel_j1(x) - sp.j1(x)) < 1e-14
    if x < 50:
        assert abs(L.orc_bessel_i0(x) / sp.i0(x) - 1) < 1e-13
        assert abs(L.orc_bessel_i1(x) - sp.i1(x)) <= 1e-13 * max(1.0, sp.i1(x))


def test_kaiser_bessel_values():
    """KB kernel: k(0) = 1, k(J/2) = 1/I0(beta), zero outside; Beatty beta."""
    beta = O.beatty_beta(4, 2.0)
    assert abs(beta - math.pi * math.sqrt(8.2)) < 1e-14
    assert abs(beta - 8.99615) < 1e-5
    assert O.kb(0.0, 4, beta) == 1.0
    assert abs(O.kb(2.0, 4, beta) - 1.0 / sp.i0(beta)) < 1e-16
    assert O.kb(2.0001, 4, beta) == 0.0
    r = 1.3
    assert abs(O.kb(r, 4, beta) - sp.i0(beta * math.sqrt(1 - (r / 2) ** 2)) / sp.i0(beta)) < 1e-15


@pytest.mark.parametrize("r", [0.0, 0.1, 0.25, 0.5, 0.7, 0.716, 0.9, 1.4])
def test_taper_closed_form_against_numerical_hankel(r):
    """g (the radial anti-aliasing filter of Eq. S~_k and Eq.
    analytic_convolution_hankel) is the 2-D Fourier transform of the radial
    KB kernel.  Pin: the closed form agrees with scipy's adaptive quadrature
    of 2 pi int k(rho) J0(2 pi rho r) rho drho, including across the point
    where the Bessel argument turns imaginary (r ~ 0.716 at J=4, beta=9)."""
    beta = O.beatty_beta(4, 2.0)
    f = lambda rho: sp.i0(beta * math.sqrt(max(0.0, 1 - (rho / 2) ** 2))) / sp.i0(beta) \
        * sp.j0(2 * math.pi * rho * r) * rho
    num, _ = si.quad(f, 0.0, 2.0, epsabs=1e-14, epsrel=1e-14, limit=200)
    assert abs(O.taper(r, 4, beta) - 2 * math.pi * num) < 1e-11


def test_taper_of_flat_kernel_is_disk_transform():
    """beta = 0 makes k the indicator of the disk |rho| <= a; its transform is
    the textbook a J1(2 pi a r) / r."""
    a = 2.0
    for r in (0.05, 0.3, 0.8):
        assert abs(O.taper(r, 4, 0.0) - a * sp.j1(2 * math.pi * a * r) / r) < 1e-13


# ---------------------------------------------------------------- radial kernel

KERNEL_POINTS = [(0.0, 0.0, 0.0), (0.4, -1.1, 0.0), (1.7, 0.6, 7.5), (-2.9, 3.3, -23.0),
                 (5.0, -4.0, 40.0), (0.2, 0.1, 120.0)]


@pytest.mark.parametrize("ru,rv,dw", KERNEL_POINTS)
def test_radial_reduction_against_2d_disk_quadrature(ru, rv, dw):
    """Eq. analytic_convolution_hankel reduces the 2-D transform of g(r) times
    the w-chirp over the window disk to a 1-D integral with J0 by radial
    symmetry (Sec. 5.1.1).  Pin: a 2-D Cartesian Gauss-Legendre quadrature
    over the disk with no Bessel function."""
    geo = tiny_geo()
    k1 = O.wkernel(math.hypot(ru, rv), dw, geo)[0]
    k2 = O.wkernel_2d(ru, rv, dw, geo)[0]
    assert abs(k1 - k2) < 1e-10 * max(1.0, abs(k2))


def test_2d_quadrature_converged():
    geo = tiny_geo()
    a = O.wkernel_2d(3.3, -2.1, 31.0, geo)[0]
    b = O.wkernel_2d(3.3, -2.1, 31.0, geo, n_gl=24, n_phi=30, n_y=30)[0]
    assert abs(a - b) < 1e-12


def test_kernel_conjugate_symmetry():
    """Sec. 3.3 / Sec. 5.1.1: K(rho, -w) = conj K(rho, w) (real taper,
    real J0, conjugate chirp)."""
    geo = tiny_geo()
    rho = np.array([0.0, 0.5, 1.9, 4.4, 9.0])
    for dw in (3.0, 17.0, 55.0):
        kp = O.wkernel(rho, dw, geo)
        km = O.wkernel(rho, -dw, geo)
        assert np.max(np.abs(km - np.conj(kp))) < 1e-13


def test_w0_kernel_is_kb_convolved_with_disk_transform():
    """At w = 0 the kernel is the transform of g restricted to the window
    disk r <= R, i.e. the KB kernel convolved with R J1(2 pi R s)/s.  Pin: that
    2-D convolution computed directly from k (not from g) by polar
    Gauss-Legendre over the KB support."""
    geo = tiny_geo()
    R, a, beta = geo.R, 2.0, geo.beta
    xs, ws = np.polynomial.legendre.leggauss(80)
    s = a * (xs + 1) / 2
    wsr = ws * a / 2
    xt, wt = np.polynomial.legendre.leggauss(160)
    th = np.pi * (xt + 1)
    wth = wt * np.pi
    S, TH = np.meshgrid(s, th, indexing="ij")
    WW = np.outer(wsr, wth)
    ks = sp.i0(beta * np.sqrt(np.clip(1 - (S / a) ** 2, 0, None))) / sp.i0(beta)
    for rho in (0.0, 0.7, 1.9, 3.1, 6.2):
        d = np.hypot(rho - S * np.cos(TH), S * np.sin(TH))
        jinc = np.where(d > 1e-12, R * sp.j1(2 * np.pi * R * d) / np.maximum(d, 1e-300),
                        np.pi * R * R)
        conv = np.sum(WW * ks * jinc * S)
        k = O.wkernel(rho, 0.0, geo)[0]
        assert abs(k.imag) < 1e-15
        assert abs(k.real - conv) < 1e-10, (rho, k, conv)


def test_w0_kernel_approaches_kb_for_wide_window():
    """As the window grows the w = 0 kernel tends to the plain KB kernel."""
    geo = O.Geometry(128, 2.0, math.radians(1.0), 4.0, alpha=16.0, max_panels=20000)
    assert geo.l_win < 0.5
    rho = np.array([0.0, 0.8, 1.6, 2.5])
    k = O.wkernel(rho, 0.0, geo)
    err = np.abs(k - O.kb(rho, 4, geo.beta))
    assert err.max() < 0.02
    geo2 = O.Geometry(128, 2.0, math.radians(1.0), 4.0, alpha=2.0)
    assert np.abs(O.wkernel(rho, 0.0, geo2) - O.kb(rho, 4, geo.beta)).max() > 3 * err.max()


def test_kernel_tolerance_is_met():
    """The adaptive quadrature meets the paper's 1e-6 tolerance (Sec. 4):
    the tol 1e-6 result is within 1e-6 max(1,|K|) of the tol 1e-13 result."""
    geo = tiny_geo()
    rng = np.random.default_rng(1)
    rho = rng.uniform(0, 18, 200)
    dw = rng.uniform(-60, 60, 200)
    lo = O.wkernel(rho, dw, geo, 1e-6, 1e-6)
    hi = O.wkernel(rho, dw, geo, 1e-13, 1e-13)
    assert np.all(np.abs(lo - hi) <= 1e-6 * np.maximum(1, np.abs(hi)))


# ---------------------------------------------------------------- direct equation

def test_direct_equation_point_sources():
    """Eq. meas_eq: a source at the phase centre gives y = flux for every
    baseline; a source at (l0, m0) gives flux/n0 e^{-2 pi i (u l0 + v m0 +
    w (n0 - 1))}."""
    geo = tiny_geo()
    uvw = W.uvw_disk(50, 60.0, 40.0, 3)
    x = np.zeros((128, 128))
    x[64, 64] = 0.7
    assert np.abs(O.direct(x, uvw, geo) - 0.7).max() < 1e-15
    x[:] = 0
    x[20, 100] = 1.3
    l0, m0 = (100 - 64) * geo.dl, (20 - 64) * geo.dl
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    ref = 1.3 / n0 * np.exp(-2j * np.pi * (uvw[:, 0] * l0 + uvw[:, 1] * m0 + uvw[:, 2] * (n0 - 1)))
    assert np.abs(O.direct(x, uvw, geo) - ref).max() < 1e-12


def test_direct_equation_conjugate_symmetry():
    """Sec. 3.3: y*(u, v, -|w|) = y(-u, -v, |w|) for a real sky."""
    geo = tiny_geo()
    uvw = W.uvw_disk(40, 60.0, 40.0, 4)
    x = W.point_sources(128, 10, 4)
    assert np.abs(O.direct(x, -uvw, geo) - np.conj(O.direct(x, uvw, geo))).max() < 1e-12


# ---------------------------------------------------------------- grid steps

def test_pad_fft_matches_naive_dft():
    """Z then F: X(q) = sum_P X_P e^{-2 pi i q (P - Npad/2)/Npad} for
    q in [-Npad/2, Npad/2), stored at q mod Npad; naive DFT on 8 -> 16."""
    geo = O.Geometry(8, 2.0, 0.1)
    rng = np.random.default_rng(0)
    xs = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    got = O.pad_fft(xs, geo)
    P = np.arange(8) + 4
    for qv in range(-8, 8):
        for qu in range(-8, 8):
            ph = np.exp(-2j * np.pi * (np.outer(qv * (P - 8), np.ones(8)) +
                                       np.outer(np.ones(8), qu * (P - 8))) / 16)
            assert abs(got[qv % 16, qu % 16] - np.sum(xs * ph)) < 1e-12


def test_fft_adjoint_pair():
    geo = O.Geometry(8, 2.0, 0.1)
    rng = np.random.default_rng(1)
    a = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    b = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    lhs = np.vdot(b, O.pad_fft(a, geo))
    rhs = np.vdot(O.fft_adjoint_crop(b, geo), a)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


# ---------------------------------------------------------------- Algorithm 1

def brute_kmeans(w, k, max_iter=100, tol=1e-3):
    """Literal Lloyd iteration with the same reading as the oracle, written
    independently: pure Python lists, no numpy."""
    w = [float(v) for v in w]
    lo, hi = min(w), max(w)
    c = [0.5 * (lo + hi)] if k == 1 else [lo + q * (hi - lo) / (k - 1) for q in range(k)]
    eps = (hi - lo) / k if hi > lo else 1.0
    lab = [0] * len(w)
    for t in range(1, max_iter + 1):
        for p, v in enumerate(w):
            d = [(cq - v) ** 2 for cq in c]
            lab[p] = d.index(min(d))
        new = []
        for q in range(k):
            mem = [v for v, l in zip(w, lab) if l == q]
            new.append(sum(mem) / len(mem) if mem else 0.0)
        delta = sum(abs(n - o) / max(abs(o), eps) for n, o in zip(new, c)) / k
        c = new
        if delta < tol:
            return lab, c, t
    return lab, c, max_iter


@pytest.mark.parametrize("seed,k", [(0, 1), (1, 2), (2, 3), (3, 5), (4, 8)])
def test_kmeans_against_brute_force(seed, k):
    rng = np.random.default_rng(seed)
    w = np.concatenate([rng.normal(mu, 3.0, 40) for mu in rng.uniform(0, 200, 4)])
    st, c, it = O.kmeans(w, k)
    lab, c2, it2 = brute_kmeans(w, k)
    assert list(st) == lab
    assert it == it2
    assert np.allclose(c, c2, rtol=1e-13, atol=1e-12)


def test_kmeans_hand_worked_example():
    """Hand-worked Algorithm 1 (tests/golden/kmeans_hand.json)."""
    with open(os.path.join(GOLDEN, "kmeans_hand.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        st, c, it = O.kmeans(np.array(case["w"], float), case["k"], case.get("max_iter", 100),
                             case.get("tol", 1e-3))
        assert list(st) == case["stack"], case["name"]
        assert np.allclose(c, case["centres"], atol=1e-12), case["name"]
        assert it == case["sweeps"], case["name"]


def test_fold_restricts_w_to_nonnegative():
    """Sec. 3.3 / Sec. 4: after the fold every w >= 0 and the |w| range is
    unchanged (0..600 after, 1200 wide before, in the paper's data)."""
    uvw = W.uvw_disk(500, 60.0, 40.0, 5)
    f, flag = O.fold(uvw)
    assert np.all(f[:, 2] >= 0)
    assert np.array_equal(flag, uvw[:, 2] < 0)
    assert np.allclose(f[flag], -uvw[flag]) and np.allclose(f[~flag], uvw[~flag])
    assert abs(f[:, 2].max() - np.abs(uvw[:, 2]).max()) < 1e-12


def test_support_rule_values():
    geo = tiny_geo()
    lw = 0.5 / geo.du
    c = lw / (math.sqrt(1 - lw * lw) * geo.du)
    assert abs(geo.c_support - c) < 1e-15
    dw = np.array([0.0, 1e-9, 1 / c, 1 / c + 1e-9, 40.0])
    assert list(O.support(dw, geo)) == [4, 6, 6, 8, 4 + 2 * math.ceil(40 * c)]


# ---------------------------------------------------------------- operator

@pytest.fixture(scope="module")
def small_case():
    geo = tiny_geo(tol_rel=1e-10, tol_abs=1e-10)
    uvw = W.uvw_disk(120, 60.0, 40.0, 7)
    x = W.point_sources(128, 20, 7)
    return geo, uvw, x


def test_gridded_operator_against_direct_equation(small_case):
    """The gridded operator (Eq. matrix_equation with the stacked factors of
    Sec. 3.1) approximates the direct measurement equation.  Pin: relative
    error at the method's accuracy class; a wrong sign, index or a dropped
    factor anywhere in S, Z, F, G or C gives O(1) errors.  Measured:
    1.2e-2 with the window disk of radius 1/2 (alpha = 1), 5e-4 at alpha = 1.5."""
    geo, uvw, x = small_case
    yd = O.direct(x, uvw, geo)
    for k, fold in ((1, False), (3, True)):
        plan = O.make_plan(uvw, geo, k, fold)
        assert O.rel_l2(O.degrid(plan, x), yd) < 2e-2
    geo15 = tiny_geo(alpha=1.5, tol_rel=1e-10, tol_abs=1e-10)
    plan = O.make_plan(uvw[:40], geo15, 2, True)
    assert O.rel_l2(O.degrid(plan, x), yd[:40]) < 1.5e-3


def test_operator_reflection_symmetry(small_case):
    """Sec. 3.3 holds for the discretised operator: Phi at (-u, -v, -w) is the
    conjugate of Phi at (u, v, w) for a real image (tap sets reflect, the
    stack centre flips sign, K(rho, -w) = conj K(rho, w))."""
    geo, uvw, x = small_case
    a = O.degrid(O.make_plan(uvw[:40], geo, 2, False), x)
    b = O.degrid(O.make_plan(-uvw[:40], geo, 2, False), x)
    assert O.rel_l2(b, np.conj(a)) < 1e-12


def test_adjoint_dot_product(small_case):
    """<Phi x, y> = <x, Phi^H y> with the real inner product (fold on, so Phi
    is R-linear and the adjoint returns Re)."""
    geo, uvw, _ = small_case
    plan = O.make_plan(uvw[:60], geo, 2, True, weights=np.linspace(0.5, 1.5, 60))
    x = W.random_image(128, 1)
    y = W.random_vis(60, 1)
    lhs = np.real(np.vdot(y, O.degrid(plan, x)))
    rhs = float(np.sum(x * O.grid(plan, y)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_circular_wrap_at_grid_edge():
    """G is a circular convolution (Sec. 2): a visibility inside the grid but
    within J_w/2 of its edge takes taps across the edge, stored at q mod Npad.
    Pin: the tap sum with every tap's DFT value computed naively at its
    unwrapped frequency q (the padded image's DFT is Npad-periodic in q)."""
    geo = tiny_geo(tol_rel=1e-10, tol_abs=1e-10)
    x = W.point_sources(128, 5, 9)
    uvw = np.array([[(geo.Npad / 2 - 0.4) * geo.du, (-geo.Npad / 2 + 0.7) * geo.du, 6.0]])
    plan = O.make_plan(uvw, geo, 1, False)
    assert not plan.dropped[0]
    y = O.degrid(plan, x)[0]
    xs = x * O.stack_correction(plan.wbar[0], geo)
    l, m = geo.pixel_lm()
    nz = np.nonzero(xs)
    J = int(plan.jw[0])
    q0u = math.floor(plan.upix[0] - J / 2) + 1
    q0v = math.floor(plan.vpix[0] - J / 2) + 1
    ref = 0
    for b in range(J):
        for a in range(J):
            qu, qv = q0u + a, q0v + b
            xq = np.sum(xs[nz] * np.exp(-2j * np.pi * geo.du * (qu * l[nz] + qv * m[nz])))
            rho = math.hypot(plan.upix[0] - qu, plan.vpix[0] - qv)
            ref += O.wkernel(rho, plan.dw[0], geo)[0] * xq
    assert q0u + J - 1 >= geo.Npad // 2 and q0v < -geo.Npad // 2
    assert abs(y - ref) < 1e-11 * abs(ref)


def test_visibilities_outside_grid_are_dropped():
    geo = tiny_geo()
    h = geo.Npad / 2 * geo.du
    uvw = np.array([[h * 1.01, 0, 0], [0, -h * 1.001, 0], [h * 0.99, -h * 0.99, 1.0]])
    plan = O.make_plan(uvw, geo, 1, False)
    assert list(plan.dropped) == [True, True, False]
    assert list(plan.jw[:2]) == [0, 0]
    y = O.degrid(plan, np.ones((128, 128)))
    assert y[0] == 0 and y[1] == 0 and y[2] != 0


@pytest.mark.parametrize("J", [4, 8])
def test_tap_box_is_exact_for_positions_one_ulp_from_integers(J):
    """The J x J box holds the J nearest grid points per axis, q in
    (u - J/2, u + J/2] (Sec. 2; half-open on the low side).  Pin: the
    footprint of one gridded visibility against that box computed in exact
    rational arithmetic, at doubles one ulp either side of integers and
    half-integers, where forming u - J/2 in floating point would round."""
    from fractions import Fraction
    geo = O.Geometry(128, 2.0, math.radians(20.0), float(J), tol_rel=1e-8, tol_abs=1e-8)
    plan = O.make_plan(np.array([[0.0, 0.0, 3.0]]), geo, 1, False)
    vals = []
    for k in (-28.0, -3.0, 0.0, 5.0, 17.5, -9.5):
        vals += [np.nextafter(k, -np.inf), k, np.nextafter(k, np.inf)]
    for u in vals:
        v = vals[(vals.index(u) + 4) % len(vals)]
        plan.upix[0], plan.vpix[0] = u, v
        grids, _, _ = O.grid_to_stacks(plan, np.array([1.0 + 0.0j]))
        g = grids[0]
        rows, cols = np.nonzero(np.abs(g) > 0)
        for pos, found in ((u, set(cols.tolist())), (v, set(rows.tolist()))):
            q0 = math.floor(Fraction(float(pos)) - Fraction(J, 2)) + 1
            want = {q % geo.Npad for q in range(q0, q0 + J)}
            assert found == want, (float(pos).hex(), J)


# ---------------------------------------------------------------- pre-sampled w-planes

@pytest.fixture(scope="module")
def table_case():
    geo = tiny_geo(tol_rel=1e-12, tol_abs=1e-12)
    uvw = W.uvw_disk(60, 60.0, 40.0, 41)
    plan = O.make_plan(uvw, geo, 2, True)
    return geo, uvw, plan, O.make_table(plan, 1e-3)


def test_table_reproduces_samples_and_meets_its_tolerance(table_case):
    """Sec. 5.1.1: bilinear interpolation between 1-D w-planes.  At sample
    points the table returns the quadrature value; in between, the error
    stays inside the tolerance the spacing was derived from; negative w is
    the conjugate (Sec. 5.1.1 / Sec. 3.3)."""
    geo, _, plan, tab = table_case
    i = np.array([0, 5, 17, tab.nr - 3])
    j = np.array([0, 2, tab.nw // 2, tab.nw - 2])
    k = O.table_kernel(tab, i * tab.hr, j * tab.hw)
    assert np.allclose(k, tab.values[j, i], atol=1e-15)
    rng = np.random.default_rng(2)
    rmax, dmax = O.table_extent(plan)
    rho = rng.uniform(0, rmax - 2, 300)
    dw = rng.uniform(-dmax, dmax, 300)
    err = np.abs(O.table_kernel(tab, rho, dw) - O.wkernel(rho, dw, geo))
    assert err.max() <= 1e-3
    assert np.allclose(O.table_kernel(tab, rho, -dw), np.conj(O.table_kernel(tab, rho, dw)))


def test_table_operator_close_to_direct_operator(table_case):
    """The tabulated operator differs from the quadrature operator by the
    interpolation error only; its adjoint pairs exactly."""
    geo, uvw, plan, tab = table_case
    x = W.point_sources(128, 10, 41)
    yq = O.degrid(plan, x)
    yt = O.degrid_table(plan, x, tab)
    assert O.rel_l2(yt, yq) < 2e-3
    xr = W.random_image(128, 4)
    yr = W.random_vis(len(uvw), 4)
    lhs = np.real(np.vdot(yr, O.degrid_table(plan, xr, tab)))
    rhs = float(np.sum(xr * O.grid_table(plan, yr, tab)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------- direction-dependent effects

@pytest.fixture(scope="module")
def dde_case():
    geo = tiny_geo(tol_rel=1e-11, tol_abs=1e-11)
    uvw = W.uvw_disk(40, 40.0, 30.0, 61)
    plan = O.make_plan(uvw, geo, 2, False)
    x = W.point_sources(128, 10, 61)
    return geo, uvw, plan, x


def test_dde_delta_is_the_plain_operator(dde_case):
    """D = delta (J_D = 1): the combined kernel is the w-kernel (Sec. 5.2)."""
    geo, uvw, plan, x = dde_case
    n = len(uvw)
    one = np.ones((n, 1), np.complex128)
    assert O.rel_l2(O.degrid_dde(plan, x, one, one), O.degrid(plan, x)) < 1e-12
    yr = W.random_vis(n, 62)
    assert O.rel_l2(O.grid_dde(plan, yr, one, one), O.grid(plan, yr)) < 1e-12


@pytest.mark.parametrize("su,sv", [(1, 0), (-2, 1), (0, -2)])
def test_dde_shifted_delta_moves_the_visibility(dde_case, su, sv):
    """D = delta at grid offset s: C(q) = [GC](u - s - q), i.e. the plain
    operator for the visibility moved by -s pixels (same stacks and supports,
    since w is unchanged)."""
    geo, uvw, plan, x = dde_case
    n, h = len(uvw), 2
    a = np.zeros((n, 2 * h + 1), np.complex128)
    b = np.zeros((n, 2 * h + 1), np.complex128)
    a[:, su + h] = 1.0
    b[:, sv + h] = 1.0
    moved = uvw.copy()
    moved[:, 0] -= su * geo.du
    moved[:, 1] -= sv * geo.du
    plan_m = O.make_plan(moved, geo, 2, False)
    assert np.array_equal(plan_m.stack, plan.stack) and np.array_equal(plan_m.jw, plan.jw)
    assert O.rel_l2(O.degrid_dde(plan, x, a, b), O.degrid(plan_m, x)) < 1e-12
    yr = W.random_vis(n, 63)
    assert O.rel_l2(O.grid_dde(plan, yr, a, b), O.grid(plan_m, yr)) < 1e-12


def test_dde_adjoint_and_linearity(dde_case):
    geo, uvw, plan, x = dde_case
    n = len(uvw)
    a, b = W.dde_kernels(n, 5, 64)
    xr = W.random_image(128, 65)
    yr = W.random_vis(n, 66)
    y = O.degrid_dde(plan, xr, a, b)
    lhs = np.real(np.vdot(yr, y))
    rhs = np.sum(xr * O.grid_dde(plan, yr, a, b))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    c = 0.3 - 1.7j
    assert O.rel_l2(O.degrid_dde(plan, xr, c * a, b), c * y) < 1e-13


def test_dde_refuses_folded_plans():
    geo = tiny_geo()
    uvw = W.uvw_disk(10, 40.0, 30.0, 67)
    plan = O.make_plan(uvw, geo, 1, True)
    assert plan.flag.any()
    one = np.ones((10, 1), np.complex128)
    with pytest.raises(ValueError):
        O.degrid_dde(plan, np.zeros((128, 128)), one, one)
