"""FP64 CPU oracle for the hybrid w-stacking w-projection operator
Phi = W G C F Z S (arXiv 1903.06555, Sec. 2-3).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg may use this package; the product (paper_1903_06555_gb300)
never imports it and shares no code with it.

The oracle follows the paper's factorisation step by step, in double
precision, with no blocking, fusion or reordering:

  fold (Sec. 3.3)  ->  k-means w-stacks (Algorithm 1)  ->  per stack k:
  S~_k (Eq. S~_k: x e^{-2 pi i wbar_k (n-1)} / (g n))  ->  Z (centred zero
  pad)  ->  F (unnormalised FFT, numpy)  ->  G C_k (Eq. GC_k: one adaptive
  Gauss-Kronrod integral of Eq. analytic_convolution_hankel per tap)  ->  W.

The adjoint is the exact conjugate transpose of the same steps, summed over
stacks (Eq. stacked adjoint) and restricted to its real part (the image is
real, so the fold makes Phi only R-linear).

Readings of points the paper leaves open (kernel normalisation, taper,
window radius, support rule, tap placement, Algorithm 1 details, quadrature
acceptance test) are stated where they are used below.

Pins (tests/test_oracle_*.py) check every function against something other
than itself: closed forms, library routines, an independent 2-D quadrature,
the direct measurement equation, brute force on tiny inputs, exactness of the
quadrature rule on polynomials, and adjoint/symmetry identities.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

from . import build as _build

_LIB = None

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_uint8_p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        for name in ("orc_bessel_j0", "orc_bessel_j1", "orc_bessel_i0", "orc_bessel_i1"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        L.orc_kb.restype = d
        L.orc_kb.argtypes = [d, d, d]
        L.orc_taper.restype = d
        L.orc_taper.argtypes = [d, d, d]
        L.orc_taper_many.restype = None
        L.orc_taper_many.argtypes = [c_double_p, i64, d, d, c_double_p]
        L.orc_chirp.restype = None
        L.orc_chirp.argtypes = [d, d, d, c_double_p]
        L.orc_wkernel.restype = None
        L.orc_wkernel.argtypes = [c_double_p, c_double_p, i64, c_double_p, c_double_p,
                                  c_double_p, c_int64_p, c_int64_p]
        L.orc_wkernel_2d.restype = None
        L.orc_wkernel_2d.argtypes = [c_double_p, c_double_p, c_double_p, i64, c_double_p,
                                     c_double_p, c_double_p, i32, i32, i32, c_double_p]
        L.orc_direct.restype = None
        L.orc_direct.argtypes = [c_double_p, c_double_p, c_double_p, i64, c_double_p, i64,
                                 c_double_p]
        for name in ("orc_degrid", "orc_grid"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [c_double_p, i64, c_double_p, c_double_p, i64, c_double_p,
                          c_double_p, c_double_p, c_int32_p, c_double_p, c_uint8_p,
                          c_double_p, c_int64_p, c_int64_p]
        L.orc_table_kernel.restype = None
        L.orc_table_kernel.argtypes = [c_double_p, c_double_p, i64, c_double_p, i64, i64, d, d,
                                       c_double_p]
        L.orc_degrid_table.restype = None
        L.orc_degrid_table.argtypes = [c_double_p, i64, c_double_p, i64, i64, d, d, i64,
                                       c_double_p, c_double_p, c_double_p, c_int32_p, c_double_p,
                                       c_uint8_p, c_double_p]
        L.orc_grid_table.restype = None
        L.orc_grid_table.argtypes = L.orc_degrid_table.argtypes
        L.orc_kmeans.restype = ctypes.c_int
        L.orc_kmeans.argtypes = [c_double_p, i64, i32, i32, d, c_int32_p, c_double_p]
        _LIB = L
    return _LIB


def _p(a, t=c_double_p):
    return a.ctypes.data_as(t)


# ----------------------------------------------------------------------------
# Gauss-Kronrod (7, 15) rule, derived here from its definition
# ----------------------------------------------------------------------------

def _legendre_power_coeffs(n):
    """Legendre P_n in the power basis, exact rationals (Bonnet recursion)."""
    p0, p1 = [Fraction(1)], [Fraction(0), Fraction(1)]
    if n == 0:
        return p0
    for k in range(1, n):
        # (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
        nxt = [Fraction(0)] * (k + 2)
        for i, c in enumerate(p1):
            nxt[i + 1] += Fraction(2 * k + 1, k + 1) * c
        for i, c in enumerate(p0):
            nxt[i] -= Fraction(k, k + 1) * c
        p0, p1 = p1, nxt
    return p1


_GK = None


def gauss_kronrod_15():
    """(nodes, kronrod weights, gauss weights) on [-1, 1], 15 entries each.

    The 7 Gauss nodes are the zeros of P_7.  The 8 added Kronrod nodes are
    the zeros of the Stieltjes polynomial E_8, the monic degree-8 polynomial
    orthogonal to x^k P_7(x) for k = 0..7; by parity E_8 is even and only odd
    k give conditions.  The 15 Kronrod weights make the rule exact for
    P_0..P_14.  Exactness up to degree 22 (Kronrod) and 13 (Gauss) is pinned
    in the tests.
    """
    global _GK
    if _GK is not None:
        return _GK
    p7 = _legendre_power_coeffs(7)

    def mom(j):  # integral of P_7(x) x^j over [-1, 1]
        s = Fraction(0)
        for i, c in enumerate(p7):
            d = i + j
            if d % 2 == 0:
                s += c * Fraction(2, d + 1)
        return s

    # E(x) = x^8 + c3 x^6 + c2 x^4 + c1 x^2 + c0, conditions k = 1, 3, 5, 7.
    rows = [[mom(k + 2 * m) for m in range(4)] for k in (1, 3, 5, 7)]
    rhs = [-mom(k + 8) for k in (1, 3, 5, 7)]
    # exact Gaussian elimination over the rationals
    n = 4
    A = [r[:] + [b] for r, b in zip(rows, rhs)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    c = [A[i][n] / A[i][i] for i in range(n)]
    quart = [1.0] + [float(c[3]), float(c[2]), float(c[1]), float(c[0])]
    ys = np.sort(np.real(np.roots(quart)))
    xs = np.sqrt(ys)

    def e8(x):
        y = x * x
        return (((y + float(c[3])) * y + float(c[2])) * y + float(c[1])) * y + float(c[0])

    def de8(x):
        y = x * x
        return 2 * x * (((4 * y + 3 * float(c[3])) * y + 2 * float(c[2])) * y + float(c[1]))

    for _ in range(3):  # Newton polish
        xs = xs - e8(xs) / de8(xs)
    xg, wg7 = np.polynomial.legendre.leggauss(7)
    nodes = np.sort(np.concatenate([xg, xs, -xs]))
    V = np.polynomial.legendre.legvander(nodes, 14).T
    b = np.zeros(15)
    b[0] = 2.0
    wk = np.linalg.solve(V, b)
    wg = np.zeros(15)
    for x, w in zip(xg, wg7):
        wg[np.argmin(np.abs(nodes - x))] = w
    _GK = (nodes, wk, wg)
    return _GK


def _rule_block():
    x, wk, wg = gauss_kronrod_15()
    return np.ascontiguousarray(np.concatenate([x, wk, wg]))


# ----------------------------------------------------------------------------
# Geometry and parameters
# ----------------------------------------------------------------------------

def beatty_beta(J: float, os_: float) -> float:
    """Kaiser-Bessel shape from Beatty, Nishimura & Pauly (2005):
    beta = pi sqrt((J/os)^2 (os - 1/2)^2 - 0.8).  The paper does not name
    its taper; this reading is the one used throughout."""
    return math.pi * math.sqrt((J / os_) ** 2 * (os_ - 0.5) ** 2 - 0.8)


@dataclass
class Geometry:
    """Image and grid geometry.

    Pixels: l_j = (j - N/2) dl, dl = fov/N (uniform in direction cosine;
    row index = m, column index = l).  Grid: Npad = os N, du = 1/(Npad dl).
    Kernel radius variable r = du * l (cycles per grid pixel); the window of
    Eq. analytic_convolution_hankel is r <= R = alpha/2, read with alpha = 1
    (the disk inscribed in the padded period).  The kernel normalisation is
    2 pi instead of the paper's 2 pi / du^2: the paper's form is the
    continuous transform over dl dm, this one matches the unnormalised DFT of
    the padded image (the two differ by du^2, a scale that the paper's power
    method normalisation of Phi removes anyway).
    """
    N: int
    os: float
    fov: float
    J: float = 4.0
    beta: float = 0.0
    alpha: float = 1.0
    tol_rel: float = 1e-12
    tol_abs: float = 1e-12
    max_panels: int = 4000

    def __post_init__(self):
        self.Npad = int(round(self.os * self.N))
        if self.Npad % 2 or self.N % 2:
            raise ValueError("N and os*N must be even")
        if self.J != int(self.J) or int(self.J) % 2 or self.J < 2:
            raise ValueError("support J must be an even integer >= 2")
        if self.beta == 0.0:
            self.beta = beatty_beta(self.J, self.os)
        self.dl = self.fov / self.N
        self.du = 1.0 / (self.Npad * self.dl)
        self.R = 0.5 * self.alpha
        self.l_win = self.R / self.du
        if self.l_win >= 1.0:
            raise ValueError("kernel window reaches the horizon")
        self.n_win = math.sqrt(1.0 - self.l_win ** 2)
        # Support rule: the chirp exp(-2 pi i dw (n(l)-1)) has local frequency
        # dw l / n; at the window edge that is dw l_win / (n_win du) grid
        # pixels, added on both sides of the KB support.
        self.c_support = self.l_win / (self.n_win * self.du)

    def params(self, tol_rel=None, tol_abs=None):
        return np.array([self.du, self.R, float(self.J), self.beta,
                         self.tol_rel if tol_rel is None else tol_rel,
                         self.tol_abs if tol_abs is None else tol_abs,
                         float(self.max_panels)], dtype=np.float64)

    def pixel_lm(self):
        ax = (np.arange(self.N) - self.N // 2) * self.dl
        l = np.broadcast_to(ax[None, :], (self.N, self.N))
        m = np.broadcast_to(ax[:, None], (self.N, self.N))
        return l, m


def geometry_from(wl, **kw) -> Geometry:
    return Geometry(wl.image_n, wl.oversample, math.radians(wl.fov_deg), float(wl.support), **kw)


# ----------------------------------------------------------------------------
# Scalar functions (wrapped C core)
# ----------------------------------------------------------------------------

def kb(rho, J, beta):
    return np.vectorize(lib().orc_kb)(rho, float(J), float(beta))


def taper(r, J, beta):
    """g(r): 2-D Fourier transform of the radial KB kernel (closed form)."""
    r = np.asarray(r, np.float64)
    flat = np.ascontiguousarray(r.ravel())
    out = np.zeros(flat.size)
    lib().orc_taper_many(_p(flat), flat.size, float(J), float(beta), _p(out))
    return out.reshape(r.shape) if r.shape else float(out[0])


def chirp(r, dw, du):
    out = np.zeros(2)
    lib().orc_chirp(float(r), float(dw), float(du), _p(out))
    return complex(out[0], out[1])


def wkernel(rho, dw, geo: Geometry, tol_rel=None, tol_abs=None, return_stats=False):
    """[GC](rho, dw) by adaptive Gauss-Kronrod bisection (one integral per point)."""
    rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), np.broadcast(rho, dw).shape)).ravel()
    dw = np.ascontiguousarray(np.broadcast_to(np.asarray(dw, np.float64), rho.shape)).ravel()
    out = np.zeros(2 * rho.size)
    ev = np.zeros(1, np.int64)
    bad = np.zeros(1, np.int64)
    lib().orc_wkernel(_p(rho), _p(dw), rho.size, _p(geo.params(tol_rel, tol_abs)),
                      _p(_rule_block()), _p(out), _p(ev, c_int64_p), _p(bad, c_int64_p))
    k = out[0::2] + 1j * out[1::2]
    if return_stats:
        return k, int(ev[0]), int(bad[0])
    return k


def wkernel_2d(rho_u, rho_v, dw, geo: Geometry, n_gl=20, n_phi=None, n_y=None):
    """The same kernel as a 2-D integral over the window disk (no Bessel)."""
    ru = np.ascontiguousarray(np.atleast_1d(np.asarray(rho_u, np.float64)))
    rv = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_v, np.float64), ru.shape))
    d = np.ascontiguousarray(np.broadcast_to(np.asarray(dw, np.float64), ru.shape))
    if n_phi is None or n_y is None:
        cyc = 2 * geo.R * float(np.max(np.hypot(ru, rv))) + float(np.max(np.abs(d))) * (1 - geo.n_win)
        n = max(4, int(math.ceil(1.5 * cyc)) + 2)
        n_phi = n_phi or n
        n_y = n_y or n
    x, w = np.polynomial.legendre.leggauss(n_gl)
    out = np.zeros(2 * ru.size)
    lib().orc_wkernel_2d(_p(ru), _p(rv), _p(d), ru.size, _p(geo.params()), _p(x), _p(w),
                         n_gl, n_phi, n_y, _p(out))
    return out[0::2] + 1j * out[1::2]


# ----------------------------------------------------------------------------
# Direct measurement equation
# ----------------------------------------------------------------------------

def direct(x, uvw, geo: Geometry):
    """Eq. meas_eq on the pixel grid (a = 1), summed over non-zero pixels."""
    l, m = geo.pixel_lm()
    nz = np.nonzero(x)
    xv = np.ascontiguousarray(x[nz], dtype=np.float64)
    lp = np.ascontiguousarray(l[nz], dtype=np.float64)
    mp = np.ascontiguousarray(m[nz], dtype=np.float64)
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    y = np.zeros(2 * uvw.shape[0])
    lib().orc_direct(_p(xv), _p(lp), _p(mp), xv.size, _p(uvw), uvw.shape[0], _p(y))
    return y[0::2] + 1j * y[1::2]


# ----------------------------------------------------------------------------
# Plan: fold, Algorithm 1, per-visibility support and grid coordinates
# ----------------------------------------------------------------------------

def fold(uvw):
    """Sec. 3.3: y*(u, v, -|w|) = y(-u, -v, |w|).  Visibilities with w < 0 are
    reflected to (-u, -v, -w) and flagged; their model value is conjugated."""
    uvw = np.array(uvw, dtype=np.float64, copy=True)
    flag = uvw[:, 2] < 0.0
    uvw[flag] *= -1.0
    return uvw, flag


def kmeans(w, k, max_iter=100, tol=1e-3):
    """Algorithm 1 (see orc_kmeans for the reading).  Returns
    (stack index per visibility, centres, sweeps)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    st = np.zeros(w.size, np.int32)
    c = np.zeros(k)
    it = lib().orc_kmeans(_p(w), w.size, int(k), int(max_iter), float(tol), _p(st, c_int32_p), _p(c))
    return st, c, it


@dataclass
class OraclePlan:
    geo: Geometry
    n_stacks: int
    flag: np.ndarray      # bool, folded visibility
    stack: np.ndarray     # int32
    wbar: np.ndarray      # centres
    dw: np.ndarray        # w - wbar_stack
    jw: np.ndarray        # int32 support, 0 when dropped
    upix: np.ndarray      # u / du after folding
    vpix: np.ndarray
    weight: np.ndarray
    dropped: np.ndarray   # bool
    sweeps: int


class SupportError(ValueError):
    pass


SUPPORT_STACK = 0   # one support per stack from its largest |dw| (default)
SUPPORT_VIS = 1     # one support per visibility from its own |dw|


def support(dw, geo: Geometry):
    """J_w = J + 2 ceil(|dw| c), c = l_win/(n_win du): the KB support widened
    on both sides by the chirp's bandwidth at the window edge."""
    return (int(geo.J) + 2 * np.ceil(np.abs(dw) * geo.c_support)).astype(np.int32)


def make_plan(uvw, geo: Geometry, n_stacks=1, conj_fold=False, weights=None,
              kmeans_max_iter=100, kmeans_tol=1e-3, max_support=64,
              support_rule=SUPPORT_STACK, centres=None, stack_jw=None) -> OraclePlan:
    """Fold, Algorithm 1, grid coordinates u/du, drop visibilities whose own
    (u, v) lies outside the padded grid [-Npad/2, Npad/2) (their taps would
    alias; the taps of every kept visibility wrap circularly, G being a
    circular convolution), then the support: per stack from the largest |dw|
    of its kept visibilities (SUPPORT_STACK) or per visibility.

    With `centres`, Algorithm 1 is replaced by one assignment of every
    visibility to its nearest given centre (lowest index on ties), and the
    centres are kept; with `stack_jw` the per-stack supports are given."""
    uvw = np.asarray(uvw, dtype=np.float64)
    if not np.all(np.isfinite(uvw)):
        raise ValueError("non-finite baseline coordinates")
    if conj_fold:
        uvw, flag = fold(uvw)
    else:
        flag = np.zeros(uvw.shape[0], bool)
    if centres is None:
        st, c, it = kmeans(uvw[:, 2], n_stacks, kmeans_max_iter, kmeans_tol)
    else:
        c = np.asarray(centres, np.float64)
        st = np.argmin((c[None, :] - uvw[:, 2:3]) ** 2, axis=1).astype(np.int32)
        it = 0
    dw = uvw[:, 2] - c[st]
    upix = uvw[:, 0] / geo.du
    vpix = uvw[:, 1] / geo.du
    h = geo.Npad // 2
    dropped = (upix < -h) | (upix >= h) | (vpix < -h) | (vpix >= h)
    if stack_jw is not None:
        jw = np.asarray(stack_jw, np.int32)[st]
    elif support_rule == SUPPORT_VIS:
        jw = support(dw, geo)
    else:
        jw = np.zeros(dw.size, np.int32)
        for k in range(n_stacks):
            s = (st == k) & ~dropped
            if s.any():
                jw[st == k] = support(np.max(np.abs(dw[s])), geo)
    jw = np.where(dropped, 0, jw).astype(np.int32)
    if jw.size and int(jw.max()) > max_support:
        raise SupportError(f"support {int(jw.max())} > {max_support}")
    wt = np.ones(uvw.shape[0]) if weights is None else np.asarray(weights, np.float64)
    return OraclePlan(geo, n_stacks, flag, st, c, dw, jw, upix, vpix, wt, dropped, it)


# ----------------------------------------------------------------------------
# Operator
# ----------------------------------------------------------------------------

def stack_correction(wbar_k, geo: Geometry):
    """[S~_k]_ii = e^{-2 pi i wbar_k (n_i - 1)} / (g(du |l_i|) n_i) with a_k = 1
    (Eq. S~_k), on the N x N pixel grid."""
    l, m = geo.pixel_lm()
    s = l * l + m * m
    if np.any(s >= 1.0):
        raise ValueError("image reaches the horizon")
    n = np.sqrt(1.0 - s)
    nm1 = -s / (1.0 + n)
    g = taper(geo.du * np.sqrt(s), geo.J, geo.beta)
    return np.exp(-2j * np.pi * wbar_k * nm1) / (g * n)


def pad_fft(xs, geo: Geometry):
    """Z then F: centre the N x N image in Npad x Npad zeros and take the
    unnormalised DFT Xhat(q) = sum_P X_P e^{-2 pi i q (P - Npad/2)/Npad};
    frequency q is stored at index q mod Npad."""
    o = (geo.Npad - geo.N) // 2
    z = np.zeros((geo.Npad, geo.Npad), np.complex128)
    z[o:o + geo.N, o:o + geo.N] = xs
    return np.fft.fft2(np.fft.ifftshift(z))


def fft_adjoint_crop(grid, geo: Geometry):
    """Adjoint of pad_fft: unnormalised inverse DFT, then crop."""
    z = np.fft.fftshift(np.fft.ifft2(grid)) * (geo.Npad * geo.Npad)
    o = (geo.Npad - geo.N) // 2
    return z[o:o + geo.N, o:o + geo.N]


def _vis_args(plan: OraclePlan, idx):
    return (np.ascontiguousarray(plan.upix[idx]), np.ascontiguousarray(plan.vpix[idx]),
            np.ascontiguousarray(plan.dw[idx]), np.ascontiguousarray(plan.jw[idx], np.int32),
            np.ascontiguousarray(plan.weight[idx]), np.ascontiguousarray(plan.flag[idx], np.uint8))


def stack_grids(plan: OraclePlan, x, stacks=None):
    """F Z S~_k x for every stack k (or the listed ones): {k: Xhat_k}."""
    geo = plan.geo
    ks = range(plan.n_stacks) if stacks is None else stacks
    return {k: np.ascontiguousarray(pad_fft(x * stack_correction(plan.wbar[k], geo), geo))
            for k in ks}


def degrid_from_grids(plan: OraclePlan, grids, idx, tol_rel=None, tol_abs=None):
    """W G C_k for the visibilities `idx` (caller order kept), given the
    stack grids.  Returns (y[idx], integrand evaluations, unconverged taps)."""
    geo = plan.geo
    idx = np.asarray(idx)
    y = np.zeros(idx.size, np.complex128)
    prm = geo.params(tol_rel, tol_abs)
    rule = _rule_block()
    ev_tot = bad_tot = 0
    for k in range(plan.n_stacks):
        pos = np.nonzero(plan.stack[idx] == k)[0]
        if pos.size == 0:
            continue
        sub = idx[pos]
        g = grids[k]
        u, v, d, j, wt, fl = _vis_args(plan, sub)
        out = np.zeros(2 * sub.size)
        ev = np.zeros(1, np.int64)
        bad = np.zeros(1, np.int64)
        lib().orc_degrid(g.view(np.float64).ctypes.data_as(c_double_p), geo.Npad, _p(prm),
                         _p(rule), sub.size, _p(u), _p(v), _p(d), _p(j, c_int32_p), _p(wt),
                         _p(fl, c_uint8_p), _p(out), _p(ev, c_int64_p), _p(bad, c_int64_p))
        y[pos] = out[0::2] + 1j * out[1::2]
        ev_tot += int(ev[0])
        bad_tot += int(bad[0])
    return y, ev_tot, bad_tot


def grid_to_stacks(plan: OraclePlan, y, idx=None, tol_rel=None, tol_abs=None):
    """(G C_k)^H W for the visibilities `idx` (y indexed like idx): one
    accumulated grid per stack.  Returns ({k: grid}, evaluations, unconverged)."""
    geo = plan.geo
    idx = np.arange(plan.flag.size) if idx is None else np.asarray(idx)
    y = np.asarray(y, np.complex128)
    prm = geo.params(tol_rel, tol_abs)
    rule = _rule_block()
    grids = {}
    ev_tot = bad_tot = 0
    for k in range(plan.n_stacks):
        pos = np.nonzero(plan.stack[idx] == k)[0]
        if pos.size == 0:
            continue
        sub = idx[pos]
        g = np.zeros((geo.Npad, geo.Npad), np.complex128)
        u, v, d, j, wt, fl = _vis_args(plan, sub)
        yk = np.ascontiguousarray(y[pos])
        ev = np.zeros(1, np.int64)
        bad = np.zeros(1, np.int64)
        lib().orc_grid(g.view(np.float64).ctypes.data_as(c_double_p), geo.Npad, _p(prm),
                       _p(rule), sub.size, _p(u), _p(v), _p(d), _p(j, c_int32_p), _p(wt),
                       _p(fl, c_uint8_p), yk.view(np.float64).ctypes.data_as(c_double_p),
                       _p(ev, c_int64_p), _p(bad, c_int64_p))
        grids[k] = g
        ev_tot += int(ev[0])
        bad_tot += int(bad[0])
    return grids, ev_tot, bad_tot


def image_from_grids(plan: OraclePlan, grids):
    """sum_k Re(conj(S~_k) Z^T F^H grid_k)."""
    geo = plan.geo
    x = np.zeros((geo.N, geo.N))
    for k, g in grids.items():
        x += np.real(np.conj(stack_correction(plan.wbar[k], geo)) * fft_adjoint_crop(g, geo))
    return x


def degrid(plan: OraclePlan, x, subset=None, tol_rel=None, tol_abs=None, return_stats=False):
    """y = Phi x (optionally only for the visibilities in `subset`)."""
    sel = np.arange(plan.flag.size) if subset is None else np.asarray(subset)
    grids = stack_grids(plan, x, sorted(set(int(k) for k in plan.stack[sel])))
    y, ev, bad = degrid_from_grids(plan, grids, sel, tol_rel, tol_abs)
    return (y, ev, bad) if return_stats else y


def grid(plan: OraclePlan, y, tol_rel=None, tol_abs=None, return_stats=False):
    """x = Re(Phi^H y): per stack, grid with the conjugate kernel, inverse
    unnormalised FFT, crop, multiply by conj(S~_k); summed over stacks."""
    grids, ev, bad = grid_to_stacks(plan, y, None, tol_rel, tol_abs)
    x = image_from_grids(plan, grids)
    return (x, ev, bad) if return_stats else x


# ----------------------------------------------------------------------------
# Direction-dependent effects (Sec. 5.2)
# ----------------------------------------------------------------------------
#
# A DDE model D_i in the uv domain, band-limited and given on the grid
# (integer offsets s, |s_u|, |s_v| <= h, J_D = 2 h + 1 taps a side), enters by
# a further convolution with the w-kernel: the combined kernel is
# (D_i * [GC])(x) = sum_s D_i(s) [GC](x - s), so visibility i degrids with
#     C_i(q) = sum_s D_i(s) [GC](|u_i/du - q - s|, dw_i)
# on the J_w + J_D - 1 box around it, and grids with its conjugate.  D_i is
# separable here, D_i(s) = a_i(s_u) b_i(s_v) (Sec. 5.2's cheaper case).  The
# fold's conjugate symmetry (Sec. 3.3) only holds for DDEs that are real in
# the image domain, so plans with folded visibilities are refused.


def dde_taps(plan: OraclePlan, i, a, b, tol_rel=None, tol_abs=None):
    """The combined taps C_i on the (J_w + J_D - 1)^2 box of visibility i,
    rows v, columns u, and the box's first grid index (q0u - h, q0v - h)."""
    geo = plan.geo
    J = int(plan.jw[i])
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    h = (a.size - 1) // 2
    q0u = int(np.floor(plan.upix[i])) - J // 2 + 1      # first tap, Sec. 2
    q0v = int(np.floor(plan.vpix[i])) - J // 2 + 1
    ku = plan.upix[i] - (q0u + np.arange(J))
    kv = plan.vpix[i] - (q0v + np.arange(J))
    rho = np.hypot(ku[None, :], kv[:, None]).ravel()
    K = wkernel(rho, np.full(rho.size, plan.dw[i]), geo, tol_rel, tol_abs).reshape(J, J)
    Jc = J + 2 * h
    C = np.zeros((Jc, Jc), np.complex128)
    # C[q] gets D(s) K[q + s - q0], i.e. K shifted by -s inside the larger box
    for sv in range(-h, h + 1):
        for su in range(-h, h + 1):
            C[h - sv:h - sv + J, h - su:h - su + J] += a[su + h] * b[sv + h] * K
    return C, q0u - h, q0v - h


def degrid_dde(plan: OraclePlan, x, a, b, tol_rel=None, tol_abs=None, subset=None):
    """y_i = W_i sum_q C_i(q) Xhat_k[q mod Npad] with the DDE kernels a[i],
    b[i] (J_D taps each, offsets -h..h); for the visibilities in `subset`
    only (caller order kept) when given."""
    if plan.flag.any():
        raise ValueError("DDE convolution needs a plan without the conjugate fold")
    geo = plan.geo
    sel = np.arange(plan.flag.size) if subset is None else np.asarray(subset)
    grids = stack_grids(plan, x, sorted(set(int(k) for k in plan.stack[sel])))
    y = np.zeros(plan.flag.size, np.complex128)
    for i in sel[~plan.dropped[sel]]:
        C, cu, cv = dde_taps(plan, i, a[i], b[i], tol_rel, tol_abs)
        n = C.shape[0]
        rows = (cv + np.arange(n)) % geo.Npad
        cols = (cu + np.arange(n)) % geo.Npad
        g = grids[int(plan.stack[i])]
        y[i] = plan.weight[i] * np.sum(C * g[np.ix_(rows, cols)])
    return y if subset is None else y[sel]


def grid_dde(plan: OraclePlan, y, a, b, tol_rel=None, tol_abs=None, subset=None):
    """x = Re(Phi_D^H y): every visibility (of `subset`, when given) spreads
    conj(C_i) W_i y_i over its box on its stack's grid; then as Phi^H."""
    if plan.flag.any():
        raise ValueError("DDE convolution needs a plan without the conjugate fold")
    geo = plan.geo
    sel = np.arange(plan.flag.size) if subset is None else np.asarray(subset)
    grids = {}
    for i in sel[~plan.dropped[sel]]:
        C, cu, cv = dde_taps(plan, i, a[i], b[i], tol_rel, tol_abs)
        n = C.shape[0]
        rows = (cv + np.arange(n)) % geo.Npad
        cols = (cu + np.arange(n)) % geo.Npad
        k = int(plan.stack[i])
        if k not in grids:
            grids[k] = np.zeros((geo.Npad, geo.Npad), np.complex128)
        grids[k][np.ix_(rows, cols)] += np.conj(C) * (plan.weight[i] * y[i])
    return image_from_grids(plan, grids)


# ----------------------------------------------------------------------------
# Pre-sampled 1-D w-planes (Sec. 5.1.1)
# ----------------------------------------------------------------------------

@dataclass
class KernelTable:
    """[GC](i hr, j hw) for i < nr, j < nw: positive rho and w only (Sec.
    5.1.1: the conjugate gives -w, radial symmetry gives negative u, v)."""
    hr: float
    hw: float
    values: np.ndarray      # complex128 (nw, nr)

    @property
    def nr(self):
        return self.values.shape[1]

    @property
    def nw(self):
        return self.values.shape[0]


def table_spacing(geo: Geometry, table_tol: float):
    """Sample spacing for a bilinear interpolation error <= table_tol.  The
    bilinear error is at most h^2/8 times the second derivative in each
    direction (half the budget each); the integrand's rho- and w-dependence
    (J0(2 pi rho r), e^{2 pi i w (1 - n(r))}) bounds those by (2 pi R)^2 and
    (2 pi (1 - n(R)))^2 times 2 pi int g r dr, taken as 1."""
    hr = math.sqrt(4.0 * table_tol) / (2.0 * math.pi * geo.R)
    hw = math.sqrt(4.0 * table_tol) / (2.0 * math.pi * (1.0 - geo.n_win))
    return hr, hw


def table_extent(plan: OraclePlan):
    """Largest tap radius and |dw| the plan can ask for: sqrt(2) J_max / 2
    (plus a margin) and the largest |dw| of its kept visibilities."""
    keep = ~plan.dropped
    jmax = int(plan.jw[keep].max()) if keep.any() else int(plan.geo.J)
    dmax = float(np.max(np.abs(plan.dw[keep]))) if keep.any() else 0.0
    return math.sqrt(2.0) * jmax / 2.0 + 2.0, dmax


def make_table(plan: OraclePlan, table_tol: float, tol_rel=None, tol_abs=None) -> KernelTable:
    hr, hw = table_spacing(plan.geo, table_tol)
    rmax, dmax = table_extent(plan)
    nr = int(math.ceil(rmax / hr)) + 2
    nw = int(math.ceil(dmax / hw)) + 2
    rho = np.arange(nr) * hr
    w = np.arange(nw) * hw
    R, Wg = np.meshgrid(rho, w)
    vals = wkernel(R.ravel(), Wg.ravel(), plan.geo, tol_rel, tol_abs).reshape(nw, nr)
    return KernelTable(hr, hw, np.ascontiguousarray(vals))


def table_kernel(table: KernelTable, rho, dw):
    rho = np.ascontiguousarray(np.atleast_1d(np.asarray(rho, np.float64)))
    dw = np.ascontiguousarray(np.broadcast_to(np.asarray(dw, np.float64), rho.shape))
    out = np.zeros(2 * rho.size)
    lib().orc_table_kernel(_p(rho), _p(dw), rho.size, table.values.view(np.float64).ctypes.data_as(
        c_double_p), table.nr, table.nw, table.hr, table.hw, _p(out))
    return out[0::2] + 1j * out[1::2]


def degrid_table(plan: OraclePlan, x, table: KernelTable, subset=None):
    """y = Phi x with every tap read from the table."""
    geo = plan.geo
    sel = np.arange(plan.flag.size) if subset is None else np.asarray(subset)
    grids = stack_grids(plan, x, sorted(set(int(k) for k in plan.stack[sel])))
    y = np.zeros(sel.size, np.complex128)
    tab = table.values.view(np.float64).ctypes.data_as(c_double_p)
    for k, g in grids.items():
        pos = np.nonzero(plan.stack[sel] == k)[0]
        sub = sel[pos]
        u, v, d, j, wt, fl = _vis_args(plan, sub)
        out = np.zeros(2 * sub.size)
        lib().orc_degrid_table(g.view(np.float64).ctypes.data_as(c_double_p), geo.Npad, tab,
                               table.nr, table.nw, table.hr, table.hw, sub.size, _p(u), _p(v),
                               _p(d), _p(j, c_int32_p), _p(wt), _p(fl, c_uint8_p), _p(out))
        y[pos] = out[0::2] + 1j * out[1::2]
    return y


def grid_table(plan: OraclePlan, y, table: KernelTable):
    """x = Re(Phi^H y) with every tap read from the table."""
    geo = plan.geo
    y = np.asarray(y, np.complex128)
    grids = {}
    tab = table.values.view(np.float64).ctypes.data_as(c_double_p)
    for k in range(plan.n_stacks):
        idx = np.nonzero(plan.stack == k)[0]
        if idx.size == 0:
            continue
        g = np.zeros((geo.Npad, geo.Npad), np.complex128)
        u, v, d, j, wt, fl = _vis_args(plan, idx)
        yk = np.ascontiguousarray(y[idx])
        lib().orc_grid_table(g.view(np.float64).ctypes.data_as(c_double_p), geo.Npad, tab,
                             table.nr, table.nw, table.hr, table.hw, idx.size, _p(u), _p(v),
                             _p(d), _p(j, c_int32_p), _p(wt), _p(fl, c_uint8_p),
                             yk.view(np.float64).ctypes.data_as(c_double_p))
        grids[k] = g
    return image_from_grids(plan, grids)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))
