/*
 * FP64 CPU oracle for the hybrid w-stacking w-projection measurement operator
 * Phi = W G C F Z S of Pratley, Johnston-Hollitt & McEwen (arXiv 1903.06555).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  The product (the CUDA library) never
 * links, loads or calls this file, and this file shares no code, header, table
 * or constant with it.
 *
 * Everything here is plain double precision, one integral per kernel tap, in
 * the order the paper states the operator:
 *   - Kaiser-Bessel interpolation kernel k(rho) and its 2-D Fourier transform
 *     g(r), the radial anti-aliasing taper of Sec. 3.1 (closed form: Lewitt
 *     1990, generalised KB of order 0 in two dimensions);
 *   - the radial w-projection kernel [GC](rho, dw) of Eq. analytic_convolution_hankel,
 *     computed by globally adaptive Gauss-Kronrod (7/15) bisection with the
 *     error estimate |K15 - G7| on the complex value;
 *   - an independent 2-D quadrature of the same kernel over the window disk
 *     (no Bessel function), used to pin the radial reduction;
 *   - the direct measurement equation (Eq. meas_eq) as a sum over pixels;
 *   - degridding G (Eq. GC_k) and its adjoint gridding G^H for one w-stack;
 *   - Algorithm 1 (k-means w-stacking), single process.
 *
 * Parameter block `prm` (doubles): [0] du (grid spacing, wavelengths),
 * [1] R (window radius in r = du * l units), [2] J (KB support, grid pixels),
 * [3] beta (KB shape), [4] relative tolerance, [5] absolute tolerance,
 * [6] maximum number of panels per integral.
 *
 * Quadrature rule block `rule` (45 doubles): 15 nodes on [-1, 1], 15 Kronrod
 * weights, 15 Gauss weights (zero at the Kronrod-only nodes).  The Python side
 * derives the rule itself from the Legendre and Stieltjes polynomials.
 */
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <limits>
#include <queue>
#include <vector>

namespace {

typedef std::complex<double> cd;
const double kPi = 3.14159265358979323846264338327950288;

double bessel_j0(double x) { return ::j0(x); }
double bessel_j1(double x) { return ::j1(x); }
double bessel_i0(double x) { return std::cyl_bessel_i(0.0, x); }
double bessel_i1(double x) { return std::cyl_bessel_i(1.0, x); }

struct Params {
  double du, R, J, beta, tol_rel, tol_abs;
  int max_panels;
  double i0beta;
  explicit Params(const double* p)
      : du(p[0]), R(p[1]), J(p[2]), beta(p[3]), tol_rel(p[4]), tol_abs(p[5]),
        max_panels(static_cast<int>(p[6])), i0beta(bessel_i0(p[3])) {}
};

// Kaiser-Bessel kernel, radial in grid pixels, support |rho| <= J/2, k(0) = 1.
double kb(double rho, double J, double beta) {
  double t = 2.0 * rho / J;
  if (std::fabs(t) > 1.0) return 0.0;
  return bessel_i0(beta * std::sqrt(1.0 - t * t)) / bessel_i0(beta);
}

// g(r) = int k(|rho|) exp(-2 pi i rho.r) d^2 rho, r in cycles per grid pixel.
// With a = J/2 and z^2 = beta^2 - (2 pi a r)^2:
//   g = 2 pi a^2 I1(z) / (z I0(beta))   for z^2 > 0,
//   g = 2 pi a^2 J1(zeta) / (zeta I0(beta)), zeta^2 = -z^2, otherwise.
double taper(double r, double J, double beta, double i0beta) {
  double a = 0.5 * J;
  double q = 2.0 * kPi * a * r;
  double z2 = beta * beta - q * q;
  double f;
  if (std::fabs(z2) < 1e-12) {
    f = 0.5 + z2 / 16.0;
  } else if (z2 > 0.0) {
    double z = std::sqrt(z2);
    f = bessel_i1(z) / z;
  } else {
    double z = std::sqrt(-z2);
    f = bessel_j1(z) / z;
  }
  return 2.0 * kPi * a * a * f / i0beta;
}

// exp(-2 pi i dw (n(r) - 1)) with n = sqrt(1 - l^2), l = r / du;
// n - 1 = -s / (1 + sqrt(1 - s)) avoids cancellation for small s = l^2.
cd chirp(double r, double dw, double du) {
  double l = r / du;
  double s = l * l;
  double nm1 = -s / (1.0 + std::sqrt(1.0 - s));
  double ph = -2.0 * kPi * dw * nm1;
  return cd(std::cos(ph), std::sin(ph));
}

// Integrand of the radial kernel: 2 pi g(r) chirp(r) J0(2 pi rho r) r.
cd radial_integrand(double r, double rho, double dw, const Params& P) {
  return 2.0 * kPi * taper(r, P.J, P.beta, P.i0beta) * chirp(r, dw, P.du) *
         bessel_j0(2.0 * kPi * rho * r) * r;
}

struct Panel {
  double a, b;
  cd val;
  double err;
  bool operator<(const Panel& o) const { return err < o.err; }
};

Panel gk_panel(double a, double b, double rho, double dw, const Params& P, const double* rule) {
  const double* x = rule;
  const double* wk = rule + 15;
  const double* wg = rule + 30;
  double c = 0.5 * (a + b), h = 0.5 * (b - a);
  cd k(0.0, 0.0), g(0.0, 0.0);
  for (int j = 0; j < 15; ++j) {
    cd f = radial_integrand(c + h * x[j], rho, dw, P);
    k += wk[j] * f;
    g += wg[j] * f;
  }
  k *= h;
  g *= h;
  Panel p{a, b, k, std::abs(k - g)};
  return p;
}

// Globally adaptive bisection on [0, R]: always split the panel with the
// largest error estimate until sum(err) <= max(tol_abs, tol_rel |sum(val)|).
cd radial_kernel(double rho, double dw, const Params& P, const double* rule,
                 int64_t* evals, bool* converged) {
  std::priority_queue<Panel> q;
  q.push(gk_panel(0.0, P.R, rho, dw, P, rule));
  int64_t n_eval = 15;
  cd total = q.top().val;
  double err = q.top().err;
  bool ok = false;
  while (true) {
    if (err <= std::max(P.tol_abs, P.tol_rel * std::abs(total))) {
      // confirm with freshly summed totals (running sums drift)
      std::priority_queue<Panel> copy = q;
      cd t2(0.0, 0.0);
      double e2 = 0.0;
      while (!copy.empty()) { t2 += copy.top().val; e2 += copy.top().err; copy.pop(); }
      total = t2;
      err = e2;
      if (err <= std::max(P.tol_abs, P.tol_rel * std::abs(total))) { ok = true; break; }
    }
    if (static_cast<int>(q.size()) >= P.max_panels) break;
    Panel worst = q.top();
    q.pop();
    double m = 0.5 * (worst.a + worst.b);
    Panel l = gk_panel(worst.a, m, rho, dw, P, rule);
    Panel r = gk_panel(m, worst.b, rho, dw, P, rule);
    n_eval += 30;
    total += l.val + r.val - worst.val;
    err += l.err + r.err - worst.err;
    q.push(l);
    q.push(r);
  }
  if (!ok) {
    cd t2(0.0, 0.0);
    while (!q.empty()) { t2 += q.top().val; q.pop(); }
    total = t2;
  }
  if (evals) *evals += n_eval;
  if (converged) *converged = ok;
  return total;
}

int64_t pmod(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

}  // namespace

extern "C" {

double orc_bessel_j0(double x) { return bessel_j0(x); }
double orc_bessel_j1(double x) { return bessel_j1(x); }
double orc_bessel_i0(double x) { return bessel_i0(x); }
double orc_bessel_i1(double x) { return bessel_i1(x); }
double orc_kb(double rho, double J, double beta) { return kb(rho, J, beta); }
double orc_taper(double r, double J, double beta) { return taper(r, J, beta, bessel_i0(beta)); }

void orc_taper_many(const double* r, int64_t n, double J, double beta, double* out) {
  double i0b = bessel_i0(beta);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = taper(r[i], J, beta, i0b);
}

void orc_chirp(double r, double dw, double du, double* out) {
  cd c = chirp(r, dw, du);
  out[0] = c.real();
  out[1] = c.imag();
}

// Radial kernel [GC](rho_i, dw_i) for n points.  out: interleaved complex.
void orc_wkernel(const double* rho, const double* dw, int64_t n, const double* prm,
                 const double* rule, double* out, int64_t* evals, int64_t* unconverged) {
  Params P(prm);
  int64_t ev = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ev, bad)
  for (int64_t i = 0; i < n; ++i) {
    int64_t e = 0;
    bool ok = true;
    cd k = radial_kernel(rho[i], dw[i], P, rule, &e, &ok);
    out[2 * i] = k.real();
    out[2 * i + 1] = k.imag();
    ev += e;
    bad += ok ? 0 : 1;
  }
  if (evals) *evals = ev;
  if (unconverged) *unconverged = bad;
}

// The same kernel as a 2-D integral over the window disk |r| <= R, without
// Bessel functions:  K = int int g(|r|) chirp(|r|) exp(-2 pi i (ru x + rv y)) dx dy.
// Outer variable x = R sin(phi), phi in [-pi/2, pi/2] (dx = R cos(phi) dphi),
// inner y in [-R cos(phi), R cos(phi)]; composite Gauss-Legendre in both with
// n_gl points per panel, n_phi and n_y panels.
void orc_wkernel_2d(const double* ru, const double* rv, const double* dw, int64_t n,
                    const double* prm, const double* gl_x, const double* gl_w, int n_gl,
                    int n_phi, int n_y, double* out) {
  Params P(prm);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    cd acc(0.0, 0.0);
    double hp = kPi / n_phi;
    for (int pp = 0; pp < n_phi; ++pp) {
      double c_phi = -0.5 * kPi + (pp + 0.5) * hp;
      for (int a = 0; a < n_gl; ++a) {
        double phi = c_phi + 0.5 * hp * gl_x[a];
        double wphi = 0.5 * hp * gl_w[a];
        double x = P.R * std::sin(phi);
        double ymax = P.R * std::cos(phi);
        double jac = P.R * std::cos(phi);
        double hy = 2.0 * ymax / n_y;
        cd inner(0.0, 0.0);
        for (int py = 0; py < n_y; ++py) {
          double c_y = -ymax + (py + 0.5) * hy;
          for (int b = 0; b < n_gl; ++b) {
            double y = c_y + 0.5 * hy * gl_x[b];
            double wy = 0.5 * hy * gl_w[b];
            double r = std::sqrt(x * x + y * y);
            double ph = -2.0 * kPi * (ru[i] * x + rv[i] * y);
            inner += wy * taper(r, P.J, P.beta, P.i0beta) * chirp(r, dw[i], P.du) *
                     cd(std::cos(ph), std::sin(ph));
          }
        }
        acc += wphi * jac * inner;
      }
    }
    out[2 * i] = acc.real();
    out[2 * i + 1] = acc.imag();
  }
}

// Direct measurement equation (Eq. meas_eq with a = 1) over the listed pixels:
// y_i = sum_p x_p / n_p exp(-2 pi i (u_i l_p + v_i m_p + w_i (n_p - 1))).
void orc_direct(const double* xv, const double* lp, const double* mp, int64_t npix,
                const double* uvw, int64_t m, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double u = uvw[3 * i], v = uvw[3 * i + 1], w = uvw[3 * i + 2];
    cd acc(0.0, 0.0);
    for (int64_t p = 0; p < npix; ++p) {
      double s = lp[p] * lp[p] + mp[p] * mp[p];
      double n = std::sqrt(1.0 - s);
      double nm1 = -s / (1.0 + n);
      double ph = -2.0 * kPi * (u * lp[p] + v * mp[p] + w * nm1);
      acc += (xv[p] / n) * cd(std::cos(ph), std::sin(ph));
    }
    y[2 * i] = acc.real();
    y[2 * i + 1] = acc.imag();
  }
}

// First tap of a J-wide box: q0 = floor(u - J/2) + 1, the smallest grid
// index above u - J/2 (the J nearest grid points, box half-open on the low
// side).  J is even, so q0 = floor(u) - J/2 + 1 exactly; forming u - J/2 in
// floating point first could round across an integer (u = -28 - 3.6e-15 with
// J = 8 gives -32 exactly) and shift the box by one.
static int64_t first_tap(double u, int J) {
  return static_cast<int64_t>(std::floor(u)) - J / 2 + 1;
}

// Degridding for one w-stack (Eq. GC_k):
//   y_i = W_i sum_{taps} [GC](|(u_i, v_i)/du - q|, dw_i) Xhat[q mod Npad],
// taps q = q0 + (a, b), a, b in [0, Jw_i), q0 = floor(u_i/du - Jw_i/2) + 1;
// conjugated when the visibility was folded.  grid: interleaved complex,
// row index = v, column index = u, frequency q stored at q mod Npad.
// Visibilities with jw == 0 are skipped (y = 0).
void orc_degrid(const double* grid, int64_t npad, const double* prm, const double* rule,
                int64_t nvis, const double* upix, const double* vpix, const double* dw,
                const int32_t* jw, const double* weight, const uint8_t* flag, double* y,
                int64_t* evals, int64_t* unconverged) {
  Params P(prm);
  int64_t ev = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : ev, bad)
  for (int64_t i = 0; i < nvis; ++i) {
    cd acc(0.0, 0.0);
    int J = jw[i];
    if (J > 0) {
      int64_t q0u = first_tap(upix[i], J);
      int64_t q0v = first_tap(vpix[i], J);
      for (int b = 0; b < J; ++b) {
        for (int a = 0; a < J; ++a) {
          double du_ = upix[i] - static_cast<double>(q0u + a);
          double dv_ = vpix[i] - static_cast<double>(q0v + b);
          double rho = std::sqrt(du_ * du_ + dv_ * dv_);
          int64_t e = 0;
          bool ok = true;
          cd k = radial_kernel(rho, dw[i], P, rule, &e, &ok);
          ev += e;
          bad += ok ? 0 : 1;
          int64_t idx = pmod(q0v + b, npad) * npad + pmod(q0u + a, npad);
          acc += k * cd(grid[2 * idx], grid[2 * idx + 1]);
        }
      }
      acc *= weight[i];
      if (flag[i]) acc = std::conj(acc);
    }
    y[2 * i] = acc.real();
    y[2 * i + 1] = acc.imag();
  }
  if (evals) *evals = ev;
  if (unconverged) *unconverged = bad;
}

// Adjoint of orc_degrid: grid[q] += conj([GC]) W_i ytilde_i with ytilde = conj(y)
// for folded visibilities.  Kernels are computed in parallel per chunk and
// scattered serially in visibility order.
void orc_grid(double* grid, int64_t npad, const double* prm, const double* rule, int64_t nvis,
              const double* upix, const double* vpix, const double* dw, const int32_t* jw,
              const double* weight, const uint8_t* flag, const double* y, int64_t* evals,
              int64_t* unconverged) {
  Params P(prm);
  int64_t ev = 0, bad = 0;
  const int64_t chunk = 512;
  int jmax = 0;
  for (int64_t i = 0; i < nvis; ++i) jmax = std::max(jmax, jw[i]);
  std::vector<cd> kbuf(static_cast<size_t>(chunk) * jmax * jmax);
  for (int64_t c0 = 0; c0 < nvis; c0 += chunk) {
    int64_t c1 = std::min(nvis, c0 + chunk);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ev, bad)
    for (int64_t i = c0; i < c1; ++i) {
      int J = jw[i];
      if (J <= 0) continue;
      int64_t q0u = first_tap(upix[i], J);
      int64_t q0v = first_tap(vpix[i], J);
      cd* kk = &kbuf[static_cast<size_t>(i - c0) * jmax * jmax];
      for (int b = 0; b < J; ++b)
        for (int a = 0; a < J; ++a) {
          double du_ = upix[i] - static_cast<double>(q0u + a);
          double dv_ = vpix[i] - static_cast<double>(q0v + b);
          int64_t e = 0;
          bool ok = true;
          kk[b * J + a] = radial_kernel(std::sqrt(du_ * du_ + dv_ * dv_), dw[i], P, rule, &e, &ok);
          ev += e;
          bad += ok ? 0 : 1;
        }
    }
    for (int64_t i = c0; i < c1; ++i) {
      int J = jw[i];
      if (J <= 0) continue;
      int64_t q0u = first_tap(upix[i], J);
      int64_t q0v = first_tap(vpix[i], J);
      cd yt(y[2 * i], y[2 * i + 1]);
      if (flag[i]) yt = std::conj(yt);
      yt *= weight[i];
      const cd* kk = &kbuf[static_cast<size_t>(i - c0) * jmax * jmax];
      for (int b = 0; b < J; ++b)
        for (int a = 0; a < J; ++a) {
          int64_t idx = pmod(q0v + b, npad) * npad + pmod(q0u + a, npad);
          cd add = std::conj(kk[b * J + a]) * yt;
          grid[2 * idx] += add.real();
          grid[2 * idx + 1] += add.imag();
        }
    }
  }
  if (evals) *evals = ev;
  if (unconverged) *unconverged = bad;
}

// Pre-sampled 1-D w-planes (Sec. 5.1.1): table[j][i] = [GC](i hr, j hw) for
// i < nr, j < nw (positive rho and w only), bilinear interpolation in
// (rho, |dw|), conjugated for dw < 0 (K(rho, -w) = conj K(rho, w)).
static cd table_kernel(double rho, double dw, const double* tab, int64_t nr, int64_t nw, double hr,
                       double hw) {
  double s = rho / hr;
  int64_t i = static_cast<int64_t>(std::floor(s));
  if (i > nr - 2) i = nr - 2;
  double fr = s - static_cast<double>(i);
  double t = std::fabs(dw) / hw;
  int64_t j = static_cast<int64_t>(std::floor(t));
  if (j > nw - 2) j = nw - 2;
  double fw = t - static_cast<double>(j);
  auto T = [&](int64_t jj, int64_t ii) {
    return cd(tab[2 * (jj * nr + ii)], tab[2 * (jj * nr + ii) + 1]);
  };
  cd lo = (1.0 - fr) * T(j, i) + fr * T(j, i + 1);
  cd hi = (1.0 - fr) * T(j + 1, i) + fr * T(j + 1, i + 1);
  cd k = (1.0 - fw) * lo + fw * hi;
  return dw < 0.0 ? std::conj(k) : k;
}

void orc_table_kernel(const double* rho, const double* dw, int64_t n, const double* tab, int64_t nr,
                      int64_t nw, double hr, double hw, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    cd k = table_kernel(rho[i], dw[i], tab, nr, nw, hr, hw);
    out[2 * i] = k.real();
    out[2 * i + 1] = k.imag();
  }
}

// Degridding / gridding of one stack with the tabulated kernel (same taps,
// weights and fold as orc_degrid / orc_grid).
void orc_degrid_table(const double* grid, int64_t npad, const double* tab, int64_t nr, int64_t nw,
                      double hr, double hw, int64_t nvis, const double* upix, const double* vpix,
                      const double* dw, const int32_t* jw, const double* weight,
                      const uint8_t* flag, double* y) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nvis; ++i) {
    cd acc(0.0, 0.0);
    int J = jw[i];
    if (J > 0) {
      int64_t q0u = first_tap(upix[i], J);
      int64_t q0v = first_tap(vpix[i], J);
      for (int b = 0; b < J; ++b)
        for (int a = 0; a < J; ++a) {
          double du_ = upix[i] - static_cast<double>(q0u + a);
          double dv_ = vpix[i] - static_cast<double>(q0v + b);
          cd k = table_kernel(std::sqrt(du_ * du_ + dv_ * dv_), dw[i], tab, nr, nw, hr, hw);
          int64_t idx = pmod(q0v + b, npad) * npad + pmod(q0u + a, npad);
          acc += k * cd(grid[2 * idx], grid[2 * idx + 1]);
        }
      acc *= weight[i];
      if (flag[i]) acc = std::conj(acc);
    }
    y[2 * i] = acc.real();
    y[2 * i + 1] = acc.imag();
  }
}

void orc_grid_table(double* grid, int64_t npad, const double* tab, int64_t nr, int64_t nw,
                    double hr, double hw, int64_t nvis, const double* upix, const double* vpix,
                    const double* dw, const int32_t* jw, const double* weight,
                    const uint8_t* flag, const double* y) {
  for (int64_t i = 0; i < nvis; ++i) {
    int J = jw[i];
    if (J <= 0) continue;
    int64_t q0u = first_tap(upix[i], J);
    int64_t q0v = first_tap(vpix[i], J);
    cd yt(y[2 * i], y[2 * i + 1]);
    if (flag[i]) yt = std::conj(yt);
    yt *= weight[i];
    for (int b = 0; b < J; ++b)
      for (int a = 0; a < J; ++a) {
        double du_ = upix[i] - static_cast<double>(q0u + a);
        double dv_ = vpix[i] - static_cast<double>(q0v + b);
        cd k = table_kernel(std::sqrt(du_ * du_ + dv_ * dv_), dw[i], tab, nr, nw, hr, hw);
        int64_t idx = pmod(q0v + b, npad) * npad + pmod(q0u + a, npad);
        cd add = std::conj(k) * yt;
        grid[2 * idx] += add.real();
        grid[2 * idx + 1] += add.imag();
      }
  }
}

// Algorithm 1 (k-means w-stacking), one process.  Centres start evenly spaced
// over [w_min, w_max] (endpoints included; the midpoint when K = 1).  Each
// sweep assigns every visibility to the nearest centre by (wbar_q - w_p)^2,
// the lowest index winning ties, then sets every centre to the mean of its
// members, or to 0 when it has none.  Iteration stops when the mean over
// centres of |wbar_new - wbar_old| / max(|wbar_old|, eps) is below tol,
// eps = (w_max - w_min) / K (1 when all w are equal), or after max_iter
// sweeps.  Returns the number of sweeps.
int orc_kmeans(const double* w, int64_t m, int k, int max_iter, double tol, int32_t* stack,
               double* centre) {
  double wmin = std::numeric_limits<double>::infinity();
  double wmax = -wmin;
  for (int64_t p = 0; p < m; ++p) {
    wmin = std::min(wmin, w[p]);
    wmax = std::max(wmax, w[p]);
  }
  if (m == 0) { wmin = 0.0; wmax = 0.0; }
  std::vector<double> c(k), sum(k);
  std::vector<int64_t> cnt(k);
  for (int q = 0; q < k; ++q)
    c[q] = (k == 1) ? 0.5 * (wmin + wmax) : wmin + q * (wmax - wmin) / (k - 1);
  double eps = (wmax - wmin) / k;
  if (!(eps > 0.0)) eps = 1.0;
  int t = 0;
  while (t < max_iter) {
    ++t;
    std::fill(sum.begin(), sum.end(), 0.0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t p = 0; p < m; ++p) {
      double best = std::numeric_limits<double>::infinity();
      int arg = 0;
      for (int q = 0; q < k; ++q) {
        double d = (c[q] - w[p]) * (c[q] - w[p]);
        if (d < best) { best = d; arg = q; }
      }
      stack[p] = arg;
      sum[arg] += w[p];
      cnt[arg] += 1;
    }
    double delta = 0.0;
    for (int q = 0; q < k; ++q) {
      double nc = cnt[q] > 0 ? sum[q] / static_cast<double>(cnt[q]) : 0.0;
      delta += std::fabs(nc - c[q]) / std::max(std::fabs(c[q]), eps);
      c[q] = nc;
    }
    delta /= k;
    if (delta < tol) break;
  }
  for (int q = 0; q < k; ++q) centre[q] = c[q];
  return t;
}

}  // extern "C"
