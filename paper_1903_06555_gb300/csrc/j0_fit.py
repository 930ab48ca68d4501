"""Coefficients of the asymptotic-form FP32 J0 in bessel_j0.cuh.

For x = pi u >= 3, J0(x) = M0(x) cos(theta0(x)) with the modulus M0 and phase
theta0 of Abramowitz & Stegun 9.2.17 (J0 = M0 cos theta0, Y0 = M0 sin theta0).
Their Hankel expansions (A&S 9.2.28-9.2.31) make sqrt(u) M0 an even function
of 1/u and u (theta0 - x + pi/4) / pi an odd one, so both are written as
polynomials in q = 1/u^2:

    J0(pi u) = u^{-1/2} F(q) cos(pi (u + D(q) / u) - pi/4),

F and D of degree 4 in q for u >= 3/pi, of degree 2 for u >= 2 (x >= 2 pi)
and of degree 1 for u >= 4.5, where the Hankel series converge fast enough
that the lower degrees keep the same accuracy.  The coefficients minimise the largest absolute error of J0
this form gives (the L-infinity fit, solved as a linear program on a dense
grid of u in [u_min, 1e5]), separately for the modulus and the phase part,
against scipy's j0 and y0.  Run it to print the constants of both fits.
"""
import numpy as np
import scipy.optimize as so
import scipy.special as sp

U_MIN = 3.0 / np.pi
DEGREE = 4
U_MIN_FAR = 2.0
DEGREE_FAR = 2
U_MIN_FARTHEST = 4.5
DEGREE_FARTHEST = 1


def modulus_and_phase(u):
    """F(q) = sqrt(u) M0 and D(q) = u (theta0 - x + pi/4) / pi at x = pi u."""
    x = np.pi * u
    j, y = sp.j0(x), sp.y0(x)
    m = np.hypot(j, y)
    corr = (np.arctan2(y, j) - (x - np.pi / 4) + np.pi) % (2 * np.pi) - np.pi
    return m * np.sqrt(u), corr / np.pi * u


def linf_fit(a, y, w, scale=1e8):
    """min_c max_i w_i |(a c - y)_i| as a linear program in (c, t); the
    weighted residuals are multiplied by `scale` so that the solver's
    absolute tolerances lie far below the errors being balanced."""
    n, k = a.shape
    aw = a * (w * scale)[:, None]
    yw = y * w * scale
    obj = np.zeros(k + 1)
    obj[-1] = 1.0
    ones = -np.ones((n, 1))
    a_ub = np.vstack([np.hstack([aw, ones]), np.hstack([-aw, ones])])
    b_ub = np.concatenate([yw, -yw])
    res = so.linprog(obj, A_ub=a_ub, b_ub=b_ub, bounds=[(None, None)] * (k + 1),
                     method="highs")
    assert res.success, res.message
    return res.x[:k]


def fit(n=20000, u_min=U_MIN, degree=DEGREE):
    u = np.geomspace(u_min, 1e5, n)
    q = 1.0 / u ** 2
    qmax = 1.0 / u_min ** 2
    f, d = modulus_and_phase(u)
    r = 1.0 / np.sqrt(u)
    # columns in the normalised variable q / qmax, so all lie in [0, 1]
    a = np.vander(q / qmax, degree + 1, increasing=True)
    back = qmax ** -np.arange(degree + 1)
    # J0 error: r * (F error) from the modulus, (F r) (pi / u) * (D error) from the phase
    cf = linf_fit(a, f, r) * back
    cd = linf_fit(a, d, f * r * np.pi / u) * back
    return cf, cd


def max_errors(cf, cd, n=300001, u_min=U_MIN):
    """Largest J0 error of each part on a grid 15x denser than the fit's."""
    u = np.geomspace(u_min, 1e5, n)
    q = 1.0 / u ** 2
    f, d = modulus_and_phase(u)
    r = 1.0 / np.sqrt(u)
    a = np.vander(q, len(cf), increasing=True)
    return (np.max(r * np.abs(a @ cf - f)), np.max(f * r * np.pi / u * np.abs(a @ cd - d)))


if __name__ == "__main__":
    for u_min, degree in ((U_MIN, DEGREE), (U_MIN_FAR, DEGREE_FAR),
                          (U_MIN_FARTHEST, DEGREE_FARTHEST)):
        cf, cd = fit(u_min=u_min, degree=degree)
        ef, ed = max_errors(cf, cd, u_min=u_min)
        print(f"// u >= {u_min:.6f}, degree {degree}: max |J0 error| from the modulus "
              f"{ef:.2e}, from the phase {ed:.2e}")
        print("F:", ", ".join(f"{c:.9e}f" for c in cf))
        print("D:", ", ".join(f"{c:.9e}f" for c in cd))
