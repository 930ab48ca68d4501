"""Nodes and weights of the Gauss-Kronrod (15, 31) rule used by the device
quadrature (phi_ops.cu), computed from the rule's definition.

The Kronrod extension of the n-point Gauss-Legendre rule adds the n + 1
zeros of the Stieltjes polynomial E_{n+1}, the polynomial of degree n + 1
orthogonal on [-1, 1] to every polynomial of degree <= n with respect to the
weight P_n(x) (Kronrod 1965).  The 2n + 1 point rule then integrates every
polynomial of degree <= 3n + 1 exactly, which fixes its weights; the Gauss
weights are those of the n-point rule alone.

E_{n+1} is found in exact rational arithmetic (its coefficients in the
Legendre basis solve a linear system of integrals of Legendre polynomials),
its zeros and the Legendre zeros to 60 digits, and the weights from the
moment equations at the same precision.  Run it to print the constants
(node x_j in [-1, 1] ascending, Kronrod weight, Gauss weight or 0):

    python gk_rule.py [n]        # default n = 15
"""
import sys

import mpmath as mp
import sympy as sy

mp.mp.dps = 60


def rule(n):
    x = sy.Symbol("x")
    pn = sy.legendre(n, x)
    basis = [sy.legendre(k, x) for k in range(n + 2)]
    # E = sum_k e_k P_k with e_{n+1} = 1 and int_{-1}^{1} P_n E x^j dx = 0, j <= n
    mom = [[sy.integrate(pn * b * x ** j, (x, -1, 1)) for b in basis] for j in range(n + 1)]
    a = sy.Matrix([row[:n + 1] for row in mom])
    rhs = sy.Matrix([-row[n + 1] for row in mom])
    e = list(a.LUsolve(rhs)) + [sy.Integer(1)]
    stieltjes = sy.Poly(sum(c * b for c, b in zip(e, basis)), x)
    legendre = sy.Poly(pn, x)

    def zeros(poly):
        coeffs = [mp.mpf(sy.Rational(c).p) / mp.mpf(sy.Rational(c).q) for c in poly.all_coeffs()]
        r = mp.polyroots(coeffs, maxsteps=400, extraprec=400)
        return sorted(mp.re(z) for z in r)

    xg = zeros(legendre)
    xk = zeros(stieltjes)
    nodes = sorted(xg + xk)
    m = len(nodes)
    # weights: exact for x^0 .. x^(2n): moments 2/(k+1) for even k, 0 for odd
    v = mp.matrix([[t ** k for t in nodes] for k in range(m)])
    b = mp.matrix([mp.mpf(2) / (k + 1) if k % 2 == 0 else 0 for k in range(m)])
    wk = mp.lu_solve(v, b)
    vg = mp.matrix([[t ** k for t in xg] for k in range(n)])
    bg = mp.matrix([mp.mpf(2) / (k + 1) if k % 2 == 0 else 0 for k in range(n)])
    wg_gauss = mp.lu_solve(vg, bg)
    wg = []
    for t in nodes:
        i = min(range(n), key=lambda j: abs(xg[j] - t))
        wg.append(wg_gauss[i] if abs(xg[i] - t) < mp.mpf(10) ** -40 else mp.mpf(0))
    return nodes, [wk[i] for i in range(m)], wg


def check(nodes, wk, wg, n):
    """Exactness: the Kronrod rule to degree 3n + 1, the Gauss rule to 2n - 1."""
    worst_k = max(abs(sum(w * t ** k for t, w in zip(nodes, wk)) -
                      (mp.mpf(2) / (k + 1) if k % 2 == 0 else 0)) for k in range(3 * n + 2))
    worst_g = max(abs(sum(w * t ** k for t, w in zip(nodes, wg)) -
                      (mp.mpf(2) / (k + 1) if k % 2 == 0 else 0)) for k in range(2 * n))
    return worst_k, worst_g


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 15
    nodes, wk, wg = rule(n)
    ek, eg = check(nodes, wk, wg, n)
    print(f"// G{n}/K{2 * n + 1}: exactness error {mp.nstr(ek, 3)} (Kronrod, degree {3 * n + 1}), "
          f"{mp.nstr(eg, 3)} (Gauss, degree {2 * n - 1})")
    for t, a, g in zip(nodes, wk, wg):
        print(f"{mp.nstr(t, 36, min_fixed=-1, max_fixed=1)}, {mp.nstr(a, 36)}, {mp.nstr(g, 36)}")
