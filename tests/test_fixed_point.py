"""The fixed-point arithmetic of deterministic gridding (csrc/fixed_point.cuh)
compiled for the host and checked against its definition in exact rational
arithmetic: fixed_point(x, e) = x 2^e rounded to the nearest integer, ties
away from zero, for FP32 and FP64 x (normal, subnormal, zero, either sign,
exact ties); from_fixed(v) = v 2^-e, in FP64 correctly rounded, in FP32
within 2 ulp of v 2^-e; and sums of the integers independent of the order
of the additions, where FP32 sums of the same terms are not."""
import os
import subprocess
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_06555_gb300", "csrc")

CODE = r"""
#include <cstdio>
#include <cstdlib>
#include <cmath>
#define PHI_HD
#include "fixed_point.cuh"
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb"); FILE* g = fopen(argv[2], "wb");
  const int mode = atoi(argv[3]);
  int e;
  if (mode == 0) {          // float x, int e -> int64
    float x;
    while (fread(&x, 4, 1, f) == 1 && fread(&e, 4, 1, f) == 1) {
      long long v = phi::fixed_point(x, e); fwrite(&v, 8, 1, g);
    }
  } else if (mode == 1) {   // double x, int e -> int64
    double x;
    while (fread(&x, 8, 1, f) == 1 && fread(&e, 4, 1, f) == 1) {
      long long v = phi::fixed_point(x, e); fwrite(&v, 8, 1, g);
    }
  } else {                  // int64 v, int e -> float, double
    long long v;
    while (fread(&v, 8, 1, f) == 1 && fread(&e, 4, 1, f) == 1) {
      float a = phi::from_fixed(v, std::ldexp(1.0f, 32 - e), std::ldexp(1.0f, -e));
      double b = phi::from_fixed(v, std::ldexp(1.0, 32 - e), std::ldexp(1.0, -e));
      fwrite(&a, 4, 1, g); fwrite(&b, 8, 1, g);
    }
  }
  fclose(f); fclose(g);
  return 0;
}
"""


def run_host(mode, records, out_dtype):
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"phi_fx_{os.getpid()}")
    with open(tmp + ".cpp", "w") as f:
        f.write(CODE)
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-I", CSRC, tmp + ".cpp", "-o", tmp],
                   check=True)
    records.tofile(tmp + ".in")
    subprocess.run([tmp, tmp + ".in", tmp + ".out", str(mode)], check=True)
    out = np.fromfile(tmp + ".out", out_dtype)
    for ext in (".cpp", ".in", ".out", ""):
        os.remove(tmp + ext)
    return out


def exact_round(x, e):
    q = Fraction(float(x)) * Fraction(2) ** int(e)
    n = abs(q)
    r = int(n)                      # floor of the magnitude
    if n - r >= Fraction(1, 2):
        r += 1                      # ties away from zero
    return -r if q < 0 else r


def fixed_point(xs, es, double):
    dt = np.dtype([("x", np.float64 if double else np.float32), ("e", np.int32)])
    rec = np.zeros(len(xs), dt)
    rec["x"], rec["e"] = xs, es
    return run_host(1 if double else 0, rec, np.int64)


def test_fixed_point_is_round_half_away_of_x_times_2_to_e():
    rng = np.random.default_rng(5)
    for double in (False, True):
        ft = np.float64 if double else np.float32
        tiny = np.finfo(ft).tiny
        special = np.array([0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 1.5, -2.5, 3.0 * 2.0 ** -30,
                            tiny, -tiny, tiny / 8, -tiny / 3, 12345.678, -0.1], ft)
        xs = np.concatenate([special,
                             (rng.standard_normal(3000) * 10.0 ** rng.uniform(-8, 8, 3000)).astype(ft)])
        # exponents that keep |x| 2^e < 2^62, from coarse (most terms round
        # to 0 or 1) to fine (the whole significand kept)
        es = []
        for x in xs:
            top = 61 - (int(np.frexp(np.float64(x))[1]) if x != 0 else 0)
            es.append(int(rng.integers(top - 60, top + 1)))
        # subnormal inputs need very large e to keep bits: use the top one
        es = np.array(es, np.int32)
        sub = np.abs(xs) < tiny
        got = fixed_point(xs, es, double)
        want = [exact_round(x, e) for x, e in zip(xs, es)]
        assert [int(v) for v in got] == want
        assert sub.sum() >= 2


def test_exact_ties_round_away_from_zero():
    xs = np.array([0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 0.75, -0.75], np.float32)
    got = fixed_point(xs, np.zeros(len(xs), np.int32), False)
    assert list(got) == [1, -1, 2, -2, 3, -3, 1, -1]
    got = fixed_point(xs.astype(np.float64), np.ones(len(xs), np.int32), True)
    assert list(got) == [1, -1, 3, -3, 5, -5, 2, -2]


def test_from_fixed_recovers_the_value():
    rng = np.random.default_rng(7)
    vs = np.concatenate([np.array([0, 1, -1, 2 ** 32, -(2 ** 32), 2 ** 61 - 1, -(2 ** 61) + 1,
                                   2 ** 31, 2 ** 32 - 1, -(2 ** 31)], np.int64),
                         rng.integers(-(2 ** 61), 2 ** 61, 5000, dtype=np.int64),
                         rng.integers(-(2 ** 20), 2 ** 20, 2000, dtype=np.int64)])
    es = rng.integers(-60, 100, len(vs)).astype(np.int32)
    dt = np.dtype([("v", np.int64), ("e", np.int32)])
    rec = np.zeros(len(vs), dt)
    rec["v"], rec["e"] = vs, es
    out = run_host(2, rec, np.dtype([("f", np.float32), ("d", np.float64)]))
    for v, e, f, d in zip(vs, es, out["f"], out["d"]):
        exact = Fraction(int(v)) * Fraction(2) ** (-int(e))
        assert d == float(exact)                              # correctly rounded
        if v != 0:
            ulp = np.spacing(np.float32(abs(float(exact))))
            assert abs(Fraction(float(f)) - exact) <= 2 * Fraction(float(ulp))
        else:
            assert f == 0.0


def test_integer_sums_do_not_depend_on_the_order():
    """The property deterministic gridding relies on: the same terms added
    in two orders give the same integer sum, and hence the same float."""
    rng = np.random.default_rng(9)
    terms = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 2, 20000)).astype(np.float32)
    e = 61 - 15 - int(np.frexp(np.float64(np.abs(terms).max()))[1])   # 2^15 >= 20000 terms
    fx = fixed_point(terms, np.full(len(terms), e, np.int32), False)
    perm = rng.permutation(len(terms))
    s1 = sum(int(v) for v in fx)
    s2 = sum(int(fx[i]) for i in perm)
    assert s1 == s2
    exact = sum(Fraction(float(t)) for t in terms)
    assert abs(Fraction(s1) / Fraction(2) ** e - exact) <= Fraction(len(terms), 2) / Fraction(2) ** e
    # FP32 running sums of the same terms in the two orders differ
    f1 = np.float32(0)
    for t in terms:
        f1 = np.float32(f1 + t)
    f2 = np.float32(0)
    for i in perm:
        f2 = np.float32(f2 + terms[i])
    assert f1 != f2
