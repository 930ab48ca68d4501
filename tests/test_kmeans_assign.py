"""The two pieces of an Algorithm 1 sweep that decide its result
(csrc/kmeans_assign.cuh), compiled for the host and checked against their
definitions: the nearest centre is argmin_q (wbar_q - w)^2 in FP64 with the
lowest q winning ties, whatever the FP32 pre-selection decides, also on
duplicated centres, empty-stack centres at 0, points on and around the
midpoints between centres and centres 1 ulp apart; the fixed-point sums
are the exact integer sums of w 2^S truncated toward zero, and the centre
formed from them lies within 2^-S of the exact mean of the members."""
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_06555_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#define PHI_HD
#include "kmeans_assign.cuh"
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb"); FILE* g = fopen(argv[2], "wb");
  int mode, k; long long n;
  if (fread(&mode, 4, 1, f) != 1 || fread(&k, 4, 1, f) != 1 || fread(&n, 8, 1, f) != 1) return 1;
  if (mode == 0) {   // nearest centre of n values among k centres
    std::vector<double> c(k); std::vector<float> cf(k), ce(k);
    if (fread(c.data(), 8, k, f) != (size_t)k) return 1;
    for (int q = 0; q < k; ++q) { cf[q] = (float)c[q]; ce[q] = phi::km_centre_err(cf[q]); }
    for (long long i = 0; i < n; ++i) {
      double w; if (fread(&w, 8, 1, f) != 1) return 1;
      int s = phi::nearest_centre(w, c.data(), cf.data(), ce.data(), k);
      fwrite(&s, 4, 1, g);
    }
  } else {           // fixed-point images, limb sums and total at scale 2^-k
    unsigned long long sum[phi::kLimbs] = {0};
    for (long long i = 0; i < n; ++i) {
      double w; if (fread(&w, 8, 1, f) != 1) return 1;
      long long v = phi::w_fixed(w, k);
      fwrite(&v, 8, 1, g);
      for (int l = 0; l < phi::kLimbs; ++l) sum[l] += phi::w_limb(v, l);
    }
    double t = phi::fixed_total(sum, k);
    fwrite(&t, 8, 1, g);
  }
  fclose(f); fclose(g);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("kmeans_assign")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    return d, exe


def run(harness, mode, k, payload):
    d, exe = harness
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        np.array([mode, k], np.int32).tofile(f)
        np.array([payload[-1].size], np.int64).tofile(f)
        for p in payload:
            np.asarray(p, np.float64).tofile(f)
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    return np.fromfile(out, np.uint8)


def scan(c, w):
    """Algorithm 1's assignment, written out: FP64 squared distances, first
    minimum."""
    d = (c[None, :] - w[:, None]) * (c[None, :] - w[:, None])
    return np.argmin(d, axis=1)


def adversarial(c, rng, n):
    """Points on, and a few ulps around, every midpoint and every centre, and
    random points over the centres' span."""
    cs = np.sort(c)
    mids = 0.5 * (cs[1:] + cs[:-1])
    pts = [rng.uniform(cs[0] - 1, cs[-1] + 1, n)]
    for m in np.concatenate([mids, cs]):
        pts.append(m + np.arange(-4, 5) * np.spacing(m))
        pts.append(np.nextafter(np.full(3, m), np.array([-np.inf, np.inf, m])))
    return np.concatenate(pts)


@pytest.mark.parametrize("case", ["spread", "duplicates", "empty_at_zero", "one_ulp", "large",
                                  "tiny", "many"])
def test_nearest_centre_is_the_fp64_scan(harness, case):
    rng = np.random.default_rng(hash(case) % 2**32)
    if case == "spread":
        c = np.sort(rng.uniform(0, 400, 8))
    elif case == "duplicates":
        c = np.array([10.0, 20.0, 20.0, 35.5, 35.5, 35.5, 60.0, 61.0])
    elif case == "empty_at_zero":
        c = np.array([3.0, 0.0, 17.25, 0.0, 90.0, 44.0, 0.0, 120.5])
    elif case == "one_ulp":
        b = 1234.5678
        c = np.array([b, np.nextafter(b, np.inf), np.nextafter(np.nextafter(b, np.inf), np.inf),
                      b + 1e-9, b - 3e-13, 2 * b, -b, 0.5 * b])
    elif case == "large":
        c = np.sort(rng.uniform(-1e7, 1e7, 16))
    elif case == "tiny":
        c = np.sort(rng.uniform(-1e-3, 1e-3, 8))
    else:
        c = np.sort(rng.uniform(0, 3000, 126))
    w = adversarial(c, rng, 20_000)
    got = run(harness, 0, c.size, [c, w]).view(np.int32)
    np.testing.assert_array_equal(got, scan(c, w))


def exact_fixed(w, S):
    """w 2^S truncated toward zero, in Python integers."""
    out = []
    for x in w:
        f = Fraction(float(x)) * (Fraction(2) ** S)
        q = abs(f.numerator) // f.denominator
        out.append(q if f >= 0 else -q)
    return out


@pytest.mark.parametrize("span", [(0.0, 380.0), (-1500.0, 1500.0), (-3e-3, 1e-3), (0.0, 0.0),
                                  (-7.0, -6.9)])
def test_fixed_point_sums_are_exact(harness, span):
    rng = np.random.default_rng(7)
    w = rng.uniform(span[0], span[1], 3000)
    w[:3] = [span[0], span[1], 0.0]
    wabs = np.max(np.abs(w))
    S = 62 - (int(np.frexp(wabs)[1]) if wabs > 0 else 0)     # as the plan chooses it
    raw = run(harness, 1, S, [w])
    v = raw[:-8].view(np.int64)
    total = raw[-8:].view(np.float64)[0]
    ref = exact_fixed(w, S)
    assert [int(t) for t in v] == ref
    assert all(abs(t) < 2**62 for t in ref)
    exact_sum = Fraction(sum(ref)) / (Fraction(2) ** S)
    # two roundings in the conversion to double, each within half an ulp
    assert abs(Fraction(total) - exact_sum) <= abs(exact_sum) * Fraction(1, 2**51) + Fraction(1, 2**1074)
    # the centre is within 2^-S of the exact mean of the members
    mean_exact = sum(Fraction(float(x)) for x in w) / len(w)
    assert abs(Fraction(total) / len(w) - mean_exact) <= Fraction(1, 2**S) + abs(mean_exact) * Fraction(1, 2**50)
