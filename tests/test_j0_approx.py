"""The device FP32 J0 (csrc/bessel_j0.cuh: Abramowitz & Stegun 9.4.1 below x = 3,
the modulus/phase form above, of degree 4 and, from x = 2 pi, of degree 2)
compiled for the host and checked against scipy."""
import os
import subprocess

import numpy as np
import scipy.special as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_06555_gb300", "csrc")


def host_j0(u, fn="j0_halfcycles"):
    code = r"""
#include <cmath>
#include <cstdio>
#include <cstdlib>
#define PHI_HD
#include <math.h>
#include "bessel_j0.cuh"
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb"); FILE* g = fopen(argv[2], "wb");
  float u;
  while (fread(&u, 4, 1, f) == 1) { float j = phi::FN(u); fwrite(&j, 4, 1, g); }
  fclose(f); fclose(g);
  return 0;
}
"""
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"phi_j0_{os.getpid()}")
    with open(tmp + ".cpp", "w") as f:
        f.write(code)
    subprocess.run(["g++", "-O2", "-ffp-contract=off", f"-DFN={fn}", "-I", CSRC, tmp + ".cpp",
                    "-o", tmp], check=True)
    np.asarray(u, np.float32).tofile(tmp + ".in")
    subprocess.run([tmp, tmp + ".in", tmp + ".out"], check=True)
    out = np.fromfile(tmp + ".out", np.float32)
    for ext in (".cpp", ".in", ".out", ""):
        os.remove(tmp + ext)
    return out


def test_j0_halfcycles_against_scipy():
    u = np.concatenate([np.linspace(0, 1.2, 4001), np.linspace(1.2, 60, 60001)]).astype(np.float32)
    got = host_j0(u).astype(np.float64)
    ref = sp.j0(np.pi * u.astype(np.float64))
    err = np.abs(got - ref)
    # 9.4.1 itself is good to 5e-8; FP32 rounding of its alternating terms
    # (up to 2.25 near x = 3) adds a few 1e-7
    assert err[np.pi * u <= 3].max() < 3.5e-7
    # beyond x = 3 the FP32 rounding of the half-cycle argument u dominates:
    # |dJ0| <~ pi ulp(u) sqrt(2 / (pi x)) plus the formula's 1e-7
    env = np.sqrt(2.0 / (np.pi * np.pi * np.maximum(u, 1e-3)))
    ulp = np.spacing(np.maximum(u, 1.0).astype(np.float32)).astype(np.float64)
    big = np.pi * u > 3
    assert np.all(err[big] <= 2e-7 + 2 * env[big] * np.pi * ulp[big])
    # rms: the formula's 1e-7 and the rounding of u (to ulp(u)/2, scaled by
    # pi) and of the phase theta0 (to ulp(theta0)/2), each uniform
    th = np.spacing(np.maximum(np.pi * u, 1.0).astype(np.float32)).astype(np.float64)
    rounding = env * np.sqrt((np.pi * ulp) ** 2 + th ** 2) / np.sqrt(24.0)
    assert np.sqrt(np.mean(err ** 2)) < 1.25 * np.hypot(1e-7, np.sqrt(np.mean(rounding ** 2)))


def test_j0_far_against_scipy():
    """The degree-2 form used for panels whose nodes all lie at u >= 2
    (x >= 2 pi): the same bounds as the degree-4 form beyond x = 3."""
    u = np.concatenate([np.linspace(2.0, 10.0, 40001), np.linspace(10.0, 130.0, 60001)]
                       ).astype(np.float32)
    got = host_j0(u, "j0_far").astype(np.float64)
    ref = sp.j0(np.pi * u.astype(np.float64))
    err = np.abs(got - ref)
    env = np.sqrt(2.0 / (np.pi * np.pi * u))
    ulp = np.spacing(u).astype(np.float64)
    assert np.all(err <= 2e-7 + 2 * env * np.pi * ulp)
    # and it agrees with the degree-4 form to the two fits' errors plus rounding
    near = host_j0(u, "j0_large").astype(np.float64)
    assert np.max(np.abs(near - got)) < 2e-7 + 4 * np.max(env * np.pi * ulp)


def test_j0_farthest_against_scipy():
    """The degree-1 form used for panels whose nodes all lie at u >= 4.5."""
    u = np.concatenate([np.linspace(4.5, 12.0, 40001), np.linspace(12.0, 130.0, 60001)]
                       ).astype(np.float32)
    got = host_j0(u, "j0_farthest").astype(np.float64)
    ref = sp.j0(np.pi * u.astype(np.float64))
    env = np.sqrt(2.0 / (np.pi * np.pi * u))
    ulp = np.spacing(u).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2e-7 + 2 * env * np.pi * ulp)
