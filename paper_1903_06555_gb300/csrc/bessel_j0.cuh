// FP32 Bessel J0 for the w-kernel integrand, argument given in half-cycles:
// j0_halfcycles(u) = J0(pi u), u >= 0.
//
// Method: Abramowitz & Stegun (1964), 9.4.1 for pi u <= 3 (polynomial in
// (x/3)^2, |error| < 5e-8) and 9.4.3 for pi u >= 3 (J0 = x^{-1/2} f0 cos theta0
// with f0 and theta0 polynomials in 3/x, |error| < 1.6e-8 and 7e-8 rad).
// The phase theta0 = pi (u + sum_k b_k t^k / pi) - pi/4 is formed in FP32 and
// handed to the hardware cosine, which reduces it by whole turns itself.  The
// argument's own FP32 rounding (relative 6e-8, i.e. 6e-6 rad at 100 rad, the
// largest phase a 64-tap support reaches) dominates that reduction's error, so
// an explicit reduction in half-cycles buys no accuracy; dropping it saves ~5
// of ~30 instructions per evaluation.  The whole evaluation costs a
// reciprocal square root, a cosine and ~20 FMA-pipe operations.
// Polynomials in s = 1/u absorb the factors (3/pi)^k, 1/pi and 1/sqrt(pi).
#pragma once

#ifndef PHI_HD
#define PHI_HD __host__ __device__
#endif

namespace phi {

PHI_HD inline float j0_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// Device: the hardware approximations with subnormals flushed (PTX .ftz):
// the asymptotic branch only sees u >= 0.95, so no subnormal input occurs,
// and the flush spares the subnormal handling around the hardware op.
PHI_HD inline float j0_rsqrt(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / sqrtf(x);
#endif
}

// cos: the hardware approximation on the device (absolute error ~5e-7 on
// [-pi, pi], growing with |a| like the FP32 rounding of a), libm on the host.
PHI_HD inline float j0_cos(float a) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
  return y;
#else
  return cosf(a);
#endif
}

// Argument split between the two formulas: x = pi u = 3.
constexpr float kJ0Split = 0.954929658551372f;

// J0(pi u) for u <= kJ0Split (A&S 9.4.1).
PHI_HD inline float j0_small(float u) {
  // 9.4.1 in z = (x/3)^2 = u^2 pi^2 / 9
  const float z = (u * u) * 1.096622711232151f;
  float p = 0.0002100f;
  p = j0_fma(p, z, -0.0039444f);
  p = j0_fma(p, z, 0.0444479f);
  p = j0_fma(p, z, -0.3163866f);
  p = j0_fma(p, z, 1.2656208f);
  p = j0_fma(p, z, -2.2499997f);
  return j0_fma(p, z, 1.0f);
}

// J0(pi u) for u > kJ0Split (A&S 9.4.3).
PHI_HD inline float j0_large(float u) {
  // 9.4.3 with t = 3/x, x = pi u.  With r = u^{-1/2} and s = r^2 = 1/u:
  // x^{-1/2} = r / sqrt(pi), t^k = (3/pi)^k s^k; both factors are folded
  // into the coefficients below.
  const float r = j0_rsqrt(u);
  const float s = r * r;
  const float c1 = 0.954929658551372f;  // 3 / pi
  const float c2 = c1 * c1, c3 = c2 * c1, c4 = c3 * c1, c5 = c4 * c1, c6 = c5 * c1;
  const float isp = 0.564189583547756f;  // 1 / sqrt(pi)
  float f0 = 0.00014476f * c6 * isp;
  f0 = j0_fma(f0, s, -0.00072805f * c5 * isp);
  f0 = j0_fma(f0, s, 0.00137237f * c4 * isp);
  f0 = j0_fma(f0, s, -0.00009512f * c3 * isp);
  f0 = j0_fma(f0, s, -0.00552740f * c2 * isp);
  f0 = j0_fma(f0, s, -0.00000077f * c1 * isp);
  f0 = j0_fma(f0, s, 0.79788456f * isp);
  // (theta0 - x + pi/4) / pi = sum_k b_k t^k / pi, k >= 1
  const float ip = 0.318309886183791f;
  float d = 0.00013558f * c6 * ip;
  d = j0_fma(d, s, -0.00029333f * c5 * ip);
  d = j0_fma(d, s, -0.00054125f * c4 * ip);
  d = j0_fma(d, s, 0.00262573f * c3 * ip);
  d = j0_fma(d, s, -0.00003954f * c2 * ip);
  d = j0_fma(d, s, -0.04166397f * c1 * ip);
  // theta0 = pi (u + sum_k b_k t^k / pi) - pi/4, reduced by the cosine itself
  const float phi = j0_fma(d, s, u);
  return (r * f0) * j0_cos(j0_fma(phi, 3.14159265358979f, -0.785398163397448f));
}

PHI_HD inline float j0_halfcycles(float u) {
  return u <= kJ0Split ? j0_small(u) : j0_large(u);
}

}  // namespace phi
