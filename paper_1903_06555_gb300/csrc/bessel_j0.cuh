// FP32 Bessel J0 for the w-kernel integrand, argument given in half-cycles:
// j0_halfcycles(u) = J0(pi u), u >= 0.
//
// Method: Abramowitz & Stegun (1964), 9.4.1 for pi u <= 3 (polynomial in
// (x/3)^2, |error| < 5e-8) and 9.4.3 for pi u >= 3 (J0 = x^{-1/2} f0 cos theta0
// with f0 and theta0 polynomials in 3/x, |error| < 1.6e-8 and 7e-8 rad).
// The cosine is taken in half-cycles, cos(theta0) = cos(pi phi) with
// phi = u - 1/4 + (theta0 - x + pi/4)/pi, reduced exactly to f = phi - n,
// |f| <= 1/2, and evaluated with the Taylor series of cos(pi f) to degree 12
// (truncation < 1e-8), so the whole evaluation costs one reciprocal square
// root and ~25 FMA-pipe operations; the argument never needs a large-argument
// trigonometric reduction.  Polynomials in s = 1/x absorb the factors 3^k.
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

PHI_HD inline float j0_rsqrt(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}

PHI_HD inline float j0_halfcycles(float u) {
  const float kPiF32 = 3.14159265358979f;
  const float x = kPiF32 * u;
  if (x <= 3.0f) {
    // 9.4.1 in z = (x/3)^2
    const float z = x * x * (1.0f / 9.0f);
    float p = 0.0002100f;
    p = j0_fma(p, z, -0.0039444f);
    p = j0_fma(p, z, 0.0444479f);
    p = j0_fma(p, z, -0.3163866f);
    p = j0_fma(p, z, 1.2656208f);
    p = j0_fma(p, z, -2.2499997f);
    return j0_fma(p, z, 1.0f);
  }
  // 9.4.3 with t = 3/x = 3 s, s = 1/x
  const float r = j0_rsqrt(x);
  const float s = r * r;
  // f0 = sum a_k t^k  ->  sum (a_k 3^k) s^k
  float f0 = 0.00014476f * 729.0f;
  f0 = j0_fma(f0, s, -0.00072805f * 243.0f);
  f0 = j0_fma(f0, s, 0.00137237f * 81.0f);
  f0 = j0_fma(f0, s, -0.00009512f * 27.0f);
  f0 = j0_fma(f0, s, -0.00552740f * 9.0f);
  f0 = j0_fma(f0, s, -0.00000077f * 3.0f);
  f0 = j0_fma(f0, s, 0.79788456f);
  // (theta0 - x + pi/4) / pi = sum b_k t^k / pi, k >= 1
  const float ip = 0.318309886183791f;
  float d = 0.00013558f * 729.0f * ip;
  d = j0_fma(d, s, -0.00029333f * 243.0f * ip);
  d = j0_fma(d, s, -0.00054125f * 81.0f * ip);
  d = j0_fma(d, s, 0.00262573f * 27.0f * ip);
  d = j0_fma(d, s, -0.00003954f * 9.0f * ip);
  d = j0_fma(d, s, -0.04166397f * 3.0f * ip);
  const float phi = (u - 0.25f) + d * s;
  const float n = rintf(phi);
  const float f = phi - n;
  const float f2 = f * f;
  // cos(pi f), |f| <= 1/2: Taylor coefficients (-1)^k pi^{2k} / (2k)!
  float c = 0.001929574309403923f;
  c = j0_fma(c, f2, -0.02580689139001406f);
  c = j0_fma(c, f2, 0.2353306303588932f);
  c = j0_fma(c, f2, -1.335262768854589f);
  c = j0_fma(c, f2, 4.058712126416768f);
  c = j0_fma(c, f2, -4.934802200544679f);
  c = j0_fma(c, f2, 1.0f);
  // cos(pi phi) = (-1)^n cos(pi f)
  const float sgn = (static_cast<int>(n) & 1) ? -1.0f : 1.0f;
  return (r * f0) * (c * sgn);
}

}  // namespace phi
