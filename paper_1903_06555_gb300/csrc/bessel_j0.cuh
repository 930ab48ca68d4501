// FP32 Bessel J0 for the w-kernel integrand, argument given in half-cycles:
// j0_halfcycles(u) = J0(pi u), u >= 0.
//
// Method: Abramowitz & Stegun (1964) 9.4.1 for pi u <= 3 (polynomial in
// (x/3)^2, |error| < 5e-8); for pi u > 3 the modulus/phase form
// J0 = M0 cos theta0 (A&S 9.2.17) with sqrt(u) M0 and the phase correction
// as degree-4 polynomials in 1/u^2 (the parities of their Hankel expansions,
// A&S 9.2.28-9.2.31), coefficients fitted by j0_fit.py in this directory
// (|error| < 5.2e-8).
// The phase theta0 = pi (u + D/u) - pi/4 is formed in FP32 and handed to the
// hardware cosine, which reduces it by whole turns itself.  The argument's own
// FP32 rounding (relative 6e-8, i.e. 6e-6 rad at 100 rad, the largest phase a
// 64-tap support reaches) dominates that reduction's error, so an explicit
// reduction buys no accuracy.  The large-argument evaluation costs a
// reciprocal square root, a cosine and ~15 FMA-pipe operations.
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

// J0(pi u) for u > kJ0Split: u^{-1/2} F(q) cos(pi (u + D(q)/u) - pi/4), q = 1/u^2,
// the modulus/phase form of A&S 9.2.17 with F and D the degree-4 L-infinity
// fits that j0_fit.py computes (J0 error <= 3.6e-8 from F, 1.6e-8 from D).
PHI_HD inline float j0_large(float u) {
  const float r = j0_rsqrt(u);
  const float s = r * r;   // 1 / u
  const float q = s * s;   // 1 / u^2
  float f = 2.949163237e-05f;
  f = j0_fma(f, q, -1.386496738e-04f);
  f = j0_fma(f, q, 4.440745370e-04f);
  f = j0_fma(f, q, -2.846068740e-03f);
  f = j0_fma(f, q, 4.501580035e-01f);
  float d = -1.531106734e-05f;
  d = j0_fma(d, q, 6.988119170e-05f);
  d = j0_fma(d, q, -1.853455306e-04f);
  d = j0_fma(d, q, 6.629692300e-04f);
  d = j0_fma(d, q, -1.266485270e-02f);
  // theta0 = pi (u + D / u) - pi/4, reduced by the cosine itself
  const float phi = j0_fma(d, s, u);
  return (r * f) * j0_cos(j0_fma(phi, 3.14159265358979f, -0.785398163397448f));
}

PHI_HD inline float j0_halfcycles(float u) {
  return u <= kJ0Split ? j0_small(u) : j0_large(u);
}

}  // namespace phi
