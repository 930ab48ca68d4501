// FP32 Bessel J0 for the w-kernel integrand, argument given in half-cycles:
// j0_halfcycles(u) = J0(pi u), u >= 0.
//
// Method: Abramowitz & Stegun (1964) 9.4.1 for pi u <= 3 (polynomial in
// (x/3)^2, |error| < 5e-8); for pi u > 3 the modulus/phase form
// J0 = M0 cos theta0 (A&S 9.2.17) with sqrt(u) M0 and the phase correction
// as degree-4 polynomials in 1/u^2 (the parities of their Hankel expansions,
// A&S 9.2.28-9.2.31), coefficients fitted by j0_fit.py in this directory
// (|error| < 5.2e-8); for u >= 2 the same form with both polynomials of
// degree 2 (|error| < 4.7e-8, two multiply-adds fewer per polynomial), and
// for u >= 4.5 of degree 1 (|error| < 4.9e-8).
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

// Lower end of the degree-2 form: x = pi u = 2 pi.
constexpr float kJ0Far = 2.0f;

// J0(pi u) for u >= kJ0Far: j0_large's form with F and D of degree 2 (the
// fit of j0_fit.py on [2, 1e5]; J0 error <= 3.9e-8 from F, 8.5e-9 from D).
PHI_HD inline float j0_far(float u) {
  const float r = j0_rsqrt(u);
  const float s = r * r;
  const float q = s * s;
  float f = 3.987198814e-04f;
  f = j0_fma(f, q, -2.842591913e-03f);
  f = j0_fma(f, q, 4.501579747e-01f);
  float d = -1.628429337e-04f;
  d = j0_fma(d, q, 6.617906817e-04f);
  d = j0_fma(d, q, -1.266492407e-02f);
  const float phi = j0_fma(d, s, u);
  return (r * f) * j0_cos(j0_fma(phi, 3.14159265358979f, -0.785398163397448f));
}

// Lower end of the degree-1 form: u = 4.5.
constexpr float kJ0Farthest = 4.5f;

// J0(pi u) for u >= kJ0Farthest: the same form with F and D of degree 1 (the
// fit of j0_fit.py on [4.5, 1e5]; J0 error <= 4.5e-8 from F, 3.6e-9 from D).
PHI_HD inline float j0_farthest(float u) {
  const float r = j0_rsqrt(u);
  const float s = r * r;
  const float q = s * s;
  const float f = j0_fma(-2.824241012e-03f, q, 4.501578963e-01f);
  const float d = j0_fma(6.546436681e-04f, q, -1.266495887e-02f);
  const float phi = j0_fma(d, s, u);
  return (r * f) * j0_cos(j0_fma(phi, 3.14159265358979f, -0.785398163397448f));
}

#if defined(__CUDACC__)
// Two arguments at once in Blackwell's paired FP32 arithmetic (f32x2 FMA
// and multiply, one instruction for both halves): the same operations, in
// the same order and rounding, as j0_small, j0_large, j0_far and
// j0_farthest on each half.
__device__ __forceinline__ float2 j0_pair(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ float2 j0_small2(float2 u) {
  const float2 z = __fmul2_rn(__fmul2_rn(u, u), j0_pair(1.096622711232151f, 1.096622711232151f));
  float2 p = j0_pair(0.0002100f, 0.0002100f);
  p = __ffma2_rn(p, z, j0_pair(-0.0039444f, -0.0039444f));
  p = __ffma2_rn(p, z, j0_pair(0.0444479f, 0.0444479f));
  p = __ffma2_rn(p, z, j0_pair(-0.3163866f, -0.3163866f));
  p = __ffma2_rn(p, z, j0_pair(1.2656208f, 1.2656208f));
  p = __ffma2_rn(p, z, j0_pair(-2.2499997f, -2.2499997f));
  return __ffma2_rn(p, z, j0_pair(1.0f, 1.0f));
}

__device__ __forceinline__ float2 j0_large2(float2 u) {
  const float2 r = j0_pair(j0_rsqrt(u.x), j0_rsqrt(u.y));
  const float2 s = __fmul2_rn(r, r);
  const float2 q = __fmul2_rn(s, s);
  float2 f = j0_pair(2.949163237e-05f, 2.949163237e-05f);
  f = __ffma2_rn(f, q, j0_pair(-1.386496738e-04f, -1.386496738e-04f));
  f = __ffma2_rn(f, q, j0_pair(4.440745370e-04f, 4.440745370e-04f));
  f = __ffma2_rn(f, q, j0_pair(-2.846068740e-03f, -2.846068740e-03f));
  f = __ffma2_rn(f, q, j0_pair(4.501580035e-01f, 4.501580035e-01f));
  float2 d = j0_pair(-1.531106734e-05f, -1.531106734e-05f);
  d = __ffma2_rn(d, q, j0_pair(6.988119170e-05f, 6.988119170e-05f));
  d = __ffma2_rn(d, q, j0_pair(-1.853455306e-04f, -1.853455306e-04f));
  d = __ffma2_rn(d, q, j0_pair(6.629692300e-04f, 6.629692300e-04f));
  d = __ffma2_rn(d, q, j0_pair(-1.266485270e-02f, -1.266485270e-02f));
  const float2 phi = __ffma2_rn(d, s, u);
  const float2 th = __ffma2_rn(phi, j0_pair(3.14159265358979f, 3.14159265358979f),
                               j0_pair(-0.785398163397448f, -0.785398163397448f));
  return __fmul2_rn(__fmul2_rn(r, f), j0_pair(j0_cos(th.x), j0_cos(th.y)));
}

__device__ __forceinline__ float2 j0_farthest2(float2 u) {
  const float2 r = j0_pair(j0_rsqrt(u.x), j0_rsqrt(u.y));
  const float2 s = __fmul2_rn(r, r);
  const float2 q = __fmul2_rn(s, s);
  const float2 f = __ffma2_rn(j0_pair(-2.824241012e-03f, -2.824241012e-03f), q,
                              j0_pair(4.501578963e-01f, 4.501578963e-01f));
  const float2 d = __ffma2_rn(j0_pair(6.546436681e-04f, 6.546436681e-04f), q,
                              j0_pair(-1.266495887e-02f, -1.266495887e-02f));
  const float2 phi = __ffma2_rn(d, s, u);
  const float2 th = __ffma2_rn(phi, j0_pair(3.14159265358979f, 3.14159265358979f),
                               j0_pair(-0.785398163397448f, -0.785398163397448f));
  return __fmul2_rn(__fmul2_rn(r, f), j0_pair(j0_cos(th.x), j0_cos(th.y)));
}

__device__ __forceinline__ float2 j0_far2(float2 u) {
  const float2 r = j0_pair(j0_rsqrt(u.x), j0_rsqrt(u.y));
  const float2 s = __fmul2_rn(r, r);
  const float2 q = __fmul2_rn(s, s);
  float2 f = j0_pair(3.987198814e-04f, 3.987198814e-04f);
  f = __ffma2_rn(f, q, j0_pair(-2.842591913e-03f, -2.842591913e-03f));
  f = __ffma2_rn(f, q, j0_pair(4.501579747e-01f, 4.501579747e-01f));
  float2 d = j0_pair(-1.628429337e-04f, -1.628429337e-04f);
  d = __ffma2_rn(d, q, j0_pair(6.617906817e-04f, 6.617906817e-04f));
  d = __ffma2_rn(d, q, j0_pair(-1.266492407e-02f, -1.266492407e-02f));
  const float2 phi = __ffma2_rn(d, s, u);
  const float2 th = __ffma2_rn(phi, j0_pair(3.14159265358979f, 3.14159265358979f),
                               j0_pair(-0.785398163397448f, -0.785398163397448f));
  return __fmul2_rn(__fmul2_rn(r, f), j0_pair(j0_cos(th.x), j0_cos(th.y)));
}
#endif

}  // namespace phi
