// Fixed-point arithmetic of deterministic gridding (plan field
// grid_deterministic = 1).  Each gridding contribution x becomes the integer
// x 2^e rounded to nearest, ties away from zero, read off the IEEE-754
// fields of x (sign, biased exponent, significand m with x = m 2^sh); the
// cell sums are then 64-bit integer additions, exact and associative, so
// the order in which the atomics land cannot change them.  The caller
// chooses e so that every |partial sum| 2^e < 2^62.
//
// Back to floating point, the magnitude of a sum, |v| = hi 2^32 + lo (hi and
// lo its top and bottom 32 bits), is hi 2^(32 - e) + lo 2^-e, and the sign
// is applied last: both parts are non-negative, so nothing cancels.  In FP64
// both products are exact and the fused add rounds once; in FP32 each part
// is rounded once before the fused add (within 2 ulp).  Either way the
// result is a function of the sum alone.  Host-compilable.
#pragma once

#ifndef PHI_HD
#define PHI_HD __host__ __device__
#endif

#include <stdint.h>
#if !defined(__CUDA_ARCH__)
#include <cmath>
#include <cstring>
#endif

namespace phi {

PHI_HD inline uint32_t fixed_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

PHI_HD inline uint64_t fixed_bits(double x) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

// m 2^sh rounded to the nearest integer, ties away from zero (m < 2^53,
// sh < 63 - 53 by the caller's choice of e).
PHI_HD inline uint64_t fixed_scale(uint64_t m, int sh) {
  if (sh >= 0) return m << (sh < 63 ? sh : 63);
  const int r = -sh < 63 ? -sh : 63;
  return (m + ((uint64_t(1) << r) >> 1)) >> r;
}

PHI_HD inline long long fixed_point(float x, int e) {
  const uint32_t b = fixed_bits(x);
  const int be = static_cast<int>((b >> 23) & 0xffu);
  const uint64_t m = be ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
  const uint64_t mag = fixed_scale(m, (be > 1 ? be : 1) - 150 + e);
  return (b >> 31) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

PHI_HD inline long long fixed_point(double x, int e) {
  const uint64_t b = fixed_bits(x);
  const int be = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t frac = b & 0xfffffffffffffull;
  const uint64_t m = be ? (frac | (uint64_t(1) << 52)) : frac;
  const uint64_t mag = fixed_scale(m, (be > 1 ? be : 1) - 1075 + e);
  return (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

// s_hi = 2^(32 - e), s_lo = 2^-e; |v| < 2^63.
PHI_HD inline float from_fixed(long long v, float s_hi, float s_lo) {
  const uint64_t mag = v < 0 ? uint64_t(0) - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  const float hi = static_cast<float>(static_cast<uint32_t>(mag >> 32));
  const float lo = static_cast<float>(static_cast<uint32_t>(mag & 0xffffffffu));
  const float r = fmaf(hi, s_hi, lo * s_lo);
  return v < 0 ? -r : r;
}

PHI_HD inline double from_fixed(long long v, double s_hi, double s_lo) {
  const uint64_t mag = v < 0 ? uint64_t(0) - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  const double hi = static_cast<double>(static_cast<uint32_t>(mag >> 32));
  const double lo = static_cast<double>(static_cast<uint32_t>(mag & 0xffffffffu));
  const double r = fma(hi, s_hi, lo * s_lo);
  return v < 0 ? -r : r;
}

}  // namespace phi
