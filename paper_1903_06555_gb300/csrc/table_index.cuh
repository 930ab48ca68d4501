// Position of a scaled radius in the pre-sampled w-plane table (Sec. 5.1.1):
// s = rho / h_rho >= 0 is split into a sample index ir = floor(s), clamped to
// the last interval, and the interpolation fraction fr = s - ir.
//
// FP32 rounds s - 1/2 to an integer by adding 1.5 * 2^23, so no conversion
// instruction is needed: for s < 2^22 the sum lies in [2^23, 2^24), where
// FP32 steps are exactly 1 and consecutive integers have consecutive bit
// patterns.  (With 2^23 itself, a sum just below 2^23 would land on a
// half-integer for s < 1/4 and give ir = -1.)  An exact integer s may come
// out as ir = s - 1, fr = 1: the same interpolated value.  Host-compilable.
#pragma once

#ifndef PHI_HD
#define PHI_HD __host__ __device__
#endif

#if !defined(__CUDA_ARCH__)
#include <cstring>
#endif

namespace phi {

PHI_HD inline int table_float_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_int(x);
#else
  int b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

// last = index of the last interval (samples - 2), last_f the same as a float.
// Beyond the table, or for a NaN, the last interval is extrapolated.
PHI_HD inline void table_index(float s, int last, float last_f, int& ir, float& fr) {
  const float big = 12582912.0f;                      // 1.5 * 2^23
  const float t = (s - 0.5f) + big;                   // nearest integer to s - 1/2, plus big
  ir = table_float_bits(t) - table_float_bits(big);
  fr = s - (t - big);
  if (!(s < last_f)) {
    ir = last;
    fr = s - last_f;
  }
}

PHI_HD inline void table_index(double s, int last, double last_f, int& ir, double& fr) {
  ir = s < last_f ? static_cast<int>(s) : last;
  fr = s - static_cast<double>(ir);
}

// w-row of a visibility: a = |dw| / h_w as one correctly rounded product (no
// contraction into a later subtraction), its row j = floor(a) clamped to the
// last pair of planes, and the fraction fw = a - j.  Every table kernel and
// the plan's w-row key use this one definition, so they agree bit for bit.
PHI_HD inline float table_w_scaled(float adw, float inv_hw) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(adw, inv_hw);
#else
  return adw * inv_hw;
#endif
}
PHI_HD inline double table_w_scaled(double adw, double inv_hw) {
#if defined(__CUDA_ARCH__)
  return __dmul_rn(adw, inv_hw);
#else
  return adw * inv_hw;
#endif
}
template <typename T>
PHI_HD inline int table_w_row(T aw, int last) {
  // the comparison also sends a NaN to the last row instead of an undefined
  // conversion
  return aw < static_cast<T>(last) ? static_cast<int>(aw) : last;
}

}  // namespace phi
