// Pieces of one Algorithm 1 sweep (k-means w-stacking) that decide its
// result: the nearest-centre assignment and the exact fixed-point sums the
// centres are formed from.  Host-compilable, so that tests can check them
// against their definitions on the CPU.
//
// Assignment: argmin_q (wbar_q - w)^2 in FP64, the lowest q winning ties.
// GB300 runs FP64 arithmetic at about 1/64 of the FP32 rate, so the sweep
// first compares FP32 distances with a bound on their error; when the
// nearest one's upper bound lies below every other centre's lower bound the
// FP64 distances order the same way, and only the remaining visibilities
// take the FP64 scan.
//
// Sums: w 2^S truncated toward zero to an integer (S chosen so that
// |w| 2^S < 2^62 for every w), taken as a 96-bit two's-complement number and
// cut into kLimbs 16-bit limbs.  Limb sums are exact integer sums whatever
// their order, so the centres do not depend on how a sweep is parallelised;
// the truncation moves a centre by less than 2^-S.
#pragma once

#include <cmath>
#include <cstdint>

#ifndef PHI_HD
#define PHI_HD __host__ __device__
#endif

#if !defined(__CUDA_ARCH__)
#include <cstring>
#endif

namespace phi {

constexpr int kLimbs = 6;
constexpr int kAcc = kLimbs + 1;   // limb sums + member count per stack

// Error bound of the FP32 distance |fl(c) - fl(w)| against the exact
// |c - w|: 2^-22 (|c| + |w|), twice the bound of the two roundings to FP32
// and the subtraction; kKmTiny covers FP32 underflow, kKmSlack the rounding
// of the bounds themselves.
constexpr float kKmErr = 2.384185791015625e-07f;   // 2^-22
constexpr float kKmTiny = 1e-30f;
constexpr float kKmSlack = 1.0000152587890625f;    // 1 + 2^-16

PHI_HD inline uint64_t km_double_bits(double w) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(w));
#else
  uint64_t b;
  std::memcpy(&b, &w, sizeof(b));
  return b;
#endif
}

// w 2^S truncated toward zero (exact integer arithmetic on w's bits).
PHI_HD inline int64_t w_fixed(double w, int S) {
  const uint64_t bits = km_double_bits(w);
  const int e = static_cast<int>((bits >> 52) & 0x7ffu);
  if (e == 0) return 0;   // zero and subnormals
  const uint64_t m = (bits & 0xfffffffffffffULL) | (1ULL << 52);
  const int sh = e - 1075 + S;
  uint64_t v = 0;
  if (sh >= 0) v = m << sh;
  else if (sh > -64) v = m >> (-sh);
  return (bits >> 63) ? -static_cast<int64_t>(v) : static_cast<int64_t>(v);
}

// Limb l (16 bits) of v sign-extended to 96 bits.
PHI_HD inline unsigned w_limb(int64_t v, int l) {
  const uint64_t lo = static_cast<uint64_t>(v);
  const unsigned hi = v < 0 ? 0xffffffffu : 0u;
  return l < 4 ? static_cast<unsigned>((lo >> (16 * l)) & 0xffffu)
               : (hi >> (16 * (l - 4))) & 0xffffu;
}

// The total sum_l sum[l] 2^(16 l) modulo 2^96 read as a signed 96-bit
// integer, times 2^-S, as a double (|total| < 2^95 for fewer than 2^33
// values of magnitude below 2^62).
PHI_HD inline double fixed_total(const unsigned long long* sum, int S) {
  unsigned __int128 t = 0;
  for (int l = 0; l < kLimbs; ++l) t += static_cast<unsigned __int128>(sum[l]) << (16 * l);
  const unsigned __int128 mask96 = (static_cast<unsigned __int128>(1) << 96) - 1;
  t &= mask96;
  const bool neg = static_cast<bool>((t >> 95) & 1);
  const unsigned __int128 mag = neg ? ((~t + 1) & mask96) : t;
  const double hi = static_cast<double>(static_cast<uint64_t>(mag >> 64));
  const double lo = static_cast<double>(static_cast<uint64_t>(mag));
  const double total = std::ldexp(std::fma(hi, 18446744073709551616.0, lo), -S);
  return neg ? -total : total;
}

// The centre's part of the FP32 distance bound: kKmErr |cf| + kKmTiny.
PHI_HD inline float km_centre_err(float cf) { return std::fma(kKmErr, std::fabs(cf), kKmTiny); }

// Nearest centre of Algorithm 1 (see above).  c: the centres; cf, ce: their
// FP32 values and km_centre_err of those.
PHI_HD inline int nearest_centre(double w, const double* c, const float* cf, const float* ce,
                                 int K) {
  const float wf = static_cast<float>(w);
  const float aw = std::fabs(wf);
  float tb = INFINITY, eb = 0.f, m2 = INFINITY;
  int qb = 0;
  for (int q = 0; q < K; ++q) {
    const float t = std::fabs(cf[q] - wf);
    const float e = std::fma(kKmErr, aw, ce[q]);
    if (t < tb) {
      m2 = std::fmin(m2, tb - eb);
      tb = t;
      eb = e;
      qb = q;
    } else {
      m2 = std::fmin(m2, t - e);
    }
  }
  if (m2 > (tb + eb) * kKmSlack) return qb;
  double best = INFINITY;
  int s = 0;  // also the stack of a non-finite w (every comparison fails)
  for (int q = 0; q < K; ++q) {
    const double d = (c[q] - w) * (c[q] - w);
    if (d < best) {
      best = d;
      s = q;
    }
  }
  return s;
}

}  // namespace phi
