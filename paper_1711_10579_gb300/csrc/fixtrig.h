// Sine and cosine of a bus angle in 64-bit fixed point, on the integer pipes.
//
// The voltage update turns (|V|, delta) into V = |V| (cos delta, sin delta)
// for every bus and scenario at every Newton iteration.  FP64 arithmetic is
// the scarce resource of this GPU, so the trigonometry runs in integers:
// the table-driven method of P. T. P. Tang (1990) -- delta = j h + r with
// h = 2^-7, (cos jh, sin jh) from a table, |r| <= 2^-8 -- with the angle,
// the table and the Taylor series of sin r and cos r in 64-bit fixed point:
//   sin r = r (1 - r^2/6 + r^4/120)             (next term < 3e-21)
//   cos r = 1 - (r^2/2 - r^4/24 + r^6/720)      (next term < 2e-24)
// and cos(jh + r), sin(jh + r) by angle addition.  Every fixed-point step
// truncates at or below 2^-60, so the results are the exact values rounded
// to FP64 within one unit in the last place.  Conversions to and from FP64
// are bit manipulations.  Only |delta| <= kHalf h = 4 is served; the caller
// falls back to sincos() outside.
//
// The same code compiles for the host (unsigned __int128 in place of the
// 64-bit multiply-high instructions), so it is tested on the CPU against
// the library sine and cosine.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PF_FX_HD __host__ __device__ __forceinline__
#else
#define PF_FX_HD inline
#endif

namespace pf {
namespace fx {

constexpr int kHalf = 512;  // table rows j = -kHalf..kHalf, angle j 2^-7

PF_FX_HD uint64_t umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

PF_FX_HD int64_t mulhi(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

PF_FX_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

PF_FX_HD uint64_t bits_of(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
#endif
}

PF_FX_HD double double_of(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, 8);
  return v;
#endif
}

// FP64 -> FP32 by truncating the significand of the IEEE-754 encoding with
// integer instructions only (a conversion instruction would run on the FP64
// pipe).  Within the FP32 normal range the result is v rounded toward zero
// (|error| < 1 FP32 ulp); magnitudes below 2^-126, zero included, become a
// zero of the same sign; magnitudes beyond the FP32 range an infinity of the
// same sign; NaN stays NaN.
PF_FX_HD float to_f32_trunc(double v) {
  const uint64_t u = bits_of(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
  const int e = (int)ex - 1023 + 127;
  const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const bool nan = ex == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
  uint32_t bits = sign | ((uint32_t)e << 23) | mant;
  bits = e <= 0 ? sign : bits;
  bits = e >= 255 ? (sign | 0x7f800000u | (nan ? 0x400000u : 0u)) : bits;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(bits);
#else
  float f;
  memcpy(&f, &bits, 4);
  return f;
#endif
}

// a as a signed Q60 number (a 2^60 rounded); false when |a| > 4 or a is not
// finite.
PF_FX_HD bool to_q60(double a, int64_t* q) {
  const uint64_t u = bits_of(a);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex > 1025) return false;  // |a| >= 8, inf or NaN
  if (ex == 0) {                // zero or subnormal
    *q = 0;
    return true;
  }
  const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // a = m 2^(ex - 1075)
  const int sh = ex - 1015;                                     // a 2^60 = m 2^sh
  uint64_t mag;
  if (sh >= 0) mag = m << sh;  // sh <= 10: below 2^63
  else if (sh > -64) mag = (m + (1ull << (-sh - 1))) >> (-sh);
  else mag = 0;
  if (mag > (1ull << 62)) return false;
  *q = (u >> 63) ? -(int64_t)mag : (int64_t)mag;
  return true;
}

// x 2^-60 as a double (|x| <= 2^62), the magnitude rounded half up.
PF_FX_HD double from_q60(int64_t x) {
  if (x == 0) return 0.0;
  const uint64_t sign = (uint64_t)x & (1ull << 63);
  const uint64_t a = x < 0 ? (uint64_t)(-x) : (uint64_t)x;
  const int p = 63 - clz64(a);  // leading bit: x 2^-60 in [2^(p-60), 2^(p-59))
  int e = p - 60;
  uint64_t m;
  if (p > 52) {
    const int sh = p - 52;
    m = (a + (1ull << (sh - 1))) >> sh;
    if (m >> 53) {
      m >>= 1;
      ++e;
    }
  } else {
    m = a << (52 - p);
  }
  return double_of(sign | ((uint64_t)(e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull));
}

// sin a and cos a for |a| <= 4; tab[2 (j + kHalf)] = cos(j 2^-7) 2^62 and
// tab[2 (j + kHalf) + 1] = sin(j 2^-7) 2^62, rounded.  False outside.
PF_FX_HD bool sincos_q(const long long* tab, double a, double* s, double* c) {
  int64_t q;
  if (!to_q60(a, &q)) return false;
  const int64_t j = (q + (1ll << 52)) >> 53;  // nearest multiple of 2^-7 (floor shift)
  const int64_t r = q - (j << 53);            // Q60, |r| <= 2^52 (2^-8)
  const bool rneg = r < 0;
  const uint64_t U = (uint64_t)(rneg ? -r : r) << 10;  // |r| in Q70, <= 2^62
  const uint64_t u2 = umulhi(U, U);                    // r^2, Q76
  const uint64_t u4 = umulhi(u2, u2);                  // r^4, Q88
  const uint64_t u6 = umulhi(u4, u2);                  // r^6, Q100
  // 2^64 / 6, 2^64 / 120, 2^64 / 24, 2^64 / 720, rounded
  const uint64_t c6 = 3074457345618258603ull, c120 = 153722867280912930ull,
                 c24 = 768614336404564651ull, c720 = 25620477880152155ull;
  const uint64_t ds = umulhi(u2, c6) - (umulhi(u4, c120) >> 12);  // r^2/6 - r^4/120, Q76
  const uint64_t sin70 = U - (umulhi(U, ds) >> 12);                // |sin r|, Q70
  const uint64_t ec = (u2 >> 1) - (umulhi(u4, c24) >> 12) + (umulhi(u6, c720) >> 24);  // Q76
  const int64_t cr = (1ll << 62) - (int64_t)((ec + (1ull << 13)) >> 14);  // cos r, Q62
  int64_t sr = (int64_t)((sin70 + (1ull << 7)) >> 8);                      // |sin r|, Q62
  if (rneg) sr = -sr;
  const long long* t = tab + 2 * (j + kHalf);
  const int64_t cj = t[0], sj = t[1];
  // Q62 x Q62 / 2^64 = Q60
  *c = from_q60(mulhi(cj, cr) - mulhi(sj, sr));
  *s = from_q60(mulhi(sj, cr) + mulhi(cj, sr));
  return true;
}

}  // namespace fx
}  // namespace pf
