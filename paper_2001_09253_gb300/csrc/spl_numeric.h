// Integer-pipe numerics shared by the kernels (and compiled on the host by the tests).
//
// On GB300 every FP64 instruction, and every conversion to or from binary64, issues at about
// 1.7 lanes/clk/SM, against ~128 for the FP32 and integer pipes.  The mixed-precision path
// therefore forms the differences of binary64 knots, values and query positions with integer
// arithmetic on their encodings, and converts between binary32 and binary64 the same way.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define SPL_HD __host__ __device__ __forceinline__
#else
#define SPL_HD inline
#endif

namespace spl {

SPL_HD uint64_t bits64(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return u;
#endif
}

SPL_HD double from_bits64(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double v;
  std::memcpy(&v, &u, 8);
  return v;
#endif
}

SPL_HD uint32_t bits32(float v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(v);
#else
  uint32_t u;
  std::memcpy(&u, &v, 4);
  return u;
#endif
}

SPL_HD float from_bits32(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float v;
  std::memcpy(&v, &u, 4);
  return v;
#endif
}

SPL_HD int clz64(uint64_t v) {  // v != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// b - a rounded to nearest-even binary32, from the encodings of two binary64 numbers with
// normal exponents.  The significands are aligned on the larger exponent with 9 guard bits
// in a signed 64-bit integer, so the difference is exact whenever the exponents differ by at
// most 9 (always the case for neighbouring knots, a query and its bracketing knots, or two
// values of similar size); for wider gaps the smaller operand loses bits below 2^-53 of the
// larger one, far under binary32 resolution.  Returns false (and leaves *out unset) for zero,
// subnormal, infinite or NaN inputs and for results outside binary32's normal range: the
// caller then takes the (rare) FP64 route.
SPL_HD bool diff_f32(double b, double a, float *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const int eb = (int)((ub >> 52) & 0x7FF), ea = (int)((ua >> 52) & 0x7FF);
  if (eb == 0 || ea == 0 || eb == 0x7FF || ea == 0x7FF) return false;
  int64_t mb = (int64_t)((ub & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  int64_t ma = (int64_t)((ua & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  if (ub >> 63) mb = -mb;
  if (ua >> 63) ma = -ma;
  int E;
  int64_t D;
  if (eb >= ea) {
    const int d = eb - ea;
    E = eb;
    const int64_t MA = (d <= 9) ? ma * ((int64_t)1 << (9 - d)) : (d >= 72 ? (ma < 0 ? -1 : 0) : (ma >> (d - 9)));
    D = mb * 512 - MA;
  } else {
    const int d = ea - eb;
    E = ea;
    const int64_t MB = (d <= 9) ? mb * ((int64_t)1 << (9 - d)) : (d >= 72 ? (mb < 0 ? -1 : 0) : (mb >> (d - 9)));
    D = MB - ma * 512;
  }
  if (D == 0) {
    *out = 0.0f;
    return true;
  }
  const uint32_t sign = D < 0 ? 1u : 0u;
  uint64_t u = D < 0 ? (uint64_t)(-D) : (uint64_t)D;  // |D| < 2^63
  int msb = 63 - clz64(u);
  int sh = msb - 23;
  uint64_t q;
  if (sh > 0) {
    q = u >> sh;
    const uint64_t rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q == (1ull << 24)) {
      q >>= 1;
      ++msb;
    }
  } else {
    q = u << (-sh);
  }
  // value = (q / 2^23) * 2^(msb + E - 1084)
  const int biased = msb + E - 1084 + 127;
  if (biased < 1 || biased > 254) return false;
  *out = from_bits32((sign << 31) | ((uint32_t)biased << 23) | ((uint32_t)q & 0x7FFFFFu));
  return true;
}

// b - a rounded to nearest-even binary32 for the common case of two binary64 numbers with
// the same sign and exponent field (neighbouring knots, a query and the knot below it): the
// encodings then differ by the exact difference in units of the shared ulp, so one integer
// subtraction and a normalisation give the result.  Returns false when the operands are not
// in one binade (or are zero, subnormal, infinite or NaN): use diff_f32 then.
SPL_HD bool diff_same_f32(double b, double a, float *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const uint32_t hb = (uint32_t)(ub >> 52), ha = (uint32_t)(ua >> 52);  // sign and exponent
  const uint32_t e = hb & 0x7FFu;
  if (hb != ha || e == 0 || e == 0x7FF) return false;
  int64_t D = (int64_t)(ub - ua);  // (b - a) / 2^(e - 1075), |D| < 2^52
  if (hb & 0x800u) D = -D;          // negative operands: larger magnitude is smaller value
  if (D == 0) {
    *out = 0.0f;
    return true;
  }
  const uint32_t sign = D < 0 ? 1u : 0u;
  const uint64_t u = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
  const int lz = clz64(u);
  const uint64_t nrm = u << lz;  // leading one at bit 63
  uint64_t q = nrm >> 40;        // 24 significant bits
  const uint64_t rem = nrm & ((1ull << 40) - 1);
  if (rem > (1ull << 39) || (rem == (1ull << 39) && (q & 1))) ++q;
  int msb = 63 - lz;
  if (q == (1ull << 24)) {
    q >>= 1;
    ++msb;
  }
  const int biased = msb + (int)e - 1075 + 127;
  if (biased < 1 || biased > 254) return false;
  *out = from_bits32((sign << 31) | ((uint32_t)biased << 23) | ((uint32_t)q & 0x7FFFFFu));
  return true;
}

// Cheapest case of diff_same_f32: same sign and exponent field, 0 <= difference < 2^31 ulps,
// and a scale 2^(e-1075) inside binary32's normal range.  The count of ulps converts to
// binary32 with one correctly rounded int32 conversion; the power-of-two scale is exact.
SPL_HD bool diff_small_f32(double b, double a, float *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const uint32_t hb = (uint32_t)(ub >> 52);
  if (hb != (uint32_t)(ua >> 52)) return false;
  const uint32_t e = hb & 0x7FFu;
  if (e < 949u || e > 1171u) return false;  // 2^(e-1075) and 2^(e-1044) within binary32's normal range
  const int64_t D = (hb & 0x800u) ? (int64_t)(ua - ub) : (int64_t)(ub - ua);
  if (D < 0 || D >= (int64_t)0x80000000LL) return false;
  const float scale = from_bits32((e - 1075u + 127u) << 23);
  *out = (float)(int32_t)D * scale;
  return true;
}

// ---- double-float ("float-float") arithmetic: value = hi + lo, |lo| <= ulp(hi)/2 ----
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum, and the FMA form of
// TwoProduct; relative accuracy of the compound operations about 2^-46.
struct F2 {
  float hi, lo;
};

SPL_HD F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return F2{s, e};
}

SPL_HD F2 fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return F2{s, b - (s - a)};
}

SPL_HD F2 two_prod(float a, float b) {
  const float p = a * b;
#ifdef __CUDA_ARCH__
  return F2{p, __fmaf_rn(a, b, -p)};
#else
  return F2{p, std::fmaf(a, b, -p)};
#endif
}

SPL_HD float fma32(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

SPL_HD float f32_of_small_uint(uint32_t v) {  // v < 2^23, exactly
  return from_bits32(0x4B000000u | v) - 8388608.0f;
}

// b - a rounded to nearest-even binary32 on the integer and FP32 pipes, for b >= a with the same
// sign and exponent field and a difference below 2^39 units of their shared ulp (widths of
// increasing knots, a query above the knot that brackets it): the ulp count D (non-negative
// whatever the operands' sign) splits as D = Dh 2^16 + Dl with Dh < 2^23 and Dl < 2^16; each part
// is exact in binary32 (the encoding of 2^23 + part, minus 2^23), and one FMA forms Dh 2^16 + Dl
// with a single rounding.  The scale 2^(e-1075) is a power of two within binary32's normal
// range, so the final product is exact.  Returns false otherwise, b < a included (the caller then
// takes a wider route).
SPL_HD bool diff_up_f32(double b, double a, float *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const uint32_t hb = (uint32_t)(ub >> 52);
  if (hb != (uint32_t)(ua >> 52)) return false;
  const uint32_t e = hb & 0x7FFu;
  if (e - 949u > 214u) return false;  // e in [949, 1163]: 2^(e-1075) and 2^(e-1075+39) normal
  const uint64_t u = (hb & 0x800u) ? ua - ub : ub - ua;
  if (u >> 39) return false;  // also b < a (u wraps to a huge count)
  const float r = fma32(f32_of_small_uint((uint32_t)(u >> 16)), 65536.0f, f32_of_small_uint((uint32_t)u & 0xFFFFu));
  *out = r * from_bits32((e - 1075u + 127u) << 23);
  return true;
}

SPL_HD F2 df_add(F2 a, F2 b) {
  F2 s = two_sum(a.hi, b.hi);
  const float e = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, e);
}

SPL_HD F2 df_neg(F2 a) { return F2{-a.hi, -a.lo}; }

SPL_HD F2 df_mul_f(F2 a, float b) {
  F2 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fma32(a.lo, b, p.lo));
}

SPL_HD F2 df_mul(F2 a, F2 b) {
  F2 p = two_prod(a.hi, b.hi);
  const float e = fma32(a.hi, b.lo, fma32(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}

// a / b with the binary32 reciprocal r ~ 1/b.hi: q1 = a.hi r, one correction from the
// double-float remainder a - q1 b.
SPL_HD F2 df_div(F2 a, F2 b, float r) {
  const float q1 = a.hi * r;
  F2 rem = df_add(a, df_neg(df_mul_f(b, q1)));
  const float q2 = rem.hi * r;
  return fast_two_sum(q1, q2);
}

// b - a as a double-float (hi = the binary32 rounding of the difference, lo = the rounding
// of what is left), from the same exact integer difference as diff_f32; about 48 correct
// bits.  Same applicability as diff_f32.
SPL_HD bool diff_f2(double b, double a, F2 *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const int eb = (int)((ub >> 52) & 0x7FF), ea = (int)((ua >> 52) & 0x7FF);
  if (eb == 0 || ea == 0 || eb == 0x7FF || ea == 0x7FF) return false;
  int64_t mb = (int64_t)((ub & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  int64_t ma = (int64_t)((ua & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  if (ub >> 63) mb = -mb;
  if (ua >> 63) ma = -ma;
  int E;
  int64_t D;
  if (eb >= ea) {
    const int d = eb - ea;
    E = eb;
    const int64_t MA = (d <= 9) ? ma * ((int64_t)1 << (9 - d)) : (d >= 72 ? (ma < 0 ? -1 : 0) : (ma >> (d - 9)));
    D = mb * 512 - MA;
  } else {
    const int d = ea - eb;
    E = ea;
    const int64_t MB = (d <= 9) ? mb * ((int64_t)1 << (9 - d)) : (d >= 72 ? (mb < 0 ? -1 : 0) : (mb >> (d - 9)));
    D = MB - ma * 512;
  }
  if (D == 0) {
    *out = F2{0.0f, 0.0f};
    return true;
  }
  // hi: D rounded to 24 significant bits (as an integer), lo: the exact remainder rounded
  const uint64_t u = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
  const int msb = 63 - clz64(u);
  const int sh = msb - 23;
  int64_t Dhi = D;
  if (sh > 0) {
    uint64_t q = u >> sh;
    const uint64_t rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    Dhi = (D < 0 ? -(int64_t)(q << sh) : (int64_t)(q << sh));
  }
  const int64_t Dlo = D - Dhi;  // exact, |Dlo| <= 2^(sh-1)
  // scale 2^(E - 1084) applied through binary32 arithmetic on exact integers
  auto to_f32 = [&](int64_t v, float *f) -> bool {
    if (v == 0) {
      *f = 0.0f;
      return true;
    }
    const uint64_t w = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
    int hb = 63 - clz64(w);
    int s2 = hb - 23;
    uint64_t mq;
    if (s2 > 0) {
      mq = w >> s2;
      const uint64_t rm = w & ((1ull << s2) - 1), hf = 1ull << (s2 - 1);
      if (rm > hf || (rm == hf && (mq & 1))) ++mq;
      if (mq == (1ull << 24)) {
        mq >>= 1;
        ++hb;
      }
    } else {
      mq = w << (-s2);
    }
    const int biased = hb + E - 1084 + 127;
    if (biased < 1 || biased > 254) return false;
    *f = from_bits32(((v < 0 ? 1u : 0u) << 31) | ((uint32_t)biased << 23) | ((uint32_t)mq & 0x7FFFFFu));
    return true;
  };
  F2 r;
  if (!to_f32(Dhi, &r.hi)) return false;
  if (!to_f32(Dlo, &r.lo)) r.lo = 0.0f;  // below binary32's range: negligible
  *out = r;
  return true;
}

// b - a as a double-float for b >= a with the same sign and exponent field (widths of increasing
// knots): the count D < 2^52 of their shared ulp is exact; hi is D rounded to 24 significant bits
// (an integer q in [2^23, 2^24] shifted, written straight into a binary32 encoding) and lo the
// exact remainder D - hi rounded to binary32 (|lo| <= 2^-24 |hi|, so hi + lo carries about 47
// bits), both times the ulp 2^(e-1075), a power of two within binary32's normal range.  Returns
// false otherwise (b < a included); the caller then takes the general route (diff_f2).
SPL_HD bool diff_up_f2(double b, double a, F2 *out) {
  const uint64_t ub = bits64(b), ua = bits64(a);
  const uint32_t hb = (uint32_t)(ub >> 52);
  if (hb != (uint32_t)(ua >> 52)) return false;
  const uint32_t e = hb & 0x7FFu;
  if (e - 949u > 200u) return false;  // e in [949, 1149]: 2^(e-1075) and 2^(e-1075+53) normal
  const uint64_t D = (hb & 0x800u) ? ua - ub : ub - ua;
  if (D >> 52) return false;          // b < a (the count wraps)
  const float scale = from_bits32((e - 1075u + 127u) << 23);
  if (D < (1ull << 24)) {             // exact in binary32
    *out = F2{(float)(uint32_t)D * scale, 0.0f};
    return true;
  }
  const int sh = 40 - clz64(D);       // msb - 23, in [1, 28]
  uint64_t q = D >> sh;
  const uint64_t rem = D & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;  // q in [2^23, 2^24]
  const int64_t lo = (int64_t)(D - (q << sh));     // |lo| <= 2^(sh-1) < 2^28
  // q in [2^23, 2^24] is 0x4A800000 + q as a binary32 encoding (2^24 rolls the exponent over);
  // the shift goes into the exponent field
  const float hi = from_bits32(0x4A800000u + (uint32_t)q + ((uint32_t)sh << 23));
  *out = F2{hi * scale, (float)(int32_t)lo * scale};
  return true;
}

// A binary64 value as a double-float on the integer pipe: hi = d rounded to binary32, lo = d - hi
// rounded to binary32 (d - hi is exact: |d - hi| <= ulp32(hi)/2 holds at most 29 significant bits;
// its rounding leaves hi + lo within 2^-48 |d|).  For |d| in binary32's normal range with room for
// lo (biased binary64 exponent in [949, 1149]) and zero; false otherwise.
SPL_HD bool f64_to_f2(double d, F2 *out) {
  const uint64_t u = bits64(d);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7FFu;
  if (e == 0u && (u << 1) == 0ull) {
    *out = F2{from_bits32((uint32_t)(u >> 32) & 0x80000000u), 0.0f};
    return true;
  }
  if (e - 949u > 200u) return false;
  const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;  // 53 bits
  uint64_t q = m >> 29;
  const uint64_t rem = m & ((1ull << 29) - 1), half = 1ull << 28;
  if (rem > half || (rem == half && (q & 1))) ++q;  // q in [2^23, 2^24]
  const int32_t lo = (int32_t)((int64_t)m - (int64_t)(q << 29));  // |lo| <= 2^28
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  // hi = q 2^(e-1075+29): the encoding of q in [2^23, 2^24] moved by e - 1075 + 29 in the exponent
  const float hi = from_bits32(sign | (0x4A800000u + (uint32_t)q + ((e - 1046u) << 23)));
  const float lo_scale = from_bits32((e - 1075u + 127u) << 23);
  *out = F2{hi, (sign ? -(float)lo : (float)lo) * lo_scale};
  return true;
}

// Double-float product with a double-float: about 2^-46 relative (two_prod of the leading parts
// plus the cross terms).
SPL_HD F2 df_mul2(F2 a, F2 b) {
  const F2 p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fma32(a.hi, b.lo, fma32(a.lo, b.hi, p.lo)));
}

// Exact binary32 -> binary64 conversion on the integer pipe (normal numbers and zero;
// subnormal, infinite and NaN inputs go through the hardware conversion).
SPL_HD double f32_to_f64(float f) {
  const uint32_t u = bits32(f);
  const uint32_t e = (u >> 23) & 0xFF;
  if (e == 0 || e == 0xFF) {
    if ((u & 0x7FFFFFFFu) == 0) return from_bits64((uint64_t)(u >> 31) << 63);
    return (double)f;
  }
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  return from_bits64(s | ((uint64_t)(e + 896) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29));
}

// binary64 -> binary32 rounded to nearest-even on the integer pipe, for values in binary32's
// normal range; others go through the hardware conversion.
SPL_HD float f64_to_f32(double d) {
  const uint64_t u = bits64(d);
  const int e = (int)((u >> 52) & 0x7FF) - 1023 + 127;
  if (e < 1 || e > 254) return (float)d;
  uint64_t m = (u & 0xFFFFFFFFFFFFFull);
  uint64_t q = m >> 29;
  const uint64_t rem = m & ((1ull << 29) - 1), half = 1ull << 28;
  if (rem > half || (rem == half && (q & 1))) ++q;
  uint32_t bits = ((uint32_t)(u >> 63) << 31) | (uint32_t)((((uint64_t)e) << 23) + q);  // carry ripples into the exponent
  if (((bits >> 23) & 0xFF) == 0xFF) return (float)d;
  return from_bits32(bits);
}

// The one-division form of section "Fast Interpolation",
//   S = (xa y_{j+1} + bx y_j + (1/6)((xa^2 - ba^2) xa y''_{j+1} + (bx^2 - ba^2) bx y''_j)) (1/ba),
// with xa = q - x_j, bx = x_{j+1} - q, ba = x_{j+1} - x_j, evaluated in double-float arithmetic
// (about 46 bits) on the integer and binary32 pipes: the differences exact (same-binade ulp
// counts), the binary64 values, y'' and 1/ba split into double-floats, the result summed back into
// binary64.  Returns false (and leaves *out unset) when an operand lies outside the routines'
// domain (knots and query not in one binade, values outside binary32's range with room for the
// low part); the caller then evaluates in binary64.
SPL_HD bool newint_f2(double q, double xj, double xj1, double yj, double yj1, double ppj, double ppj1, double inv_ba,
                      double *out) {
  F2 xa, bx, ba, y0, y1, p0, p1, ib;
  if (!diff_up_f2(q, xj, &xa) || !diff_up_f2(xj1, q, &bx) || !diff_up_f2(xj1, xj, &ba)) return false;
  if (!f64_to_f2(yj, &y0) || !f64_to_f2(yj1, &y1) || !f64_to_f2(ppj, &p0) || !f64_to_f2(ppj1, &p1) ||
      !f64_to_f2(inv_ba, &ib))
    return false;
  constexpr float kSixthHi = (float)(1.0 / 6.0);
  constexpr float kSixthLo = (float)(1.0 / 6.0 - (double)kSixthHi);
  const F2 ba2 = df_mul2(ba, ba);
  const F2 C = df_mul2(df_mul2(df_add(df_mul2(xa, xa), df_neg(ba2)), xa), p1);
  const F2 D = df_mul2(df_mul2(df_add(df_mul2(bx, bx), df_neg(ba2)), bx), p0);
  const F2 lower = df_add(df_mul2(xa, y1), df_mul2(bx, y0));
  const F2 sum = df_add(lower, df_mul2(df_add(C, D), F2{kSixthHi, kSixthLo}));
  const F2 S = df_mul2(sum, ib);
  *out = f32_to_f64(S.hi) + f32_to_f64(S.lo);
  return true;
}

}  // namespace spl
