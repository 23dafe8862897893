// Binary32 arithmetic on binary64 inputs, shared by the mixed-precision kernels: exact
// differences of binary64 operands rounded once to binary32, the integer-pipe conversions between
// the formats, the binary32 quotient and the one-division form of "Fast Interpolation".
#pragma once
#include "spl_device.cuh"
#include "spl_numeric.h"

namespace spl {

// ---- out-of-line FP64 fallbacks (never speculated) ----
static __device__ __noinline__ float sub_f64_f32(double b, double a) { return (float)(b - a); }
static __device__ __noinline__ float cvt_f64_f32(double d) { return (float)d; }
static __device__ __noinline__ double cvt_f32_f64(float f) { return (double)f; }
static __device__ __noinline__ F2 sub_f64_f2(double b, double a) {
  const double d = b - a;
  const float hi = (float)d;
  return F2{hi, (float)(d - (double)hi)};
}

// neighbouring operands (same binade and a small difference almost always).  For two finite
// numbers with the same sign and exponent field the FP64 subtraction is exact (Sterbenz) and
// the conversion rounds the exact difference once, exactly as the integer routes do: one FP64
// subtraction and one conversion instead of ~60 integer instructions; other pairs take the
// integer routes.
__device__ __forceinline__ float dif32_near(double b, double a) {
  const unsigned hb = (unsigned)(bits64(b) >> 32), ha = (unsigned)(bits64(a) >> 32);
  if (((hb ^ ha) >> 20) == 0u && ((hb >> 20) & 0x7FFu) != 0x7FFu) return (float)(b - a);
  float v;
  if (diff_small_f32(b, a, &v)) return v;
  if (diff_same_f32(b, a, &v)) return v;
  if (diff_f32(b, a, &v)) return v;
  return sub_f64_f32(b, a);
}

// b - a rounded once to binary32 for b >= a (widths of increasing knots, a query above its
// bracketing knot), without FP64 instructions in the common case (the integer/FP32 route of
// diff_up_f32): for kernels that are throughput-bound with many warps in flight, where the FP64
// pipe (~1/64 of the FP32 rate) is the scarce unit; other pairs as dif32_near.
static __device__ __noinline__ float dif32_near_slow(double b, double a) { return dif32_near(b, a); }
__device__ __forceinline__ float dif32_up(double b, double a) {
  float v;
  if (diff_up_f32(b, a, &v)) return v;
  // wider same-binade pairs (small knots: an ulp count of 2^39 or more) on the integer pipe too
  if (diff_same_f32(b, a, &v)) return v;
  // out of line: inlined, the FP64 subtraction of dif32_near's Sterbenz case was evaluated
  // speculatively for every operand pair (measured: the FP64 pipe twice as busy)
  return dif32_near_slow(b, a);
}

__device__ __forceinline__ F2 dif2(double b, double a) {
  F2 v;
  if (diff_f2(b, a, &v)) return v;
  return sub_f64_f2(b, a);
}
// the same out of line: the fallback of the same-binade and in-range routes, rare, kept out of
// the refinement's unrolled rows (instruction-cache footprint)
static __device__ __noinline__ F2 dif2_slow(double b, double a) { return dif2(b, a); }

__device__ __forceinline__ float to_f32(double d) {
  const uint64_t u = bits64(d);
  const int e = (int)((u >> 52) & 0x7FF) - 1023 + 127;
  if (e >= 1 && e <= 253) return f64_to_f32(d);  // normal binary32 range, no carry into Inf
  return cvt_f64_f32(d);
}

__device__ __forceinline__ double to_f64(float f) {
  const uint32_t e = (bits32(f) >> 23) & 0xFF;
  if (e != 0 && e != 0xFF) return f32_to_f64(f);
  if ((bits32(f) & 0x7FFFFFFFu) == 0) return from_bits64((uint64_t)(bits32(f) >> 31) << 63);
  return cvt_f32_f64(f);
}

// Difference of two values (often in different binades): one FP64 subtraction, exact or
// rounded to 53 bits, then the integer-pipe narrowing.  The FP64 pipe is otherwise nearly
// idle in this kernel, so this is cheaper than the integer route for unrelated operands.
__device__ __forceinline__ float dy32(double b, double a) { return to_f32(b - a); }

__device__ __forceinline__ F2 f2_of(double v) {
  const float hi = to_f32(v);
  return F2{hi, (float)(v - (double)hi)};  // once per tile (end slopes)
}

__device__ __forceinline__ float quot32(float num, float den, float r) {
  float q = num * r;
  float rem = fmaf(-den, q, num);
  return fmaf(rem, r, q);
}

// "Fast Interpolation" in binary32, with xa = x - x_j and bx = x_{j+1} - x.
__device__ __forceinline__ float newint32(float xa, float bx, float yj, float yj1, float ppj, float ppj1,
                                          float ba, float inv_ba) {
  float ba2 = ba * ba;
  float lower = xa * yj1 + bx * yj;
  float C = (xa * xa - ba2) * xa * ppj1;
  float D = (bx * bx - ba2) * bx * ppj;
  return (lower + (1.0f / 6.0f) * (C + D)) * inv_ba;
}

__device__ __forceinline__ void prefetch_l2m(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_l1m(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}


}  // namespace spl
