// Host build of the library's integer-pipe numerics, exposed to ctypes by the tests.
#include "spl_numeric.h"

extern "C" {
int t_diff_f32(double b, double a, float *out) { return spl::diff_f32(b, a, out) ? 1 : 0; }
double t_f32_to_f64(float f) { return spl::f32_to_f64(f); }
float t_f64_to_f32(double d) { return spl::f64_to_f32(d); }
}

extern "C" {
int t_diff_f2(double b, double a, float *hi, float *lo) {
  spl::F2 r;
  if (!spl::diff_f2(b, a, &r)) return 0;
  *hi = r.hi;
  *lo = r.lo;
  return 1;
}
void t_df_div(float ah, float al, float bh, float bl, float *qh, float *ql) {
  float r = 1.0f / bh;
  spl::F2 q = spl::df_div(spl::F2{ah, al}, spl::F2{bh, bl}, r);
  *qh = q.hi;
  *ql = q.lo;
}
void t_df_add(float ah, float al, float bh, float bl, float *sh, float *sl) {
  spl::F2 q = spl::df_add(spl::F2{ah, al}, spl::F2{bh, bl});
  *sh = q.hi;
  *sl = q.lo;
}
void t_df_mul_f(float ah, float al, float b, float *ph, float *pl) {
  spl::F2 q = spl::df_mul_f(spl::F2{ah, al}, b);
  *ph = q.hi;
  *pl = q.lo;
}
}

extern "C" {
int t_diff_same_f32(double b, double a, float *out) { return spl::diff_same_f32(b, a, out) ? 1 : 0; }
}

extern "C" {
int t_diff_small_f32(double b, double a, float *out) { return spl::diff_small_f32(b, a, out) ? 1 : 0; }
int t_diff_up_f32(double b, double a, float *out) { return spl::diff_up_f32(b, a, out) ? 1 : 0; }
}

extern "C" {
void t_two_sum(float a, float b, float *s, float *e) {
  spl::F2 r = spl::two_sum(a, b);
  *s = r.hi;
  *e = r.lo;
}
void t_two_prod(float a, float b, float *p, float *e) {
  spl::F2 r = spl::two_prod(a, b);
  *p = r.hi;
  *e = r.lo;
}
void t_df_mul(float ah, float al, float bh, float bl, float *ph, float *pl) {
  spl::F2 q = spl::df_mul(spl::F2{ah, al}, spl::F2{bh, bl});
  *ph = q.hi;
  *pl = q.lo;
}
}

extern "C" {
int t_diff_up_f2(double b, double a, float *hi, float *lo) {
  spl::F2 r;
  if (!spl::diff_up_f2(b, a, &r)) return 0;
  *hi = r.hi;
  *lo = r.lo;
  return 1;
}
int t_f64_to_f2(double d, float *hi, float *lo) {
  spl::F2 r;
  if (!spl::f64_to_f2(d, &r)) return 0;
  *hi = r.hi;
  *lo = r.lo;
  return 1;
}
}

extern "C" {
int t_newint_f2(double q, double xj, double xj1, double yj, double yj1, double ppj, double ppj1, double inv_ba,
                double *out) {
  return spl::newint_f2(q, xj, xj1, yj, yj1, ppj, ppj1, inv_ba, out) ? 1 : 0;
}
}
