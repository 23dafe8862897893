// Host build of the library's integer-pipe numerics, exposed to ctypes by the tests.
#include "spl_numeric.h"

extern "C" {
int t_diff_f32(double b, double a, float *out) { return spl::diff_f32(b, a, out) ? 1 : 0; }
double t_f32_to_f64(float f) { return spl::f32_to_f64(f); }
float t_f64_to_f32(double d) { return spl::f64_to_f32(d); }
}
