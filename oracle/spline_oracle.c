/*
 * Plain FP64 CPU oracle for cubic-spline fit + evaluation (Hornbeck,
 * "Fast Cubic Spline Interpolation", arXiv 2001.09253).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA path, and the product never
 * calls it.
 *
 * Build: single-threaded, -O2 -ffp-contract=off (no fused multiply-add, so
 * every product and sum is rounded separately, as written).
 *
 * Readings of the paper that this file fixes (each also in the design notes):
 *   - "natural" end: an end slope strictly greater than 0.99e30 (section
 *     "Start and End Derivatives").  +inf is natural; NaN or -inf is an
 *     invalid argument.
 *   - Clamped last row: a_n = h, b_n = 2h (the equation just before the
 *     matrix-form listing in "Start and End Derivatives"; the printed matrix
 *     entries have a_n and b_n swapped).
 *   - Diagonal b_j is formed as 2(a_j + c_j), which equals 2(x_{j+1}-x_{j-1})
 *     of eq. (init_val) in exact arithmetic and keeps b = 2(a + c) exact in
 *     floating point (the dominance argument of "Generating Second
 *     Derivatives").
 *   - Query grid ("Quality Checks", the linspace of the interpolated-curve
 *     check; "Curve Interpolation", step 8): x_k = x_0 + k*step with
 *     step = (x_{n-1} - x_0)/(M-1), product and sum rounded separately, the
 *     last point forced to x_{n-1}; M = 1 gives the single point x_0.
 *   - Bracket: j(q) = largest i in [0, n-2] with x_i < q, or 0 if none
 *     (strict <, so a query equal to a knot takes the interval on its left;
 *     queries past the last knot extrapolate with the last cubic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORC_OK 0
#define ORC_INVALID_ARG 1
#define ORC_NOT_INCREASING 2
#define ORC_NONFINITE 3

/* Paper, section "Start and End Derivatives": an end derivative above
 * 0.99e30 selects the natural condition (y'' = 0) at that end. */
static int is_natural(double slope) { return slope > 0.99e30; }

/* Input checks of new_second_derivative (its asserts: more than two knots,
 * strictly increasing knots).  Finite values are an added requirement. */
int orc_validate(int64_t n, const double *x, const double *y, double yp1, double ypn) {
  if (n < 3 || x == 0 || y == 0) return ORC_INVALID_ARG;
  if (isnan(yp1) || isnan(ypn)) return ORC_INVALID_ARG;
  if ((isinf(yp1) && yp1 < 0) || (isinf(ypn) && ypn < 0)) return ORC_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(x[i]) || !isfinite(y[i])) return ORC_NONFINITE;
  for (int64_t i = 1; i < n; ++i)
    if (!(x[i] > x[i - 1])) return ORC_NOT_INCREASING;
  return ORC_OK;
}

/* Row j of the tridiagonal system for y''.
 * Interior rows, section "Generating Second Derivatives", eq. (init_val) and
 * the coefficient list below the matrix form:
 *     a_j = x_j - x_{j-1},  c_j = x_{j+1} - x_j,  b_j = 2(a_j + c_j),
 *     d_j = 6((y_{j+1}-y_j)/(x_{j+1}-x_j) - (y_j-y_{j-1})/(x_j-x_{j-1})).
 * First row, section "Start and End Derivatives": clamped slope y'_1 gives
 *     b = 2(x_1 - x_0), c = x_1 - x_0, d = 6((y_1-y_0)/(x_1-x_0) - y'_1);
 * natural gives y''_0 = 0, i.e. b = 1, c = 0, d = 0.
 * Last row: clamped slope y'_n gives
 *     a = x_{n-1} - x_{n-2}, b = 2a, d = 6(y'_n - (y_{n-1}-y_{n-2})/(x_{n-1}-x_{n-2}));
 * natural gives y''_{n-1} = 0, i.e. a = 0, b = 1, d = 0. */
static void system_row(int64_t n, const double *x, const double *y, double yp1, double ypn,
                       int64_t j, double *a, double *b, double *c, double *d) {
  if (j == 0) {
    *a = 0.0;
    if (is_natural(yp1)) { *b = 1.0; *c = 0.0; *d = 0.0; return; }
    double h = x[1] - x[0];
    *b = 2.0 * h;
    *c = h;
    *d = 6.0 * ((y[1] - y[0]) / h - yp1);
    return;
  }
  if (j == n - 1) {
    *c = 0.0;
    if (is_natural(ypn)) { *a = 0.0; *b = 1.0; *d = 0.0; return; }
    double h = x[n - 1] - x[n - 2];
    *a = h;
    *b = 2.0 * h;
    *d = 6.0 * (ypn - (y[n - 1] - y[n - 2]) / h);
    return;
  }
  double aj = x[j] - x[j - 1];
  double cj = x[j + 1] - x[j];
  *a = aj;
  *c = cj;
  *b = 2.0 * (aj + cj);
  *d = 6.0 * ((y[j + 1] - y[j]) / cj - (y[j] - y[j - 1]) / aj);
}

/* Second derivatives y''[0..n-1]: the system above solved by Thomas'
 * algorithm, section "Implementation":
 *     c'_1 = c_1/b_1,  d'_1 = d_1/b_1,
 *     c'_i = c_i/(b_i - a_i c'_{i-1}),  d'_i = (d_i - a_i d'_{i-1})/(b_i - a_i c'_{i-1}),
 *     y''_n = d'_n,  y''_i = d'_i - c'_i y''_{i+1}.
 * d' is kept in ypp and c' in cp (n doubles, caller-owned), as that section
 * describes.  Returns an ORC_* status; ypp is written only on ORC_OK. */
int orc_fit(int64_t n, const double *x, const double *y, double yp1, double ypn,
            double *ypp, double *cp) {
  int st = orc_validate(n, x, y, yp1, ypn);
  if (st != ORC_OK) return st;
  double a, b, c, d;
  system_row(n, x, y, yp1, ypn, 0, &a, &b, &c, &d);
  cp[0] = c / b;
  ypp[0] = d / b;
  for (int64_t i = 1; i < n; ++i) {
    system_row(n, x, y, yp1, ypn, i, &a, &b, &c, &d);
    double den = b - a * cp[i - 1];
    cp[i] = c / den;
    ypp[i] = (d - a * ypp[i - 1]) / den;
  }
  for (int64_t i = n - 2; i >= 0; --i) ypp[i] = ypp[i] - cp[i] * ypp[i + 1];
  return ORC_OK;
}

/* Uniform query grid (reading stated in the file header). */
void orc_grid(int64_t n, const double *x, int64_t m, double *xq) {
  if (m <= 0) return;
  if (m == 1) { xq[0] = x[0]; return; }
  double step = (x[n - 1] - x[0]) / (double)(m - 1);
  for (int64_t k = 0; k < m; ++k) {
    double t = (double)k * step;
    xq[k] = t + x[0];
  }
  xq[m - 1] = x[n - 1];
}

/* Bracketing by the monotone sweep of section "Quality Checks" (the loop
 * that advances the lower index while the next knot lies below the query),
 * with the index held at or below n-2.  Valid for non-decreasing queries. */
void orc_bracket_sweep(int64_t n, const double *x, int64_t m, const double *xq, int64_t *jq) {
  int64_t i = 0;
  for (int64_t k = 0; k < m; ++k) {
    while (i + 1 < n - 1 && x[i + 1] < xq[k]) ++i;
    jq[k] = i;
  }
}

/* Bracketing of one query straight from its definition, by bisection on the
 * sorted knots: the largest i in [0, n-2] with x_i < q, or 0 if none.
 * Serves arbitrary (unsorted) query arrays. */
int64_t orc_bracket_one(int64_t n, const double *x, double q) {
  /* count of knots x_0..x_{n-2} strictly below q */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (x[mid] < q) lo = mid + 1; else hi = mid;
  }
  int64_t j = lo - 1;
  if (j < 0) j = 0;
  return j;
}

void orc_bracket_any(int64_t n, const double *x, int64_t m, const double *xq, int64_t *jq) {
  for (int64_t k = 0; k < m; ++k) jq[k] = orc_bracket_one(n, x, xq[k]);
}

/* Interpolated value on the interval [x_j, x_{j+1}], section "Fast
 * Interpolation", the variation derived there from eq. (nr_formula):
 *     y = (y_j (x_{j+1}-x) + y_{j+1} (x-x_j) + V/6) / (x_{j+1}-x_j),
 *     V = y''_j (x_{j+1}-x)((x_{j+1}-x)^2 - (x_{j+1}-x_j)^2)
 *       + y''_{j+1} (x-x_j)((x-x_j)^2 - (x_{j+1}-x_j)^2). */
double orc_interp(double q, double xj, double xj1, double yj, double yj1, double ppj, double ppj1) {
  double right = xj1 - q;   /* x_{j+1} - x */
  double left = q - xj;     /* x - x_j     */
  double width = xj1 - xj;  /* x_{j+1} - x_j */
  double w2 = width * width;
  double v = ppj * right * (right * right - w2) + ppj1 * left * (left * left - w2);
  return (yj * right + yj1 * left + v / 6.0) / width;
}

void orc_eval(int64_t n, const double *x, const double *y, const double *ypp, int64_t m,
              const double *xq, const int64_t *jq, double *yq) {
  (void)n;
  for (int64_t k = 0; k < m; ++k) {
    int64_t j = jq[k];
    yq[k] = orc_interp(xq[k], x[j], x[j + 1], y[j], y[j + 1], ypp[j], ypp[j + 1]);
  }
}

/* The whole path for one instance: fit, uniform grid of m queries, sweep
 * bracketing, interpolation.  xq/jq/yq may be NULL when m == 0.  Scratch is
 * allocated here.  Returns an ORC_* status. */
int orc_fit_eval(int64_t n, const double *x, const double *y, double yp1, double ypn,
                 int64_t m, double *ypp, double *xq, int64_t *jq, double *yq) {
  if (m < 0) return ORC_INVALID_ARG;
  double *cp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!cp) return ORC_INVALID_ARG;
  int st = orc_fit(n, x, y, yp1, ypn, ypp, cp);
  free(cp);
  if (st != ORC_OK || m == 0) return st;
  orc_grid(n, x, m, xq);
  orc_bracket_sweep(n, x, m, xq, jq);
  orc_eval(n, x, y, ypp, m, xq, jq, yq);
  return ORC_OK;
}
