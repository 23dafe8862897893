// Plain FP64 fit + evaluation, fused, one thread per tile of knots.
//
// The fit is the tridiagonal system of eq. (init_val) ("Generating Second Derivatives")
// with the end rows of "Start and End Derivatives", solved by the Thomas recurrences of
// "Implementation"; the evaluation is the one-division form of "Fast Interpolation" at
// the uniform grid of "Curve Interpolation".
//
// Parallel decomposition (GB300 design, not in the paper).  The serial Thomas sweep is cut
// into tiles of L knots, each solved by one thread in two passes over per-warp scratch in
// global memory (lane-interleaved, so warp accesses are coalesced when the lanes move
// together):
//   1. forward elimination of the tile's rows (and of the rows past it that start the back
//      substitution, when the next lane does not hold them), storing c', d' and 1/h.  Its start:
//      a halo grown backwards from the tile from the guess c' = d' = 0 until the product of the
//      per-row bounds a_i / (1.5 a_i + 2 c_i) (< 2/3, from b = 2(a + c) and c' <= 1/2) is below
//      2^-110, or, for a chained tile, the exact c' and a linear correction of d' (see TileRows);
//      2^-110 is far below binary64 resolution because d' at the halo start may exceed the
//      solution inside the tile by many orders of magnitude (knot gaps spread over many
//      decades);
//   2. back substitution from 48 rows past the tile, from the guess y'' = d' (its error is
//      multiplied by c'_i <= c_i / (1.5 a_i + 2 c_i) < 1/2 per row: typically ~0.27, ~1e-27
//      after 48 rows; 3.6e-15 in the worst case), fused with the evaluation of the queries
//      whose interval lies in the tile, walking the uniform grid and the knots down together
//      (the monotone sweep of "Quality Checks", reversed), with the fit's 1/h_j.
//
// GB300 notes: FP64 runs at ~1.7 lanes/clk/SM here and a few warps per SM sub-partition cannot
// keep the pipe busy through their own dependency chains; one CTA of 14 warps per SM measured
// best (13, 15 and 16 warps are slower: more tiles also means more per-tile work).  Global
// scratch leaves the shared memory unused.  Comparisons run on integer keys, divisions as a
// MUFU seed + 3 DFMAs, and the next row's width, reciprocal and slope are computed while the
// current row's elimination is in flight.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_numeric.h"

namespace spl {

constexpr int kThreads = 448;           // 14 warps per CTA
constexpr int kCtasPerSm = 1;
constexpr int kHaloB = 48;              // back-substitution start past the tile end
constexpr int kHaloFMax = 192;          // forward-elimination halo, worst case: (2/3)^192
constexpr int kHaloFMin = 16;
constexpr int kFields = 3;              // c', d' (then y''), 1/h
constexpr int kHaloC = 16;              // c'-only rows before a chained tile: error factor <= 1/12 per row
constexpr int kLane0Short = 56;         // the first lane of a group runs a full halo: its tile is shorter
constexpr int kMRows = 192;             // sensitivity rows kept per lane: (2/3)^192 < 2^-110

// Per-warp scratch: rows relative to the tile start, fields, lanes.
struct Scratch64 {
  double *base;  // rows x kFields x 32 lanes
  double *mb;    // kMRows x 32 lanes: sensitivities of a chained tile's d' to d'_{s0-1}
  int lane;
  __device__ __forceinline__ double &at(long long row, int f) const {
    return base[(((size_t)row * kFields + f) << 5) + lane];
  }
  __device__ __forceinline__ double &m(int row) const { return mb[(row << 5) + lane]; }
};

// Evaluation of one query, "Fast Interpolation": with ba = x_{j+1}-x_j, xa = x-x_j,
// bx = x_{j+1}-x,  y = (xa y_{j+1} + bx y_j + (1/6)((xa^2-ba^2) xa y''_{j+1}
//                                                  + (bx^2-ba^2) bx y''_j)) / ba.
__device__ __forceinline__ double newint64(double q, double xj, double xj1, double yj, double yj1,
                                           double ppj, double ppj1, double ba, double inv_ba) {
  double xa = q - xj;
  double bx = xj1 - q;
  double ba2 = ba * ba;
  double lower = xa * yj1 + bx * yj;
  double C = (xa * xa - ba2) * xa * ppj1;
  double D = (bx * bx - ba2) * bx * ppj;
  return (lower + (1.0 / 6.0) * (C + D)) * inv_ba;
}

// 2t for a normal t by incrementing its exponent (integer pipe); other values take an
// out-of-line FP64 multiply, so that it is never evaluated speculatively.
__device__ __noinline__ double twice_slow(double t) { return 2.0 * t; }
__device__ __forceinline__ double twice(double t) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(t);
  const unsigned e = (unsigned)(u >> 52) & 0x7FFu;
  if (e - 1u < 0x7FDu) return __longlong_as_double((long long)(u + (1ull << 52)));
  return twice_slow(t);
}

__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Start row of the forward halo of a tile beginning at s0 (see the header comment).  Rows are
// scanned eight at a time with independent loads; the halo may end up a few rows longer than
// the bound requires.
__device__ long long halo_start(const double *x, long long n, long long s0) {
  if (s0 <= kHaloFMin + 8) return 0;
  float prod = 1.0f;
  // bound of row i uses a_i = h_{i-1} = x_i - x_{i-1} and c_i = h_i = x_{i+1} - x_i
  double xr = (s0 + 1 < n) ? x[s0 + 1] : x[s0];  // x_{i+1} for the first row i = s0
  long long i = s0;
  for (int cnt = 0; cnt < kHaloFMax; cnt += 8) {
    if (i - 8 <= 0) return 0;
    double xv[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) xv[u] = x[i - u];  // x_i .. x_{i-8}
    float c;
    if (!diff_same_f32(xr, xv[0], &c) || !(s0 + 1 < n)) c = -1.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float a;
      if (!diff_same_f32(xv[u], xv[u + 1], &a)) a = -1.0f;
      const float f = (a > 0.0f && c > 0.0f) ? a / (1.5f * a + 2.0f * c) : 0.6667f;
      prod *= f * 1.0001f;
      c = a;
    }
    xr = xv[7];  // x_{i'+1} of the next chunk's first row i' = i - 8
    i -= 8;      // rows s0 .. i+1 are covered; the guess goes on row i
    if (cnt + 8 >= kHaloFMin && prod < 0x1p-110f) return i;
  }
  return max(s0 - kHaloFMax, 0LL);
}

// Forward state after row r: c'_r, d'_r, h_r, s_r, the precomputed interval r+1
// (xn = x_{r+2}, yn = y_{r+2}, hn = h_{r+1}, ihn = 1/h_{r+1}, sn = s_{r+1}), and the knot and
// value of the row after that, loaded one step ahead (xl = x_{r+3}, yl = y_{r+3}).
struct Fwd64 {
  double cp, dp, h, s;
  double xn, yn, hn, ihn, sn;
  double xl, yl;
};

// Rows of a tile.  Plain geometry: tile k covers [kL, (k+1)L), each tile starting its forward
// elimination a halo earlier.  Grouped geometry (instances whose tiles are aligned to warps,
// flag bit 0): the 32 tiles of a warp cover 32L - kHaloB - kLane0Short consecutive rows.
//   * Every lane but the last takes the rows past its tile (the back substitution's start)
//     from the next lane's forward sweep; the last lane computes them, so its tile is kHaloB
//     rows shorter.
//   * Only the first lane runs a halo (its tile is kLane0Short rows shorter).  The others are
//     chained: they start at their first row with the exact c' (kHaloC rows of the c'
//     recurrence alone before it) and the guess d' = 0, and keep the sensitivity M_i of their
//     d'_i to the true d'_{s0-1}, which is linear: d'_i = d'_i(guess) + M_i d'_{s0-1}.  After
//     the sweep a warp scan over the lanes' affine maps gives every lane its d'_{s0-1}, and the
//     rows with |M_i| >= 2^-110 are corrected.
struct TileRows {
  long long s0, e0;
  bool succ;   // the next lane holds rows [e0, e0 + kHaloB) of its own forward sweep
  bool chain;  // chained start (see above)
};

__device__ __forceinline__ TileRows tile_rows_of(const Inst &I, long long tile) {
  const long long n = I.n, L = I.tile_rows;
  TileRows T;
  if (I.pad & 1) {
    const long long lane = tile & 31;
    const long long g0 = (tile >> 5) * (32 * L - kHaloB - kLane0Short);
    T.s0 = lane == 0 ? g0 : g0 + lane * L - kLane0Short;
    const long long len = lane == 0 ? L - kLane0Short : (lane == 31 ? L - kHaloB : L);
    T.e0 = min(T.s0 + len, n);
    T.succ = lane < 31 && T.e0 < n;
    T.chain = lane > 0;
  } else {
    T.s0 = tile * L;
    T.e0 = min(T.s0 + L, n);
    T.succ = false;
    T.chain = false;
  }
  return T;
}

// What the forward sweep hands to the lane scan.
struct FwdOut {
  long long rlast;  // last row of the sweep
  double A, B;      // d' of the tile's last row as computed, and its sensitivity M there
  int K;            // stored sensitivities (rows s0 .. s0+K-1)
  unsigned bad;     // input checks of the tile's rows
};

// Forward elimination of a tile (rows from the halo start, or from s0 when chained, to
// rlast) into the scratch.
__device__ FwdOut tile_forward(const Inst &I, const TileRows &T, const Scratch64 &S) {
  const long long n = I.n;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = T.s0, e0 = T.e0;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  unsigned bad = 0;  // input checks of the tile's rows, made as the forward sweep passes them
  // ---- 1. start: halo guess, or exact c'_{s0-1} for a chained tile ----
  long long r;
  double cp_start = 0.0;
  if (T.chain) {
    const long long i0 = max(s0 - 1 - kHaloC, 0LL);
    double c = (i0 == 0 && !nat0) ? 0.5 : 0.0;  // exact at row 0, a guess elsewhere
    double xb = x[i0 + 1];
    double hp = xb - x[i0];
    for (long long i = i0 + 1; i <= s0 - 1; ++i) {
      const double xc = x[i + 1];
      const double hi = xc - xb;
      c = hi * rcp64(twice(hp + hi) - hp * c);
      hp = hi;
      xb = xc;
    }
    cp_start = c;
    r = s0 - 1;
  } else {
    r = halo_start(x, n, s0);  // row whose (c', d') the state holds
  }
  Fwd64 F;
  F.hn = F.ihn = F.sn = 0.0;
  F.xl = F.yl = 0.0;
  // interval j (= r+1 of the state) when it exists: uses x_{j+1}, y_{j+1} (loaded one step
  // earlier) and issues the loads of x_{j+2}, y_{j+2} for the next step; row j is checked
  auto precompute_next = [&](long long j) {
    if (j <= n - 2) {
      const double x2 = F.xl, y2 = F.yl;
      if (j + 2 < n) {
        if (j + 18 < n) {
          if (first_in_block(x + j + 18)) prefetch_l1(x + j + 18);
          if (first_in_block(y + j + 18)) prefetch_l1(y + j + 18);
        }
        F.xl = x[j + 2];
        F.yl = y[j + 2];
      }
      if (j >= s0 && j < e0) bad |= row_check(F.xn, F.yn, true, x2);
      F.hn = x2 - F.xn;
      F.ihn = rcp64(F.hn);
      F.sn = quot64(y2 - F.yn, F.hn, F.ihn);
      F.xn = x2;
      F.yn = y2;
    } else if (j == n - 1 && j >= s0 && j < e0) {
      bad |= row_check(F.xn, F.yn, false, 0.0);
    }
  };
  {
    const double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    const double h = x1 - x0, ih = rcp64(h), sl = quot64(y1 - y0, h, ih);
    F.h = h; F.s = sl; F.xn = x1; F.yn = y1;
    if (T.chain) {                    // exact c'_{s0-1}, guess d'_{s0-1} = 0 (corrected later)
      F.cp = cp_start;
      F.dp = 0.0;
    } else if (r == 0 && !nat0) {     // clamped start: c'_0 = 1/2, d'_0 = 3(s_0 - y'_0)/h_0
      F.cp = 0.5;
      F.dp = 3.0 * (sl - I.yp1) * ih;
    } else {                          // natural start, or the halo guess
      F.cp = 0.0;
      F.dp = 0.0;
    }
    if (r >= s0) {                    // r == s0 == 0: row 0 is this tile's first row
      S.at(0, 0) = F.cp; S.at(0, 1) = F.dp; S.at(0, 2) = ih;
      bad |= row_check(x0, y0, true, x1);
    }
    if (r + 2 < n) {
      F.xl = x[r + 2];
      F.yl = y[r + 2];
    }
    precompute_next(r + 1);
  }
  FwdOut out;
  out.A = 0.0;
  out.B = 0.0;
  double M = 1.0;       // sensitivity of d'_r to d'_{s0-1} (chained tiles)
  int K = 0;
  bool track = T.chain;
  const long long rlast = T.succ ? e0 - 1 : min(e0 + kHaloB, n) - 1;
  while (r < rlast) {
    const long long j = r + 1;
    double cpj, dpj, ihj = 0.0, iden;
    const double a = F.h;  // a_j = h_{j-1}
    if (j <= n - 2) {
      const double hj = F.hn, sj = F.sn;
      ihj = F.ihn;
      const double den = twice(F.h + hj) - F.h * F.cp;
      iden = rcp64(den);
      cpj = hj * iden;
      dpj = (6.0 * (sj - F.s) - F.h * F.dp) * iden;
      F.h = hj; F.s = sj;
      precompute_next(j + 1);  // independent of the elimination chain above
    } else {  // j == n-1: last row
      cpj = 0.0;
      const double den = 2.0 * F.h - F.h * F.cp;
      iden = rcp64(den);
      dpj = nat1 ? 0.0 : (6.0 * (I.ypn - F.s) - F.h * F.dp) * iden;
    }
    F.cp = cpj; F.dp = dpj;
    r = j;
    if (j >= s0) {
      S.at(j - s0, 0) = cpj; S.at(j - s0, 1) = dpj; S.at(j - s0, 2) = ihj;
    }
    if (track) {  // d'_j = (r_j - a_j d'_{j-1}) / den_j: the sensitivity picks up -a_j / den_j
      M *= (j == n - 1 && nat1) ? 0.0 : -a * iden;
      S.m(K++) = M;
      const int ex = (int)((__double_as_longlong(M) >> 52) & 0x7FF);
      if (ex < 1023 - 110 || K == kMRows) track = false;
    }
    if (j == e0 - 1) {
      out.A = dpj;
      out.B = track ? M : 0.0;
    }
  }
  out.rlast = rlast;
  out.K = K;
  out.bad = bad;
  return out;
}

// Chained tile: add M_i d'_{s0-1} to the stored d' of its first K rows.
__device__ void tile_correct(const FwdOut &o, double delta, const Scratch64 &S) {
  for (int k = 0; k < o.K; ++k) S.at(k, 1) = fma(S.m(k), delta, S.at(k, 1));
}

// First query whose bracket index is >= s (first_query's result): the estimate
// floor((x_s - x_0) / step) from binary64 arithmetic (within one of the answer: the grid points
// are rounded sums) checked on the two grid points around it by their keys, with the bisection
// for a miss or non-finite operands.  Four grid points instead of ~2 log2(m).
__device__ __forceinline__ long long first_query_est(const Grid &G, double inv_step, const double *x, long long s) {
  if (s == 0 || G.m == 0) return 0;
  if (G.m >= 2) {
    const double v = x[s];
    const double e = (v - G.x0) * inv_step;
    if (finite64(v) && e > -2.0 && e < 9.0e15) {  // false for NaN
      const long long kv = dkey(v);
      long long k = max(min((long long)e, G.m - 1), -1LL);  // ~ the last grid point at or below v
      const bool lo_ok = k < 0 || dkey(G.at(k)) <= kv;
      const bool hi_ok = k + 1 >= G.m || dkey(G.at(k + 1)) > kv;
      if (lo_ok && hi_ok) return k + 1;
    }
  }
  return first_query(G, x, s);
}

// Back substitution from rlast (y''_{rlast} := d'_{rlast}, exact when rlast == n-1), fused
// with the evaluation: row t's y'' completes interval t, whose queries are evaluated right
// away, walking the grid downwards.  With T.succ the rows past the tile come from the next
// lane's scratch (rows it computed after its own halo).
__device__ void tile_backward_eval(const Inst &I, const TileRows &T, long long rlast, const Scratch64 &S) {
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = T.s0, e0 = T.e0;
  const long long te = e0 - 1 - s0;  // last row of the tile (local)
  double Y;
  long long t;
  if (T.succ) {
    const Scratch64 Sn{S.base, S.mb, S.lane + 1};  // the next lane's tile starts at row e0
    long long u = min(e0 + kHaloB, n) - 1 - e0;
    Y = Sn.at(u, 1);
    for (--u; u >= 0; --u) Y = Sn.at(u, 1) - Sn.at(u, 0) * Y;
    t = te;
  } else {
    const long long tl = rlast - s0;
    Y = S.at(tl, 1);
    t = tl - 1;
  {  // rows past the tile: the recurrence alone, loads of eight rows first
    constexpr int kB = 8;
    for (; t - (kB - 1) > te; t -= kB) {
      double cc[kB], dd[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        cc[u] = S.at(t - u, 0);
        dd[u] = S.at(t - u, 1);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) Y = dd[u] - cc[u] * Y;
    }
    for (; t > te; --t) Y = S.at(t, 1) - S.at(t, 0) * Y;
  }
  }
  // here Y = y''_{t+1}: y''_{e0} (t = te), or y''_{n-1} when the tile ends at row n-1 (t = te - 1)
  if (t == te - 1 && I.ypp) I.ypp[n - 1] = Y;

  // queries of the tile: k in [klo, khi], x_k > x_{s0} (first_query) and x_k <= x_{e0} when
  // e0 <= n-2; interval t takes those with x_t < x_k (the lowest interval all the rest).  The
  // loop runs one query per iteration, walking the rows down as far as the query needs, so
  // that the lanes of a warp do the same FP64 work per iteration whatever the spread of the
  // queries over their intervals.
  const bool evaluate = (m > 0 && s0 <= n - 2);
  const Grid G = make_grid(x, n, m);
  const double inv_step = (evaluate && m >= 2) ? rcp64(G.step) : 0.0;
  const long long klo = evaluate ? first_query_est(G, inv_step, x, s0) : 0;
  long long k = evaluate ? ((e0 <= n - 2) ? first_query_est(G, inv_step, x, e0) - 1 : m - 1) : -1;
  if (t < 0) return;  // a one-row tile at the end of the instance
  // current row t: y''_t (Yt), y''_{t+1} (Yt1), its knot, value, 1/h and width; the next row
  // down is loaded one step ahead
  double Yt1 = Y;
  double xt1 = x[s0 + t + 1], yt1 = y[s0 + t + 1];
  double xt = x[s0 + t], yt = y[s0 + t], iht = S.at(t, 2);
  double Yt = S.at(t, 1) - S.at(t, 0) * Yt1;
  if (I.ypp) I.ypp[s0 + t] = Yt;
  double c_n = 0.0, d_n = 0.0, ih_n = 0.0, x_n = 0.0, y_n = 0.0;
  auto load_next = [&](long long row) {  // row t-1
    if (row >= 0) {
      if (row >= 8) {
        prefetch_l1(&S.at(row - 8, 0)); prefetch_l1(&S.at(row - 8, 1)); prefetch_l1(&S.at(row - 8, 2));
        if (first_in_block(x + s0 + row - 8)) prefetch_l1(x + s0 + row - 8);
        if (first_in_block(y + s0 + row - 8)) prefetch_l1(y + s0 + row - 8);
      }
      c_n = S.at(row, 0); d_n = S.at(row, 1); ih_n = S.at(row, 2);
      x_n = x[s0 + row]; y_n = y[s0 + row];
    }
  };
  load_next(t - 1);
  auto step_down = [&]() {  // t -> t-1: one back-substitution step
    --t;
    Yt1 = Yt; xt1 = xt; yt1 = yt;
    xt = x_n; yt = y_n; iht = ih_n;
    Yt = d_n - c_n * Yt1;
    if (I.ypp) I.ypp[s0 + t] = Yt;
    load_next(t - 1);
  };
  long long kxt = dkey(xt);
  double q = k >= klo ? G.at(k) : 0.0;  // the next query is formed one iteration ahead
  for (; k >= klo; --k) {
    const long long kq = dkey(q);
    const double qn = k > klo ? G.at(k - 1) : 0.0;
    while (t > 0 && kq <= kxt) {
      step_down();
      kxt = dkey(xt);
    }
    I.yq[k] = newint64(q, xt, xt1, yt, yt1, Yt, Yt1, xt1 - xt, iht);
    if (I.jq) I.jq[k] = (int32_t)(s0 + t);
    q = qn;
  }
  while (t > 0) step_down();
}

// Persistent CTAs; each warp fetches 32 tiles at a time from a counter zeroed before the
// launch, so tiles of uneven length (ragged tails, small instances) balance across SMs.
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    fused_f64_kernel(const Inst *__restrict__ insts, int ninst, long long total_tiles,
                     unsigned long long *__restrict__ counter, double *__restrict__ scratch, long long rows_cap) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double *wbase = scratch + (size_t)warp * (rows_cap * kFields + kMRows) * 32;
  const Scratch64 S{wbase, wbase + (size_t)rows_cap * kFields * 32, (int)(threadIdx.x & 31)};
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total_tiles) break;
    const long long t = (long long)base + lane;
    // every lane takes part in the warp barriers and the scan; lanes without a tile, or with
    // an empty one, idle
    Inst I;
    TileRows T;
    T.s0 = T.e0 = 0;
    T.succ = T.chain = false;
    FwdOut o;
    o.rlast = -1;
    o.A = o.B = 0.0;
    o.K = 0;
    o.bad = 0;
    if (t < total_tiles) {
      const int i = find_inst(insts, ninst, t);
      I = insts[i];
      T = tile_rows_of(I, t - I.tile_begin);
      if (T.s0 < I.n) o = tile_forward(I, T, S);
    }
    // d'_{s0-1} of every chained lane: inclusive scan of the maps delta -> A + B delta (the
    // first lane of a group has B = 0), then the previous lane's result
    double sa = o.A, sb = o.B;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double pa = __shfl_up_sync(0xffffffffu, sa, off), pb = __shfl_up_sync(0xffffffffu, sb, off);
      if (lane >= off) {
        sa = fma(sb, pa, sa);
        sb *= pb;
      }
    }
    const double delta = __shfl_up_sync(0xffffffffu, sa, 1);
    if (o.rlast >= 0 && T.chain) tile_correct(o, delta, S);
    __syncwarp();  // the next lane's corrected forward rows are in the scratch
    if (o.rlast >= 0) {
      tile_backward_eval(I, T, o.rlast, S);
      if (o.bad) atomicOr(I.status, o.bad);
    }
    __syncwarp();  // the scratch is reused by the next batch of tiles
  }
}

size_t ring_bytes_f64(long long threads, int tile_rows) {
  const long long warps = (threads + 31) / 32;
  return (size_t)warps * (((size_t)tile_rows + kHaloB) * kFields + kMRows) * 32 * sizeof(double);
}

int f64_threads_per_sm() { return kThreads * kCtasPerSm; }

int overhang_rows_f64() { return kHaloB; }

int lane0_short_rows_f64() { return kLane0Short; }

long long threads_f64(int sm_count, long long total_tiles) {
  int blocks, bt;
  spread_grid(sm_count * kCtasPerSm, total_tiles, kThreads, &blocks, &bt);
  return (long long)blocks * bt;
}

cudaError_t launch_fused_f64(const Inst *d_insts, int ninst, long long total_tiles, double *scratch,
                             int tile_rows, int sm_count, unsigned long long *counter, cudaStream_t stream) {
  int blocks, bt;
  spread_grid(sm_count * kCtasPerSm, total_tiles, kThreads, &blocks, &bt);
  fused_f64_kernel<<<(unsigned)blocks, (unsigned)bt, 0, stream>>>(d_insts, ninst, total_tiles, counter, scratch,
                                                                  (long long)tile_rows + kHaloB);
  return cudaGetLastError();
}

}  // namespace spl
