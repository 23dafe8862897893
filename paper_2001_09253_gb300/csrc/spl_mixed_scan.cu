// Warp-cooperative binary32 fit + evaluation ("scan" form of the mixed-precision path).
//
// The binary32 path of every mixed-precision launch: the
// tridiagonal system of eq. (init_val) with the end rows of "Start and End Derivatives", the
// Thomas recurrences of "Implementation", and the one-division form of "Fast Interpolation" on
// the grid of "Curve Interpolation", in binary32 arithmetic on exact, once-rounded differences of
// the binary64 inputs.  A warp solves one tile of rows, kStepS = 128 consecutive rows per step, lane
// l holding the kVS = 4 consecutive rows R + 4l .. R + 4l + 3, so that the recurrences become a
// short sequential part inside each lane and a warp scan across the lanes:
//   * c'_j = c_j / (b_j - a_j c'_{j-1}) contracts an error in c'_{j-1} by at least 12 per row
//     (b = 2(a + c) and c' <= 1/2 give |dc'_j/dc'_{j-1}| = ac/(b - a c')^2 <= ac/(1.5a + 2c)^2
//     <= 1/12), so three relaxation passes over a lane's four rows, each starting from the
//     previous lane's output of the pass before (lane 0 from the carried c'_{R-1}), reach the
//     sequential values: the guess error 1/4 shrinks to 12^-8 / 4 < 2^-30 before the last pass;
//   * d'_j = (d_j - a_j d'_{j-1}) / den_j and the back substitution y''_j = d'_j - c'_j y''_{j+1}
//     are affine maps t -> A t + B: each lane composes its four, an inclusive warp scan (the
//     second one from the top lane down) composes the lanes', and each lane then applies its own
//     four maps to the value entering it;
//   * the queries of a step's intervals are evaluated 32 at a time, lane-parallel, from the top
//     query down: each finds its interval by a 5-step search over the lanes' first knots
//     (shuffles of order-preserving integer keys, so brackets stay bit-identical to the
//     sequential sweep) and a 3-key search among the four knots of that lane (shared memory).
// A tile starts its forward sweep kHaloS = 64 rows early from a guessed state (the guess error in
// d' decays by at most 2/3 per row: (2/3)^64 < 2^-37) and its back substitution kOvS = 32 rows
// past its end from y'' = 0 (the error decays by c' < 1/2 per row).  The forward results (c', d',
// binary32 width and value) of every row of the tile and its halo live in the warp's shared
// memory (16 bytes per row, transposed within a step so that lanes touch consecutive words); the
// back substitution overwrites (c', d') in place by what the evaluation needs besides the width and
// value (1/width, y''); no global scratch is used, so DRAM sees only the inputs and outputs.
#include <algorithm>
#include <atomic>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_mixed_math.cuh"
#include "spl_numeric.h"

namespace spl {

constexpr int kVS = 4;                 // consecutive rows per lane in a step
constexpr int kStepS = 32 * kVS;       // rows per warp step
constexpr int kHaloS = 64;             // forward rows before a tile
constexpr int kOvS = 32;               // back-substitution start past a tile
constexpr int kWarpsS = 20;            // warps per CTA (one CTA per SM; 12 / 16 / 20 measured: more is faster)
constexpr int kThreadsS = 32 * kWarpsS;
// The serving loop, which carries the scheduler and all three tile modes, runs 16 warps per SM: at
// 20 (96 registers) it spilled 408 bytes per thread; at 16 (128 registers) 124, with served
// latency p50 0.051 -> 0.043 ms and saturation 289k -> 336k requests/s on GB300 (12 warps: p50
// 0.041 ms, saturation 301k)
constexpr int kServeThreadsS = 32 * 16;
// longest tile the shared-memory scratch holds: 544 + the 64-row halo + the 32-row overlap = 640
// rows, five whole steps (512-row tiles used the same five steps for 608 rows: 6 % more steps per
// point; batched launches 21 % slower)
constexpr int kTileMaxS = 544;
constexpr int kRowsCapS = (kTileMaxS + kHaloS + kOvS + kStepS - 1) / kStepS * kStepS;
constexpr unsigned kFullS = 0xffffffffu;
constexpr long long kKeyInf = 0x7FF0000000000000LL;  // key of +inf: above every finite knot

// Shared memory of one warp.  w: per row of the tile's forward range, (c', d', h, y) after the
// forward sweep and (1/h, y'', h, y) after the back substitution; within each step of 128 rows the
// row R + 4l + v sits at v*32 + l.  keys: order-preserving keys of the knots of the current
// back-substitution step (same transposition), and of x_{R+128} at index 128.
struct ScanSmem {
  float4 w[kRowsCapS];
  long long keys[kStepS + 2];
};
constexpr size_t kSmemPerWarpS = sizeof(ScanSmem);

__device__ __forceinline__ double shfl_f64(double v, int src) {
  return __longlong_as_double(__shfl_sync(kFullS, __double_as_longlong(v), src));
}
__device__ __forceinline__ long long shfl_i64(long long v, int src) { return __shfl_sync(kFullS, v, src); }
__device__ __forceinline__ int wpos(int row_in_step) { return (row_in_step & 3) * 32 + (row_in_step >> 2); }

// Inverse of dkey (the -0 it folds comes back as +0).
__device__ __forceinline__ double key_to_double(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// kCG: through L2 only (ld.global.cg): the persistent serving loop reads buffers that other SMs,
// or earlier requests at the same addresses, may have left in this SM's L1.
template <bool kCG, typename T>
__device__ __forceinline__ T ldx(const T *p) {
  if (kCG) return __ldcg(p);
  return *p;
}

// Least k in [0, m] with x_k > v on the uniform grid, one value per lane: the estimate
// floor((v - x_0) / step) from binary64 arithmetic (within one of the answer: the grid points are
// rounded sums) checked on the two grid points around it by their keys, with a walk for the rare
// miss.  Lanes with need = false return 0 (their FP64 work is shared by the warp anyway).
__device__ __forceinline__ long long grid_first_above(const Grid &G, double inv_step, bool need, double v) {
  if (!need || G.m == 0) return 0;
  const long long kv = dkey(v);
  if (G.m == 1) return dkey(G.x0) <= kv ? 1 : 0;
  const double e = (v - G.x0) * inv_step;
  long long k = (e >= 0.0) ? (long long)e : -1;  // ~ the last grid point at or below v
  k = max(min(k, G.m - 1), -1LL);
  const bool lo_ok = k < 0 || dkey(G.at(k)) <= kv;
  const bool hi_ok = k + 1 >= G.m || dkey(G.at(k + 1)) > kv;
  if (lo_ok && hi_ok) return k + 1;
  long long kk = k + 1;
  while (kk > 0 && dkey(G.at(kk - 1)) > kv) --kk;
  while (kk < G.m && dkey(G.at(kk)) <= kv) ++kk;
  return kk;
}

// The uniform grid of the instance: x_0, x_{n-1}, step = (x_{n-1} - x_0)/(m - 1) as the correctly
// rounded quotient (quot64 equals the IEEE division bit for bit) and 1/step for estimates.
template <bool kCG>
__device__ __forceinline__ Grid grid_of(const double *x, long long n, long long m, double *inv_step) {
  Grid g;
  g.x0 = ldx<kCG>(x);
  g.xl = ldx<kCG>(x + n - 1);
  g.m = m;
  g.step = 0.0;
  *inv_step = 0.0;
  if (m >= 2) {
    const double den = i2d_exact(m - 1);
    g.step = quot64(g.xl - g.x0, den, rcp64(den));
    *inv_step = rcp64(g.step);
  }
  return g;
}

// Forward state carried from the last row of one step to the next: c', d', width and slope of
// the last row's interval (double-float in the refinement), and the refinement's Z.
struct CarryS {
  float c, d, z;
  F2 h, s;
};

// Loads of a lane's rows j0 .. j0+4 (the fifth is the next lane's first: the width and slope of
// the fourth row's interval need it).  `full`: every row exists.
template <bool kCG, typename T>
__device__ __forceinline__ void load5(const T *__restrict__ p, long long j0, long long n, bool full, T (&v)[kVS + 1]) {
  if (full) {
#pragma unroll
    for (int u = 0; u <= kVS; ++u) v[u] = ldx<kCG>(p + j0 + u);
  } else {
#pragma unroll
    for (int u = 0; u <= kVS; ++u) v[u] = (j0 + u < n) ? ldx<kCG>(p + j0 + u) : T(0);
  }
}

// Forward elimination of one step: rows R .. R+127 of the tile's forward range [f0, f1), written
// to the step's shared-memory slice.  kEdge: the step holds row 0, row n-1 or rows past f1 (or
// loads past n); otherwise every row is an interior row of the system.
// End conditions of an instance (section "Start and End Derivatives"), decided once per tile.
struct EndsS {
  bool nat0, nat1;
  float yp1, ypn;  // binary32 end slopes (clamped ends)
  F2 yp1F, ypnF;   // double-float end slopes (the refinement's residual)
};

template <int kMode, bool kEdge>
__device__ __forceinline__ void fwd_step(const Inst &I, const EndsS &E, long long R, long long f1, int lane,
                                         const double (&xv)[kVS + 1], const double (&yv)[kVS + 1],
                                         const float (&zv)[kVS + 1], CarryS &C, float4 *__restrict__ ws,
                                         unsigned &bad) {
  const long long n = I.n;
  const long long j0 = R + (long long)kVS * lane;
  const bool nat0 = E.nat0, nat1 = E.nat1;
  F2 h[kVS], s[kVS];
#pragma unroll
  for (int v = 0; v < kVS; ++v) {
    const long long j = j0 + v;
    const bool hasn = !kEdge || j <= n - 2;
    h[v] = F2{0.0f, 0.0f};
    s[v] = F2{0.0f, 0.0f};
    if (hasn) {
      if (kMode == 2) {
        // exact widths as double-floats (same binade: the integer ulp count), value differences
        // as the binary64 difference split in two (the rounding the binary64 slopes see too)
        if (!diff_up_f2(xv[v + 1], xv[v], &h[v])) h[v] = dif2_slow(xv[v + 1], xv[v]);
        F2 dy;
        if (!f64_to_f2(yv[v + 1] - yv[v], &dy)) dy = dif2_slow(yv[v + 1], yv[v]);
        s[v] = df_div(dy, h[v], rcp32(h[v].hi));
      } else {
        h[v].hi = dif32_up(xv[v + 1], xv[v]);
        s[v].hi = quot32(dy32(yv[v + 1], yv[v]), h[v].hi, rcp32(h[v].hi));
      }
    } else if (kEdge && j == n - 1 && !nat1) {
      // clamped last row: the interior row with a zero width above and the end slope in place
      // of the slope above (a = h_{n-2}, b = 2 h_{n-2}, c = 0, d = 6 (y'_n - s_{n-2}))
      s[v] = kMode == 2 ? E.ypnF : F2{E.ypn, 0.0f};
    }
    if (kMode != 2 && (!kEdge || j < f1)) bad |= row_check(xv[v], yv[v], hasn, xv[v + 1]);
  }
  // the interval below the lane's first row: the previous lane's last, or the carry
  F2 hm{__shfl_up_sync(kFullS, h[kVS - 1].hi, 1), 0.0f}, sm{__shfl_up_sync(kFullS, s[kVS - 1].hi, 1), 0.0f};
  float zm = 0.0f;
  if (kMode == 2) {
    hm.lo = __shfl_up_sync(kFullS, h[kVS - 1].lo, 1);
    sm.lo = __shfl_up_sync(kFullS, s[kVS - 1].lo, 1);
    zm = __shfl_up_sync(kFullS, zv[kVS - 1], 1);
  }
  if (lane == 0) {
    hm = C.h;
    sm = C.s;
    zm = C.z;
  }
  // rows: a y''_{j-1} + b y''_j + c y''_{j+1} = d (the refinement: the same matrix, d the residual)
  float a[kVS], b[kVS], c[kVS], d[kVS];
#pragma unroll
  for (int v = 0; v < kVS; ++v) {
    const F2 hp = v ? h[v - 1] : hm, sp = v ? s[v - 1] : sm;
    a[v] = hp.hi;
    c[v] = h[v].hi;
    b[v] = 2.0f * (hp.hi + h[v].hi);
    if (kMode == 2) {
      const float z0 = zv[v], z1 = zv[v + 1], zp = v ? zv[v - 1] : zm;
      const F2 dd = df_mul_f(df_add(s[v], df_neg(sp)), 6.0f);
      const F2 az = df_add(df_add(df_mul_f(hp, zp), df_mul_f(df_add(hp, h[v]), 2.0f * z0)), df_mul_f(h[v], z1));
      const F2 res = df_add(dd, df_neg(az));
      d[v] = res.hi + res.lo;
    } else {
      d[v] = 6.0f * (s[v].hi - sp.hi);
    }
    if (kEdge) {
      // identity rows: natural ends (y'' = 0: the refinement's correction is -Z there) and the
      // rows past the sweep; the clamped end rows are general rows (see above and the carry)
      const long long j = j0 + v;
      if (j >= f1 || (j == 0 && nat0) || (j == n - 1 && nat1)) {
        a[v] = 0.0f;
        b[v] = 1.0f;
        c[v] = 0.0f;
        d[v] = (kMode == 2 && j < f1) ? -zv[v] : 0.0f;
      }
    }
  }
  // c' by relaxation (see the file header): two passes from the guess 1/4 with the MUFU
  // reciprocal alone, the third with the refined reciprocal that the d' step uses
  float t = (lane == 0) ? C.c : 0.25f;
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int v = 0; v < kVS; ++v) t = c[v] * rcp_approx32(fmaf(-a[v], t, b[v]));
    t = __shfl_up_sync(kFullS, t, 1);
    if (lane == 0) t = C.c;
  }
  float cp[kVS], iden[kVS];
#pragma unroll
  for (int v = 0; v < kVS; ++v) {
    iden[v] = rcp32(fmaf(-a[v], t, b[v]));
    cp[v] = c[v] * iden[v];
    t = cp[v];
  }
  // d': the maps t -> A t + B of the lane's rows, composed, scanned over the lanes, applied
  float A[kVS], B[kVS];
#pragma unroll
  for (int v = 0; v < kVS; ++v) {
    A[v] = -a[v] * iden[v];
    B[v] = d[v] * iden[v];
  }
  float PA = A[0], PB = B[0];
#pragma unroll
  for (int v = 1; v < kVS; ++v) {
    PB = fmaf(A[v], PB, B[v]);
    PA *= A[v];
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float A2 = __shfl_up_sync(kFullS, PA, off), B2 = __shfl_up_sync(kFullS, PB, off);
    if (lane >= off) {
      PB = fmaf(PA, B2, PB);
      PA *= A2;
    }
  }
  const float tA = __shfl_up_sync(kFullS, PA, 1), tB = __shfl_up_sync(kFullS, PB, 1);
  float dpv = (lane == 0) ? C.d : fmaf(tA, C.d, tB);
  float dp[kVS];
#pragma unroll
  for (int v = 0; v < kVS; ++v) {
    dp[v] = fmaf(A[v], dpv, B[v]);
    dpv = dp[v];
  }
#pragma unroll
  for (int v = 0; v < kVS; ++v)
    ws[v * 32 + lane] = make_float4(cp[v], dp[v], h[v].hi, kMode == 1 ? 0.0f : to_f32(yv[v]));
  C.c = __shfl_sync(kFullS, cp[kVS - 1], 31);
  C.d = __shfl_sync(kFullS, dp[kVS - 1], 31);
  C.h.hi = __shfl_sync(kFullS, h[kVS - 1].hi, 31);
  C.s.hi = __shfl_sync(kFullS, s[kVS - 1].hi, 31);
  if (kMode == 2) {
    C.h.lo = __shfl_sync(kFullS, h[kVS - 1].lo, 31);
    C.s.lo = __shfl_sync(kFullS, s[kVS - 1].lo, 31);
    C.z = __shfl_sync(kFullS, zv[kVS - 1], 31);
  }
}

// One tile: rows [s0, e0) of instance I.  kMode 0: fit + evaluation; 1: fit only, the binary32
// y'' to I.z (first pass of the refined path); 2: one refinement step of I.z (the residual
// r = d - A Z in double-float arithmetic from exact double-float widths and value differences,
// A delta = r solved with the binary32 matrix), y'' = Z + delta, and the evaluation.
template <int kMode, bool kCG = false>
__device__ void scan_tile(const Inst &I, long long tile, ScanSmem &S, int lane) {
  const long long n = I.n, TR = I.tile_rows;
  if (TR < 1 || TR > kTileMaxS) {  // never launched by the host: the scratch would not hold it
    if (lane == 0) atomicOr(I.status, kStBadTile);
    return;
  }
  const long long s0 = tile * TR, e0 = min(s0 + TR, n);
  const long long f0 = max(s0 - kHaloS, 0LL), f1 = min(e0 + kOvS, n);
  const int nsteps = (int)((f1 - f0 + kStepS - 1) / kStepS);
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const float *__restrict__ z = I.z;
  unsigned bad = 0;
  EndsS E;
  E.nat0 = is_natural(I.yp1);
  E.nat1 = is_natural(I.ypn);
  E.yp1 = E.nat0 ? 0.0f : to_f32(I.yp1);
  E.ypn = E.nat1 ? 0.0f : to_f32(I.ypn);
  E.yp1F = (kMode == 2 && !E.nat0) ? f2_of(I.yp1) : F2{0.0f, 0.0f};
  E.ypnF = (kMode == 2 && !E.nat1) ? f2_of(I.ypn) : F2{0.0f, 0.0f};

  // ---- forward sweep, rows f0 .. f1-1, one step of 128 rows at a time; loads one step ahead ----
  // The carry into row f0: zero width below row 0 and, for a clamped first row, the end slope in
  // place of the slope below, which makes row 0 the general row a = 0, b = 2 h_0, c = h_0,
  // d = 6 (s_0 - y'_1) (section "Start and End Derivatives").
  CarryS C;
  C.c = C.d = C.z = 0.0f;
  C.h = C.s = F2{0.0f, 0.0f};
  if (f0 == 0 && !E.nat0) C.s = kMode == 2 ? E.yp1F : F2{E.yp1, 0.0f};
  double xn[kVS + 1], yn[kVS + 1];
  float zn[kVS + 1];
  {
    const long long j0 = f0 + (long long)kVS * lane;
    const bool full = f0 + kStepS + 1 <= n;
    load5<kCG>(x, j0, n, full, xn);
    load5<kCG>(y, j0, n, full, yn);
    if (kMode == 2) load5<kCG>(z, j0, n, full, zn);
  }
  for (int st = 0; st < nsteps; ++st) {
    const long long R = f0 + (long long)st * kStepS;
    double xv[kVS + 1], yv[kVS + 1];
    float zv[kVS + 1];
#pragma unroll
    for (int u = 0; u <= kVS; ++u) {
      xv[u] = xn[u];
      yv[u] = yn[u];
      zv[u] = kMode == 2 ? zn[u] : 0.0f;
    }
    if (st + 1 < nsteps) {
      const long long Rn = R + kStepS, j0 = Rn + (long long)kVS * lane;
      const bool full = Rn + kStepS + 1 <= n;
      load5<kCG>(x, j0, n, full, xn);
      load5<kCG>(y, j0, n, full, yn);
      if (kMode == 2) load5<kCG>(z, j0, n, full, zn);
    }
    float4 *ws = S.w + st * kStepS;
    const bool edge = R == 0 || R + kStepS > f1 || R + kStepS + 1 > n;
    // the refinement pass keeps one copy of its (long, double-float) step, with the edge checks:
    // two copies overflowed the instruction cache when warps sat in different phases (batched
    // launches: "no instruction" stalls 12 per issue)
    if (kMode == 2 || edge) fwd_step<kMode, true>(I, E, R, f1, lane, xv, yv, zv, C, ws, bad);
    else fwd_step<kMode, false>(I, E, R, f1, lane, xv, yv, zv, C, ws, bad);
  }
  __syncwarp();

  // ---- back substitution from row f1-1 down to s0, step by step, fused with the evaluation ----
  const long long m = I.m;
  const bool evaluate = kMode != 1 && m > 0 && s0 <= n - 2;
  Grid G;
  G.x0 = G.xl = G.step = 0.0;
  G.m = 0;
  const int st_lo = (int)((s0 - f0) / kStepS);
  // First query above the lowest knot of each step's intervals (lane s, steps above the bottom
  // one), above x_{s0} (lane st_lo: the tile's first query) and above x_{e0} (lane 31: past the
  // tile's last query), all at once; the queries of step s are [bnd_s, bnd of the step above).
  long long bnd = 0, klo = 0, khi = 0;
  if (evaluate) {
    double inv_step;
    G = grid_of<kCG>(x, n, m, &inv_step);
    bool need = false;
    long long r = 0;
    if (lane == 31) {
      r = e0;
      need = e0 < n - 1;
    } else if (lane >= st_lo && lane < nsteps) {
      r = max(f0 + (long long)lane * kStepS, s0);
      need = r > 0 && r < min(e0, n - 1);
    }
    const double v = need ? ldx<kCG>(x + r) : 0.0;
    need = need && finite64(v);
    bnd = grid_first_above(G, inv_step, need, v);
    if (lane == 31 && e0 >= n - 1) bnd = m;
    khi = __shfl_sync(kFullS, bnd, 31);
    klo = min(__shfl_sync(kFullS, bnd, st_lo), khi);
  }

  float ycarry = 0.0f;  // value of the recurrence at the row above the step (a guess above f1-1)
  double xb[kVS + 1];
  float zb[kVS + 1];
  {
    const long long j0 = f0 + (long long)(nsteps - 1) * kStepS + (long long)kVS * lane;
    if (evaluate) load5<kCG>(x, j0, n, false, xb);
    if (kMode == 2) load5<kCG>(z, j0, n, false, zb);
  }
  for (int st = nsteps - 1; st >= st_lo; --st) {
    const long long R = f0 + (long long)st * kStepS;
    const long long j0 = R + (long long)kVS * lane;
    double xc[kVS + 1];
    float zc[kVS + 1];
#pragma unroll
    for (int u = 0; u <= kVS; ++u) {
      xc[u] = evaluate ? xb[u] : 0.0;
      zc[u] = kMode == 2 ? zb[u] : 0.0f;
    }
    if (st > st_lo) {  // the step below lies inside the forward range: every row exists
      const long long jb = j0 - kStepS;
      if (evaluate) load5<kCG>(x, jb, n, true, xb);
      if (kMode == 2) load5<kCG>(z, jb, n, true, zb);
    }
    float4 *ws = S.w + st * kStepS;
    float4 cd[kVS];
#pragma unroll
    for (int v = 0; v < kVS; ++v) cd[v] = ws[v * 32 + lane];
    float A[kVS], B[kVS];
#pragma unroll
    for (int v = 0; v < kVS; ++v) {
      const bool act = j0 + v < f1;
      A[v] = act ? -cd[v].x : 1.0f;
      B[v] = act ? cd[v].y : 0.0f;
    }
    // the lane's maps composed from its top row down, then a suffix scan over the lanes
    float FA = A[kVS - 1], FB = B[kVS - 1];
#pragma unroll
    for (int v = kVS - 2; v >= 0; --v) {
      FB = fmaf(A[v], FB, B[v]);
      FA *= A[v];
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float A2 = __shfl_down_sync(kFullS, FA, off), B2 = __shfl_down_sync(kFullS, FB, off);
      if (lane + off < 32) {
        FB = fmaf(FA, B2, FB);
        FA *= A2;
      }
    }
    const float tA = __shfl_down_sync(kFullS, FA, 1), tB = __shfl_down_sync(kFullS, FB, 1);
    float tv = (lane == 31) ? ycarry : fmaf(tA, ycarry, tB);
    float val[kVS];  // y''_j, or the correction delta_j of the refinement
#pragma unroll
    for (int v = kVS - 1; v >= 0; --v) {
      val[v] = fmaf(A[v], tv, B[v]);
      tv = val[v];
    }
    ycarry = __shfl_sync(kFullS, val[0], 0);
    // outputs of the tile's own rows
#pragma unroll
    for (int v = 0; v < kVS; ++v) {
      const long long j = j0 + v;
      if (j >= s0 && j < e0) {
        if (kMode == 1) I.z[j] = val[v];
        // widened by the hardware conversion (exact): measured faster than the integer-pipe route
        // here, whose code, repeated per row, weighs on the instruction cache in batched launches
        else if (I.ypp) I.ypp[j] = kMode == 2 ? (double)zc[v] + (double)val[v] : (double)val[v];
      }
    }
    if (!evaluate) continue;
    // what the evaluation needs, in place: (1/width, y'') over (c', d'), next to the width and
    // value the forward sweep left; and the step's knot keys
#pragma unroll
    for (int v = 0; v < kVS; ++v) {
      const float pp = kMode == 2 ? zc[v] + val[v] : val[v];
      const float hh = cd[v].z;
      reinterpret_cast<float2 *>(ws + v * 32 + lane)[0] = make_float2(hh > 0.0f ? rcp32(hh) : 0.0f, pp);
      S.keys[v * 32 + lane] = (j0 + v < n) ? dkey(xc[v]) : kKeyInf;
    }
    if (lane == 31) S.keys[kStepS] = (j0 + kVS < n) ? dkey(xc[kVS]) : kKeyInf;
    __syncwarp();
    const long long ilo = max(R, s0), ihi = min(min(R + kStepS, e0), n - 1);
    if (ihi > ilo) {
      // queries of this step's intervals: [kb0, khi), khi carried from the step above; the
      // queries below kb0 (q <= x_ilo) belong to the steps below
      const long long kb0 = (ilo == s0) ? klo : max(min(__shfl_sync(kFullS, bnd, st), khi), klo);
      const long long K0 = S.keys[lane];  // key of the lane's first knot (row R + 4 lane)
      const int imin = (int)(ilo - R), imax = (int)(ihi - R) - 1;
      const float4 *wst = S.w + st * kStepS;
      const float4 *wup = wst + kStepS;  // row R + 128 (the step above): right end of interval R + 127
      // one query per lane and round, every lane through every shuffle; stores only for k < khi.
      // (Two queries per lane and round measured slower: the longer loop body costs more in
      // instruction fetch, with warps in different phases, than the second chain hides.)
      for (long long kb = kb0; kb < khi; kb += 32) {
        const long long kk = kb + lane;
        const double q = G.at(min(kk, khi - 1));
        const long long kq = dkey(q);
        // interval: largest i in [imin, imax] with x_{R+i} < q; first the lane among the
        // lanes' first knots, then the row among that lane's four
        int L = 0;
#pragma unroll
        for (int stp = 16; stp >= 1; stp >>= 1) {
          const long long kc = shfl_i64(K0, L + stp);
          if (kc < kq) L += stp;
        }
        int i = 4 * L;
#pragma unroll
        for (int v = 1; v < kVS; ++v) i += (S.keys[v * 32 + L] < kq) ? 1 : 0;
        i = max(min(i, imax), imin);
        if (kk < khi) {
          const float4 wj = wst[wpos(i)];
          const float4 wj1 = (i + 1 < kStepS) ? wst[wpos(i + 1)] : wup[0];
          const double xj = key_to_double(S.keys[wpos(i)]);
          const float xa = dif32_up(q, xj);
          I.yq[kk] = (double)newint32(xa, wj.z - xa, wj.w, wj1.w, wj.y, wj1.y, wj.z, wj.x);
          if (I.jq) I.jq[kk] = (int32_t)(R + i);
        }
      }
      khi = kb0;
    }
    __syncwarp();
  }
  if (bad) atomicOr(I.status, bad);
}

template <int kMode>
__global__ void __launch_bounds__(kThreadsS, 1)
    mixed_scan_kernel(const Inst *__restrict__ insts, int ninst, long long total_tiles,
                      unsigned long long *__restrict__ counter, const Inst one) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  ScanSmem &S = reinterpret_cast<ScanSmem *>(smem_raw)[threadIdx.x >> 5];
  const unsigned long long last_claim = (unsigned long long)total_tiles + gridDim.x * (blockDim.x >> 5) - 1;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) {
      t = atomicAdd(counter, 1ull);
      // every warp ends with one claim past the tiles, so the claim numbered last_claim is the
      // launch's final operation on the counter: it leaves the counter at zero for the next launch
      if (t == last_claim) atomicExch(counter, 0ull);
    }
    t = __shfl_sync(kFullS, t, 0);
    if ((long long)t >= total_tiles) break;
    const Inst I = insts ? insts[find_inst(insts, ninst, (long long)t)] : one;
    scan_tile<kMode>(I, (long long)t - I.tile_begin, S, lane);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// Persistent serving loop (continuous batching).  Warp 0 of CTA 0 is the scheduler: it reads
// request entries that the host appends to a ring in mapped host memory, installs each in its
// device slot, maps the request's tiles into the device tile map and publishes them by
// advancing `published`.  Every other warp is a worker: it claims one tile ticket at a time and,
// once the ticket is published, solves that tile of that request with the warp-cooperative
// binary32 fit + evaluation above (scan_tile<0>, in the warp's own shared memory).  The warp
// finishing a request's last tile writes the request's status and sequence number to mapped host
// memory.  All waits are bounded: the scheduler leaves after `idle_ns` without work or at
// `deadline_ns`, and sets `stop`; workers leave once stop is set and every published tile is
// claimed.  The host relaunches the loop when new work arrives.  Launched cooperatively (one CTA
// per SM), so the scheduler and the workers are co-resident.
// Tile tickets of a served request: its tiles once, or twice with refinement (first pass, then
// the refinement pass with the evaluation).
__device__ __forceinline__ unsigned long long serve_tickets(const Inst &I) {
  return (unsigned long long)I.ntiles * ((I.pad & kServeRefined) ? 2ull : 1ull);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kServeThreadsS, 1) serve_kernel(ServeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const bool scheduler = (blockIdx.x == 0 && threadIdx.x < 32);
  const unsigned long long t_start = globaltimer_ns();
  volatile unsigned long long *published = a.published;
  volatile unsigned *stop = a.stop;

  if (scheduler && (a.fault_flags & 1u)) return;  // failure-detection tests: no work is published
  if (scheduler) {
    ScanSmem &S0 = reinterpret_cast<ScanSmem *>(smem_raw)[0];  // this warp's slot (never a worker's)
    unsigned long long consumed = *a.consumed;
    unsigned long long last_work = t_start;
    unsigned sleep_ns = 64;
    if (lane == 0) *a.h_alive = 1u;
    for (;;) {
      const unsigned long long tail = *a.h_tail;
      if (consumed < tail) {
        __threadfence_system();  // the entries were written before the tail: read them after
        // up to kRingBatch entries per round trip to mapped host memory: every 8-byte word of the
        // batch is loaded at once (lane l: words l, l + 32, ...) into this warp's shared memory,
        // which no worker uses, then the entries are installed one by one
        constexpr int kWords = (int)(sizeof(ServeEntry) / 8);
        constexpr int kRingBatch = 16;
        static_assert(kRingBatch * kWords * 8 <= (int)sizeof(((ScanSmem *)0)->w), "ring batch fits the warp's buffer");
        unsigned long long *buf = reinterpret_cast<unsigned long long *>(S0.w);
        const int avail = (int)min(tail - consumed, (unsigned long long)kRingBatch);
        const int total = avail * kWords;
#pragma unroll 4
        for (int idx = lane; idx < total; idx += 32) {
          const int e = idx / kWords, w = idx - e * kWords;
          const volatile unsigned long long *src =
              reinterpret_cast<const volatile unsigned long long *>(a.h_ring + ((consumed + e) % a.rcap));
          buf[idx] = src[w];
        }
        __syncwarp();
        for (int e = 0; e < avail; ++e) {
          ServeEntry ent;
          unsigned long long *dst = reinterpret_cast<unsigned long long *>(&ent);
          for (int w = 0; w < kWords; ++w) dst[w] = buf[e * kWords + w];
          const unsigned slot = ent.slot;
          if (lane == 0) {
            ent.inst.status = a.slot_status + slot;
            a.slot_inst[slot] = ent.inst;
            a.slot_first[slot] = ent.first_tile;
            a.slot_done[slot] = 0u;
            a.slot_status[slot] = 0u;
            a.slot_seq[slot] = ent.seq;
          }
          const unsigned long long nt = serve_tickets(ent.inst);
          for (unsigned long long i = lane; i < nt; i += 32) a.tile_slot[(ent.first_tile + i) % a.tile_cap] = slot;
          __threadfence();
          __syncwarp();
          if (lane == 0) *published = ent.first_tile + nt;
        }
        consumed += (unsigned long long)avail;
        if (lane == 0) {
          *a.consumed = consumed;
          *a.h_consumed = consumed;
          __threadfence_system();
        }
        __syncwarp();
        last_work = globaltimer_ns();
        sleep_ns = 64;
        continue;
      }
      const unsigned long long now = globaltimer_ns();
      if (*a.h_stop || now - last_work > a.idle_ns || now - t_start > a.deadline_ns) break;
      __nanosleep(sleep_ns);
      if (sleep_ns < 2048) sleep_ns <<= 1;
    }
    if (lane == 0) {
      *stop = 1u;
      __threadfence();
    }
    return;
  }

  // workers: one ticket per warp; lane 0 waits for it (bounded) and the warp solves the tile.
  // SM 0 runs the scheduler alone: beside busy worker warps its installs slowed down exactly
  // when the workers were loaded (saturation 272k -> 288k requests/s without them)
  if (blockIdx.x == 0) return;
  ScanSmem &S = reinterpret_cast<ScanSmem *>(smem_raw)[threadIdx.x >> 5];
  for (;;) {
    unsigned long long t = 0;
    int state = 0;  // 1: the ticket is published; 2: no more work
    if (lane == 0) {
      t = atomicAdd(a.claimed, 1ull);
      unsigned sleep_ns = 64;
      for (;;) {
        if (*published > t) {
          state = 1;
          break;
        }
        if (*stop) {
          __threadfence();
          state = (*published > t) ? 1 : 2;
          break;
        }
        if (globaltimer_ns() - t_start > a.deadline_ns + 1000000000ull) {  // the scheduler stops first
          atomicOr(a.err, 1u);
          state = 2;
          break;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 4096) sleep_ns <<= 1;
      }
      __threadfence();
    }
    __syncwarp();
    state = __shfl_sync(0xffffffffu, state, 0);
    if (state != 1) break;
    t = __shfl_sync(0xffffffffu, t, 0);
    __threadfence();
    // the slot's entries were written by the scheduler after this SM may have cached an earlier
    // request's: read them from L2 (a slot is reused once its request completes)
    const unsigned slot = __ldcg(a.tile_slot + t % a.tile_cap);
    static_assert(sizeof(Inst) % 8 == 0, "Inst is copied in 8-byte words");
    Inst I;
    {
      const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.slot_inst + slot);
      unsigned long long *dst = reinterpret_cast<unsigned long long *>(&I);
#pragma unroll
      for (int w = 0; w < (int)(sizeof(Inst) / 8); ++w) dst[w] = __ldcg(src + w);
    }
    const long long local = (long long)(t - __ldcg(a.slot_first + slot));
    bool ok = true;
    if (!(I.pad & kServeRefined)) {
      scan_tile<0, true>(I, local, S, lane);
    } else if (local < I.ntiles) {  // refinement, first pass: binary32 y'' into the request's Z
      scan_tile<1, true>(I, local, S, lane);
    } else {
      // second pass: once every first-pass tile of the request is done (its tiles were claimed
      // before this one and never wait, so this wait ends; it is bounded all the same)
      if (lane == 0) {
        unsigned sleep_ns = 32;
        while (*(volatile unsigned *)(a.slot_done + slot) < (unsigned)I.ntiles) {
          if (globaltimer_ns() - t_start > a.deadline_ns + 1000000000ull) {
            atomicOr(a.err, 1u);
            ok = false;
            break;
          }
          __nanosleep(sleep_ns);
          if (sleep_ns < 1024) sleep_ns <<= 1;
        }
        __threadfence();
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      __syncwarp();
      if (ok) scan_tile<2, true>(I, local - I.ntiles, S, lane);
    }
    if (!ok) continue;  // the loop's error flag is raised: the host times the request out
    __threadfence();
    __syncwarp();
    if (lane == 0) {
      const unsigned done = atomicAdd(a.slot_done + slot, 1u) + 1u;
      if (done == (unsigned)serve_tickets(I)) {
        __threadfence();
        const unsigned st = *(volatile unsigned *)(a.slot_status + slot);
        a.h_done[2 * slot] = st;
        __threadfence_system();
        a.h_done[2 * slot + 1] = __ldcg(a.slot_seq + slot);
        __threadfence_system();
      }
    }
    __syncwarp();
  }
}

namespace {
// The kernels take more than the default 48 KB of dynamic shared memory: allowed once per device
// (the attribute belongs to the device's context).
constexpr int kMaxDevS = 64;
std::atomic<unsigned> g_smem_ok[kMaxDevS];
cudaError_t allow_smem() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevS && g_smem_ok[dev].load(std::memory_order_acquire)) return cudaSuccess;
  const int bytes = (int)(kSmemPerWarpS * kWarpsS);
  e = cudaFuncSetAttribute(mixed_scan_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mixed_scan_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mixed_scan_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevS) g_smem_ok[dev].store(1u, std::memory_order_release);
  return e;
}
}  // namespace

cudaError_t launch_serve(const ServeArgs &args, int sm_count, cudaStream_t stream) {
  const cudaError_t attr = allow_smem();
  if (attr != cudaSuccess) return attr;
  ServeArgs copy = args;
  void *params[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)serve_kernel, dim3((unsigned)sm_count), dim3(kServeThreadsS), params,
                                     kSmemPerWarpS * (kServeThreadsS / 32), stream);
}

int serve_tile_rows(int tile_rows) {
  return std::min(kTileMaxS, std::max(32, (tile_rows + 31) / 32 * 32));
}
int serve_tile_max() { return kTileMaxS; }

int scan_mixed_threads_per_sm() { return kThreadsS; }
int scan_mixed_tile_max() { return kTileMaxS; }

// rows of one tile: a multiple of 32, at most the shared-memory capacity.  One instance of at most
// 32 rows per resident warp: 32-row tiles, one wave of tiles of a single 128-row step each (with
// the halo and the overlap; latency of one refined request up to 3e4 knots 0.030 -> 0.022 ms on
// GB300); larger ones about two tiles per resident warp, of at least 128 rows (shorter tiles
// there need a second wave: 0.037 -> 0.055 ms at 3e5 knots).
int scan_mixed_tile_rows(long long total_points, int sm_count, int count) {
  const long long warps = (long long)sm_count * kWarpsS;
  if (count == 1 && total_points <= 32 * warps) return 32;
  long long L = count > 1 ? kTileMaxS : (total_points + 2 * warps - 1) / (2 * warps);
  L = (L + 31) / 32 * 32;
  return (int)std::max<long long>(std::min<long long>(L, kTileMaxS), 128);
}

long long threads_scan_mixed(int sm_count, long long total_tiles) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles * 32, kThreadsS, &blocks, &bt);
  return (long long)blocks * bt;
}

cudaError_t launch_scan_mixed(const Inst *d_insts, const Inst *h_one, int ninst, long long total_tiles, int sm_count,
                              unsigned long long *counter, cudaStream_t stream, int mode) {
  if ((!d_insts && (!h_one || ninst != 1)) || !counter) return cudaErrorInvalidValue;
  const cudaError_t attr = allow_smem();
  if (attr != cudaSuccess) return attr;
  int blocks, bt;
  spread_grid(sm_count, total_tiles * 32, kThreadsS, &blocks, &bt);
  const size_t smem = kSmemPerWarpS * (size_t)(bt / 32);
  Inst one{};
  if (!d_insts) one = *h_one;
  const dim3 g((unsigned)blocks), b((unsigned)bt);
  switch (mode) {
    case 1: mixed_scan_kernel<1><<<g, b, smem, stream>>>(d_insts, ninst, total_tiles, counter, one); break;
    case 2: mixed_scan_kernel<2><<<g, b, smem, stream>>>(d_insts, ninst, total_tiles, counter, one); break;
    default: mixed_scan_kernel<0><<<g, b, smem, stream>>>(d_insts, ninst, total_tiles, counter, one); break;
  }
  return cudaGetLastError();
}

}  // namespace spl
