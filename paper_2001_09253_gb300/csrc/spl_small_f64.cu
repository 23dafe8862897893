// Plain FP64 fit + evaluation of one small instance by one CTA (latency path).
//
// Same system and arithmetic as the fused FP64 kernel (spl_fused_f64.cu): the tridiagonal system
// of eq. (init_val) with the end rows of "Start and End Derivatives", Thomas' recurrences of
// "Implementation", the one-division form of "Fast Interpolation" on the grid of "Curve
// Interpolation"; slopes as correctly rounded quotients, brackets on integer keys.
//
// On this part a warp's FP64 instruction holds its sub-partition's FP64 unit for ~64 cycles, so a
// small instance's time is the FP64 chain of its longest thread.  Here the instance's rows are cut
// into kThreadsSF pieces of L = ceil(n / kThreadsSF) rows (8 at n = 1,000), one per thread of one
// CTA (one warp per sub-partition), and every recurrence is split the same way:
//   * c'_j: each thread runs the c' recurrence alone over the kWarmSF rows before its piece from a
//     guess (an error in c' shrinks 12-fold per row: 12^-16 < 2^-57) and then over its own rows;
//   * d'_j: each thread runs its rows from the guess d'_{s-1} = 0, recording the sensitivity M_j of
//     d'_j to the true d'_{s-1} (d' is affine in it); a block scan of the pieces' affine maps gives
//     every thread its true d'_{s-1}, and the stored d' are corrected (d'_j += M_j d'_{s-1});
//   * y''_j = d'_j - c'_j y''_{j+1}: each piece composes its rows into one affine map of the value
//     above it; a block scan from the last piece down gives every piece y'' of the row above it;
//   * each thread then back-substitutes and evaluates the queries of its own intervals.
// The rows' c', d' (then y'') and sensitivities live in shared memory (kMaxRowsSF rows).
#include <algorithm>
#include <atomic>

#include "spl_device.cuh"
#include "spl_internal.h"

namespace spl {

constexpr int kThreadsSF = 128;   // one warp per sub-partition
constexpr int kWarpsSF = kThreadsSF / 32;
constexpr int kMaxRowsSF = 4096;  // rows the shared memory holds
constexpr int kWarmSF = 16;       // c'-only rows before a piece

struct SmallSmem {
  double cp[kMaxRowsSF], dp[kMaxRowsSF], mm[kMaxRowsSF];
  double wa[kWarpsSF], wb[kWarpsSF];  // per-warp totals of the block scans
  long long kfirst[kThreadsSF + 1];   // first query of each piece
  double step, inv_step;
};

// Row j's coefficients a, b, c and right-hand side d (section "Generating Second Derivatives"
// and the end rows of "Start and End Derivatives"); hm, h: widths of intervals j-1 and j; sm, s:
// their slopes (only those that exist are read).
struct Row64 {
  double a, b, c, d;
};
__device__ __forceinline__ Row64 row64(long long j, long long n, bool nat0, bool nat1, double yp1, double ypn,
                                       double hm, double h, double sm, double s) {
  Row64 r;
  if (j == 0) {
    r.a = 0.0;
    if (nat0) { r.b = 1.0; r.c = 0.0; r.d = 0.0; }
    else { r.b = 2.0 * h; r.c = h; r.d = 6.0 * (s - yp1); }
  } else if (j == n - 1) {
    r.c = 0.0;
    if (nat1) { r.a = 0.0; r.b = 1.0; r.d = 0.0; }
    else { r.a = hm; r.b = 2.0 * hm; r.d = 6.0 * (ypn - sm); }
  } else {
    r.a = hm;
    r.c = h;
    r.b = 2.0 * (hm + h);
    r.d = 6.0 * (s - sm);
  }
  return r;
}

// Composition of affine maps t -> A + B t: (first then second).
__device__ __forceinline__ void compose(double A1, double B1, double A2, double B2, double &A, double &B) {
  A = fma(B2, A1, A2);
  B = B2 * B1;
}

// Inclusive block scan of the maps (A, B) in thread order (lower threads applied first); returns
// the composition of all maps of the threads below this one (exclusive), as (EA, EB).
__device__ void block_scan_up(double A, double B, double *wa, double *wb, double &EA, double &EB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const double A2 = __shfl_up_sync(0xffffffffu, A, off), B2 = __shfl_up_sync(0xffffffffu, B, off);
    if (lane >= off) compose(A2, B2, A, B, A, B);
  }
  if (lane == 31) {
    wa[warp] = A;
    wb[warp] = B;
  }
  __syncthreads();
  double PA = 0.0, PB = 1.0;  // maps of the warps below
  for (int w = 0; w < warp; ++w) compose(PA, PB, wa[w], wb[w], PA, PB);
  double XA = __shfl_up_sync(0xffffffffu, A, 1), XB = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) {
    XA = 0.0;
    XB = 1.0;
  }
  compose(PA, PB, XA, XB, EA, EB);
  __syncthreads();
}

// Inclusive block scan in reverse thread order (higher threads applied first); returns the
// composition of the maps of the threads above this one.
__device__ void block_scan_down(double A, double B, double *wa, double *wb, double &EA, double &EB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const double A2 = __shfl_down_sync(0xffffffffu, A, off), B2 = __shfl_down_sync(0xffffffffu, B, off);
    if (lane + off < 32) compose(A2, B2, A, B, A, B);
  }
  if (lane == 0) {
    wa[warp] = A;
    wb[warp] = B;
  }
  __syncthreads();
  double PA = 0.0, PB = 1.0;  // maps of the warps above
  for (int w = kWarpsSF - 1; w > warp; --w) compose(PA, PB, wa[w], wb[w], PA, PB);
  double XA = __shfl_down_sync(0xffffffffu, A, 1), XB = __shfl_down_sync(0xffffffffu, B, 1);
  if (lane == 31) {
    XA = 0.0;
    XB = 1.0;
  }
  compose(PA, PB, XA, XB, EA, EB);
  __syncthreads();
}

// Least k in [0, m] with x_k > v on the grid (binary64 estimate, checked on its two neighbours).
__device__ long long first_above_small(const Grid &G, double inv_step, double v) {
  const long long kv = dkey(v);
  if (G.m == 1) return dkey(G.x0) <= kv ? 1 : 0;
  const double e = (v - G.x0) * inv_step;
  long long k = (e >= 0.0) ? (long long)e : -1;
  k = max(min(k, G.m - 1), -1LL);
  while (k >= 0 && dkey(G.at(k)) > kv) --k;
  while (k + 1 < G.m && dkey(G.at(k + 1)) <= kv) ++k;
  return k + 1;
}

__global__ void __launch_bounds__(kThreadsSF, 1) small_f64_kernel(const Inst *__restrict__ insts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem &S = *reinterpret_cast<SmallSmem *>(smem_raw);
  const Inst I = insts[blockIdx.x];
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const int t = threadIdx.x;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  if (n > kMaxRowsSF) {  // never launched by the host: the shared memory would not hold it
    if (t == 0) atomicOr(I.status, kStBadTile);
    return;
  }
  const long long L = (n + kThreadsSF - 1) / kThreadsSF;
  const long long s0 = min((long long)t * L, n), e0 = min(s0 + L, n);
  const bool has = s0 < e0;
  unsigned bad = 0;

  // ---- forward: c' warm-up, then the piece's rows from the guess d'_{s0-1} = 0 ----
  // (the first piece starts at row 0, whose a = 0 makes its map of the guess a constant)
  double cp = 0.0, dp = 0.0, M = 1.0, hm = 0.0, sm = 0.0;
  if (has && s0 > 0) {
    const long long r0 = max(s0 - kWarmSF, 0LL);
    double xc = x[r0 + 1];
    double hp = xc - x[r0];  // h_{r0}
    if (r0 == 0) {
      cp = nat0 ? 0.0 : 0.5;  // c'_0 exactly
    } else {                  // row r0 from the guess c'_{r0-1} = 1/4
      const double hb = x[r0] - x[r0 - 1];
      cp = hp * rcp64(2.0 * (hb + hp) - 0.25 * hb);
    }
    for (long long j = r0 + 1; j < s0; ++j) {  // interior rows: c'_j = h_j / (2(h_{j-1} + h_j) - h_{j-1} c'_{j-1})
      const double xn = x[j + 1];
      const double h = xn - xc;
      cp = h * rcp64(2.0 * (hp + h) - hp * cp);
      hp = h;
      xc = xn;
    }
    hm = hp;  // h_{s0-1}
    sm = quot64(y[s0] - y[s0 - 1], hm, rcp64(hm));
  }
  for (long long j = s0; j < e0; ++j) {
    const double xj = x[j], yj = y[j];
    double h = 0.0, sl = 0.0;
    if (j <= n - 2) {
      const double xn = x[j + 1], yn = y[j + 1];
      bad |= row_check(xj, yj, true, xn);
      h = xn - xj;
      sl = quot64(yn - yj, h, rcp64(h));
    } else {
      bad |= row_check(xj, yj, false, 0.0);
    }
    const Row64 r = row64(j, n, nat0, nat1, I.yp1, I.ypn, hm, h, sm, sl);
    const double iden = rcp64(r.b - r.a * cp);
    cp = r.c * iden;
    dp = (r.d - r.a * dp) * iden;
    M *= -r.a * iden;
    S.cp[j] = cp;
    S.dp[j] = dp;
    S.mm[j] = M;
    hm = h;
    sm = sl;
  }
  // ---- the true d'_{s0-1} of every piece: block scan of the maps delta -> dp + M delta ----
  double EA, EB;
  block_scan_up(has ? dp : 0.0, has ? M : 1.0, S.wa, S.wb, EA, EB);
  const double delta = EA;  // the first piece's map is constant, so everything below composes to one
  for (long long j = s0; j < e0; ++j) S.dp[j] = fma(S.mm[j], delta, S.dp[j]);
  // ---- back substitution: each piece's map of the y'' above it, block scan from the top ----
  double P = 0.0, Q = 1.0;
  for (long long j = e0 - 1; j >= s0; --j) {
    const double c = S.cp[j], d = S.dp[j];
    P = fma(-c, P, d);
    Q *= -c;
  }
  double FA, FB;
  block_scan_down(has ? P : 0.0, has ? Q : 1.0, S.wa, S.wb, FA, FB);
  double Y = FA;  // y'' of row e0 (the last piece's map is constant: c'_{n-1} = 0)
  for (long long j = e0 - 1; j >= s0; --j) {
    Y = S.dp[j] - S.cp[j] * Y;
    S.dp[j] = Y;
    if (I.ypp) I.ypp[j] = Y;
  }
  if (bad) atomicOr(I.status, bad);
  if (m == 0) return;
  // ---- evaluation: the grid (once), each piece's first query, then its queries ----
  if (t == 0) {
    Grid G0 = make_grid(x, n, m);
    S.step = G0.step;
    S.inv_step = (m >= 2) ? rcp64(G0.step) : 0.0;
  }
  __syncthreads();
  Grid G;
  G.x0 = x[0];
  G.xl = x[n - 1];
  G.m = m;
  G.step = S.step;
  S.kfirst[t] = (!has || s0 == 0) ? 0 : (s0 > n - 2 ? m : first_above_small(G, S.inv_step, x[s0]));
  if (t == 0) S.kfirst[kThreadsSF] = m;
  __syncthreads();
  if (!has || s0 > n - 2) return;
  long long k = S.kfirst[t];
  const long long khi = (e0 <= n - 2) ? S.kfirst[t + 1] : m;  // the next piece's first query
  long long j = s0;
  const long long jmax = min(e0, n - 1) - 1;  // last interval of the piece
  double xj = x[j], xj1 = x[j + 1];
  long long kx1 = dkey(xj1);
  double ih = rcp64(xj1 - xj);
  for (; k < khi; ++k) {
    const double q = G.at(k);
    const long long kq = dkey(q);
    while (j < jmax && kx1 < kq) {
      ++j;
      xj = xj1;
      xj1 = x[j + 1];
      kx1 = dkey(xj1);
      ih = rcp64(xj1 - xj);
    }
    const double ba = xj1 - xj, xa = q - xj, bx = xj1 - q;
    const double ppj = S.dp[j], ppj1 = S.dp[j + 1];
    const double lower = xa * y[j + 1] + bx * y[j];
    const double C = (xa * xa - ba * ba) * xa * ppj1;
    const double D = (bx * bx - ba * ba) * bx * ppj;
    I.yq[k] = (lower + (1.0 / 6.0) * (C + D)) * ih;
    if (I.jq) I.jq[k] = (int32_t)j;
  }
}

namespace {
constexpr int kMaxDevSF = 64;
std::atomic<unsigned> g_small_ok[kMaxDevSF];
}  // namespace

int small_f64_max_rows() { return kMaxRowsSF; }

cudaError_t launch_small_f64(const Inst *d_insts, int ninst, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev >= 0 && dev < kMaxDevSF && g_small_ok[dev].load(std::memory_order_acquire))) {
    e = cudaFuncSetAttribute(small_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevSF) g_small_ok[dev].store(1u, std::memory_order_release);
  }
  small_f64_kernel<<<(unsigned)ninst, kThreadsSF, sizeof(SmallSmem), stream>>>(d_insts);
  return cudaGetLastError();
}

}  // namespace spl
