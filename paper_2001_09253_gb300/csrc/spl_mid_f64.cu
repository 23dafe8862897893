// Plain FP64 fit + evaluation of one mid-size instance by a grid of co-resident CTAs (latency path).
//
// Same system and arithmetic as the fused FP64 kernel (spl_fused_f64.cu): the tridiagonal system
// of eq. (init_val) with the end rows of "Start and End Derivatives", Thomas' recurrences of
// "Implementation", the one-division form of "Fast Interpolation" on the grid of "Curve
// Interpolation"; slopes as correctly rounded quotients, brackets on integer keys.
//
// The one-CTA kernel (spl_small_f64.cu) spread over G CTAs of kThreadsMF threads: CTA b owns the
// rows [b Lb, (b+1) Lb), its threads pieces of L = Lb / kThreadsMF rows, with L chosen so that
// G <= the SM count (a cooperative launch: every CTA is resident at once).  The CTA's c', d' and
// sensitivities live in shared memory, and up to 4,096 rows per CTA also its x and y; up to
// 9,600 rows the x and y are read from global memory instead.  On this part a warp's
// FP64 instruction holds its sub-partition's FP64 unit for ~64 cycles, so the time is the FP64
// chain of a piece; more CTAs give shorter pieces.  Every recurrence is split as in the one-CTA
// kernel, plus one exchange between CTAs per direction:
//   * c'_j: each thread runs the c' recurrence alone over the kWarmMF rows before its piece from a
//     guess (an error in c' shrinks 12-fold per row: 12^-16 < 2^-57), then over its own rows;
//   * d'_j is affine in d'_{s-1}: a block scan of the pieces' maps gives each thread its d'_{s-1}
//     as a map of the d' entering the CTA, and the CTA's own map (d' leaving it as a map of the d'
//     entering it) goes to global memory; warp 0 composes the maps of all CTAs below (a warp scan
//     over 32 CTAs at a time; CTA 0's map is a constant, row 0 having a = 0);
//   * y''_j = d'_j - c'_j y''_{j+1} likewise from the top: each CTA publishes the map of its first
//     row's y'' in terms of the y'' past its end, and composes the maps of all CTAs above (the last
//     one's is a constant, c'_{n-1} = 0);
//   * each thread then back-substitutes and evaluates the queries of its own intervals.
// The waits for other CTAs' maps are bounded (kWaitNsMF of GPU time); when one runs out the CTA
// records kStWaitTimeout and carries on, and the request completes with SPL_ERR_TIMEOUT.
#include <algorithm>
#include <atomic>

#include "spl_device.cuh"
#include "spl_internal.h"

namespace spl {

constexpr int kThreadsMF = 128;   // one warp per sub-partition
constexpr int kWarpsMF = kThreadsMF / 32;
constexpr int kMaxRowsMF = 4096;  // rows of one CTA with x and y staged in shared memory
constexpr int kMaxRowsBigMF = 9600;  // rows of one CTA without the staging (c', d', sensitivities only)
constexpr int kWarmMF = 16;       // c'-only rows before a piece
constexpr int kTargetRowsMF = 1;  // rows per thread while there are SMs to spare (1, 2, 4, 8, 16 measured: 1 best)
constexpr int kOneCtaMaxMF = 512; // up to this many rows one CTA (up to 4 rows per thread) beats the exchange
constexpr int kMaxCtasMF = 256;   // exchange slots
constexpr unsigned long long kWaitNsMF = 200000000ull;

// One CTA's maps in the exchange area.  A map is published when its flag holds the launch's tag:
// 1 in an area zeroed before the launch, else the launch's own number (an area that outlives
// launches then holds only older numbers, so it needs no clearing).
struct MidExchange {
  double fa, fb;     // d' at the CTA's last row = fa + fb * (d' at the row before its first)
  double ba, bb;     // y'' at the CTA's first row = ba + bb * (y'' at the row past its last)
  unsigned long long fflag, bflag;
};
static_assert(sizeof(MidExchange) == 48, "exchange slot layout");

// Shared memory: this head, then c', d' and the sensitivities of the CTA's Lb rows and, when the
// kernel stages them, x and y of rows [r_lo, r_hi) (warm-up rows, the CTA's, one past).
struct MidSmem {
  double wa[kWarpsMF], wb[kWarpsMF];   // per-warp totals of the block scans
  double ta, tb;                       // the CTA's total map of a block scan
  long long kfirst[kThreadsMF + 1];    // first query of each piece, and of the row past the CTA
  double step, inv_step;
  double din, yend;                    // d' entering the CTA, y'' past its last row
  unsigned fail;
};
constexpr size_t kHeadMF = (sizeof(MidSmem) + 15) / 16 * 16;
__host__ __device__ constexpr size_t mid_smem_bytes(long long Lb, bool stage) {
  return kHeadMF + 8 * (size_t)(3 * Lb + (stage ? 2 * (Lb + kWarmMF + 2) : 0));
}
static_assert(mid_smem_bytes(kMaxRowsMF, true) <= 232448 && mid_smem_bytes(kMaxRowsBigMF, false) <= 232448,
              "one CTA's shared memory");

struct RowMF {
  double a, b, c, d;
};
__device__ __forceinline__ RowMF row_mf(long long j, long long n, bool nat0, bool nat1, double yp1, double ypn,
                                        double hm, double h, double sm, double s) {
  RowMF r;
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

// Affine maps t -> A + B t; (A1, B1) applied first, then (A2, B2).
__device__ __forceinline__ void compose_mf(double A1, double B1, double A2, double B2, double &A, double &B) {
  A = fma(B2, A1, A2);
  B = B2 * B1;
}

// Block scan in thread order (lower threads applied first): (EA, EB) = the maps of the threads
// below this one; the CTA's total map to S.ta, S.tb.
__device__ void scan_up_mf(double A, double B, MidSmem &S, double &EA, double &EB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const double A2 = __shfl_up_sync(0xffffffffu, A, off), B2 = __shfl_up_sync(0xffffffffu, B, off);
    if (lane >= off) compose_mf(A2, B2, A, B, A, B);
  }
  if (lane == 31) {
    S.wa[warp] = A;
    S.wb[warp] = B;
  }
  __syncthreads();
  double PA = 0.0, PB = 1.0;
  for (int w = 0; w < warp; ++w) compose_mf(PA, PB, S.wa[w], S.wb[w], PA, PB);
  double XA = __shfl_up_sync(0xffffffffu, A, 1), XB = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) {
    XA = 0.0;
    XB = 1.0;
  }
  compose_mf(PA, PB, XA, XB, EA, EB);
  if (threadIdx.x == kThreadsMF - 1) compose_mf(PA, PB, A, B, S.ta, S.tb);
  __syncthreads();
}

// Block scan in reverse thread order (higher threads applied first): (EA, EB) = the maps of the
// threads above this one; the CTA's total map to S.ta, S.tb.
__device__ void scan_down_mf(double A, double B, MidSmem &S, double &EA, double &EB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const double A2 = __shfl_down_sync(0xffffffffu, A, off), B2 = __shfl_down_sync(0xffffffffu, B, off);
    if (lane + off < 32) compose_mf(A2, B2, A, B, A, B);
  }
  if (lane == 0) {
    S.wa[warp] = A;
    S.wb[warp] = B;
  }
  __syncthreads();
  double PA = 0.0, PB = 1.0;
  for (int w = kWarpsMF - 1; w > warp; --w) compose_mf(PA, PB, S.wa[w], S.wb[w], PA, PB);
  double XA = __shfl_down_sync(0xffffffffu, A, 1), XB = __shfl_down_sync(0xffffffffu, B, 1);
  if (lane == 31) {
    XA = 0.0;
    XB = 1.0;
  }
  compose_mf(PA, PB, XA, XB, EA, EB);
  if (threadIdx.x == 0) compose_mf(PA, PB, A, B, S.ta, S.tb);
  __syncthreads();
}

__device__ __forceinline__ unsigned long long gtimer_mf() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp 0: the composition of the published maps of the `count` CTAs k0, k0 + dir, ..., in that
// order (the first one is a constant map): returns its constant term.  Waits (bounded) for each
// map's flag to hold `tag`; *fail is set on every lane when any wait ran out.
__device__ double compose_published(const MidExchange *ex, int k0, int count, int dir, bool fwd,
                                    unsigned long long tag, unsigned *fail) {
  const int lane = threadIdx.x & 31;
  unsigned late = 0u;
  double PA = 0.0, PB = 1.0;
  for (int base = 0; base < count; base += 32) {
    const int i = base + lane;
    double A = 0.0, B = 1.0;
    if (i < count) {
      const MidExchange *e = ex + (k0 + dir * i);
      const volatile unsigned long long *flag = fwd ? &e->fflag : &e->bflag;
      const unsigned long long t0 = gtimer_mf();
      unsigned sleep_ns = 32;
      while (*flag != tag) {
        if (gtimer_mf() - t0 > kWaitNsMF) {
          late = 1u;
          break;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns <<= 1;
      }
      __threadfence();
      A = __ldcg(fwd ? &e->fa : &e->ba);
      B = __ldcg(fwd ? &e->fb : &e->bb);
    }
    for (int off = 1; off < 32; off <<= 1) {
      const double A2 = __shfl_up_sync(0xffffffffu, A, off), B2 = __shfl_up_sync(0xffffffffu, B, off);
      if (lane >= off) compose_mf(A2, B2, A, B, A, B);
    }
    const int last = min(31, count - 1 - base);
    const double CA = __shfl_sync(0xffffffffu, A, last), CB = __shfl_sync(0xffffffffu, B, last);
    compose_mf(PA, PB, CA, CB, PA, PB);
  }
  if (__any_sync(0xffffffffu, late != 0u)) *fail = 1u;
  return PA;
}

__device__ void publish_mf(MidExchange *e, double A, double B, bool fwd, unsigned long long tag) {
  if (fwd) {
    e->fa = A;
    e->fb = B;
  } else {
    e->ba = A;
    e->bb = B;
  }
  __threadfence();
  atomicExch(fwd ? &e->fflag : &e->bflag, tag);
}

// Least k in [0, m] with x_k > v on the grid (binary64 estimate, checked on its two neighbours).
__device__ long long first_above_mf(const Grid &G, double inv_step, double v) {
  const long long kv = dkey(v);
  if (G.m == 1) return dkey(G.x0) <= kv ? 1 : 0;
  const double e = (v - G.x0) * inv_step;
  long long k = (e >= 0.0) ? (long long)e : -1;
  k = max(min(k, G.m - 1), -1LL);
  while (k >= 0 && dkey(G.at(k)) > kv) --k;
  while (k + 1 < G.m && dkey(G.at(k + 1)) <= kv) ++k;
  return k + 1;
}

// kStage: x and y of the CTA's rows staged in shared memory (Lb <= kMaxRowsMF); otherwise read from
// global memory (Lb <= kMaxRowsBigMF: larger instances, whose rows no longer fit beside them).
// The descriptor is *inst, or `one` (a kernel parameter) when inst is null; `launch` is the
// launch's number for an exchange area that is not cleared before it, 0 for a zeroed one.
template <bool kStage>
__global__ void __launch_bounds__(kThreadsMF, 1)
    mid_f64_kernel(const Inst *__restrict__ inst, const Inst one, MidExchange *__restrict__ ex,
                   long long Lb, unsigned fault, unsigned long long launch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MidSmem &S = *reinterpret_cast<MidSmem *>(smem_raw);
  double *const cpS = reinterpret_cast<double *>(smem_raw + kHeadMF);
  double *const dpS = cpS + Lb;
  double *const mmS = dpS + Lb;
  const Inst I = inst ? *inst : one;
  const unsigned long long tag = launch ? launch : 1ull;
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const int t = threadIdx.x, b = blockIdx.x, G = gridDim.x;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  if (Lb > (kStage ? kMaxRowsMF : kMaxRowsBigMF) || Lb % kThreadsMF != 0 || G > kMaxCtasMF) {  // never launched by the host
    if (t == 0) atomicOr(I.status, kStBadTile);
    return;
  }
  const long long L = Lb / kThreadsMF;
  const long long c0 = min((long long)b * Lb, n), c1 = min(c0 + Lb, n);
  const long long s0 = min(c0 + (long long)t * L, c1), e0 = min(s0 + L, c1);
  const bool has = s0 < e0;
  const bool withhold = (fault & 1u) && b == G - 1;  // failure-detection tests: the others time out
  if (t == 0) S.fail = 0u;
  unsigned bad = 0;
  // kStage: every x and y the CTA reads (the warm-up rows before it, its rows, one past) into
  // shared memory in one coalesced pass, so the row loops below wait on no global load
  const double *__restrict__ XS = x;  // XS[j] = x_j (from shared memory for j in [r_lo, r_hi))
  const double *__restrict__ YS = y;
  if (kStage) {
    double *const sx = mmS + Lb;
    double *const sy = sx + (Lb + kWarmMF + 2);
    const long long r_lo = max(c0 - kWarmMF - 1, 0LL), r_hi = min(c1 + 1, n);
    for (long long r = r_lo + t; r < r_hi; r += kThreadsMF) {
      sx[r - r_lo] = x[r];
      sy[r - r_lo] = y[r];
    }
    __syncthreads();
    XS = sx - r_lo;
    YS = sy - r_lo;
  }

  // ---- forward: c' warm-up, then the piece's rows from the guess d'_{s0-1} = 0 ----
  double cp = 0.0, dp = 0.0, M = 1.0, hm = 0.0, sm = 0.0;
  if (has && s0 > 0) {
    const long long r0 = max(s0 - kWarmMF, 0LL);
    double xc = XS[r0 + 1];
    double hp = xc - XS[r0];  // h_{r0}
    if (r0 == 0) {
      cp = nat0 ? 0.0 : 0.5;  // c'_0 exactly
    } else {                  // row r0 from the guess c'_{r0-1} = 1/4
      const double hb = XS[r0] - XS[r0 - 1];
      cp = hp * rcp64(2.0 * (hb + hp) - 0.25 * hb);
    }
    for (long long j = r0 + 1; j < s0; ++j) {  // interior rows: c'_j = h_j / (2(h_{j-1} + h_j) - h_{j-1} c'_{j-1})
      const double xn = XS[j + 1];
      const double h = xn - xc;
      cp = h * rcp64(2.0 * (hp + h) - hp * cp);
      hp = h;
      xc = xn;
    }
    hm = hp;  // h_{s0-1}
    sm = quot64(YS[s0] - YS[s0 - 1], hm, rcp64(hm));
  }
  for (long long j = s0; j < e0; ++j) {
    const double xj = XS[j], yj = YS[j];
    double h = 0.0, sl = 0.0;
    if (j <= n - 2) {
      const double xn = XS[j + 1], yn = YS[j + 1];
      bad |= row_check(xj, yj, true, xn);
      h = xn - xj;
      sl = quot64(yn - yj, h, rcp64(h));
    } else {
      bad |= row_check(xj, yj, false, 0.0);
    }
    const RowMF r = row_mf(j, n, nat0, nat1, I.yp1, I.ypn, hm, h, sm, sl);
    const double iden = rcp64(r.b - r.a * cp);
    cp = r.c * iden;
    dp = (r.d - r.a * dp) * iden;
    M *= -r.a * iden;
    cpS[j - c0] = cp;
    dpS[j - c0] = dp;
    mmS[j - c0] = M;
    hm = h;
    sm = sl;
  }
  // ---- d' entering each piece: block scan, then the maps of the CTAs below (warp 0), while
  // warp 1 forms the query grid's step (off the critical path: the other warps wait anyway) ----
  double EA, EB;
  scan_up_mf(has ? dp : 0.0, has ? M : 1.0, S, EA, EB);
  if (t == 0 && !withhold) publish_mf(ex + b, S.ta, S.tb, true, tag);
  if (t < 32) {
    unsigned fail = 0u;
    const double din = (b > 0) ? compose_published(ex, 0, b, 1, true, tag, &fail) : 0.0;
    if (t == 0) {
      S.din = din;
      if (fail) S.fail = 1u;
    }
  } else if (t == 32 && m > 0) {
    const Grid G0 = make_grid(x, n, m);
    S.step = G0.step;
    S.inv_step = (m >= 2) ? rcp64(G0.step) : 0.0;
  }
  __syncthreads();
  Grid Gd;
  Gd.x0 = x[0];
  Gd.xl = x[n - 1];
  Gd.m = m;
  Gd.step = S.step;
  const double delta = fma(EB, S.din, EA);
  for (long long j = s0; j < e0; ++j) dpS[j - c0] = fma(mmS[j - c0], delta, dpS[j - c0]);
  // ---- back substitution: each piece's map of the y'' above it, block scan, the CTAs above ----
  double P = 0.0, Q = 1.0;
  for (long long j = e0 - 1; j >= s0; --j) {
    const double c = cpS[j - c0], d = dpS[j - c0];
    P = fma(-c, P, d);
    Q *= -c;
  }
  double FA, FB;
  scan_down_mf(has ? P : 0.0, has ? Q : 1.0, S, FA, FB);
  if (t == 0 && !withhold) publish_mf(ex + b, S.ta, S.tb, false, tag);
  if (t < 32) {
    unsigned fail = 0u;
    const double yend = (b < G - 1) ? compose_published(ex, G - 1, G - 1 - b, -1, false, tag, &fail) : 0.0;
    if (t == 0) {
      S.yend = yend;
      if (fail) S.fail = 1u;
    }
  } else if (m > 0) {
    // meanwhile warps 1..3: the first query of every piece (threads without rows: s0 = c1, the
    // row past the CTA) and of the row past the CTA
    for (int i = t - 32; i <= kThreadsMF; i += kThreadsMF - 32) {
      const long long si = min(c0 + (long long)i * L, c1);
      S.kfirst[i] = (si == 0) ? 0 : (si > n - 2 ? m : first_above_mf(Gd, S.inv_step, XS[si]));
    }
  }
  __syncthreads();
  double Y = fma(FB, S.yend, FA);  // y'' of row e0
  for (long long j = e0 - 1; j >= s0; --j) {
    Y = dpS[j - c0] - cpS[j - c0] * Y;
    dpS[j - c0] = Y;
    if (I.ypp) I.ypp[j] = Y;
  }
  if (t == 0 && S.fail) bad |= kStWaitTimeout;
  if (bad) atomicOr(I.status, bad);
  if (m == 0) return;
  // ---- evaluation of the piece's queries (the grid step and the first queries from above) ----
  if (!has || s0 > n - 2) return;
  long long k = S.kfirst[t];
  const long long khi = (e0 <= n - 2) ? S.kfirst[t + 1] : m;  // the next piece's first query
  long long j = s0;
  const long long jmax = min(e0, n - 1) - 1;  // last interval of the piece
  double xj = XS[j], xj1 = XS[j + 1];
  long long kx1 = dkey(xj1);
  double ih = rcp64(xj1 - xj);
  for (; k < khi; ++k) {
    const double q = Gd.at(k);
    const long long kq = dkey(q);
    while (j < jmax && kx1 < kq) {
      ++j;
      xj = xj1;
      xj1 = XS[j + 1];
      kx1 = dkey(xj1);
      ih = rcp64(xj1 - xj);
    }
    const double ba = xj1 - xj, xa = q - xj, bx = xj1 - q;
    const double ppj = dpS[j - c0];
    const double ppj1 = (j + 1 < c1) ? dpS[j + 1 - c0] : S.yend;  // past the CTA: the next CTA's first row
    const double lower = xa * YS[j + 1] + bx * YS[j];
    const double C = (xa * xa - ba * ba) * xa * ppj1;
    const double D = (bx * bx - ba * ba) * bx * ppj;
    I.yq[k] = (lower + (1.0 / 6.0) * (C + D)) * ih;
    if (I.jq) I.jq[k] = (int32_t)j;
  }
}

namespace {
constexpr int kMaxDevMF = 64;
std::atomic<unsigned> g_mid_ok[kMaxDevMF];
}  // namespace

uint64_t mid_f64_exchange_bytes() { return (uint64_t)kMaxCtasMF * sizeof(MidExchange); }

// Rows per CTA for n points on sm_count SMs: one CTA up to kOneCtaMaxMF rows; beyond, kTargetRowsMF
// rows per thread while that needs no more CTAs than SMs, else as few more as fit one CTA per SM;
// 0 when n is beyond the path (SMs x kMaxRowsBigMF knots).  Measured on GB300 (one request, device
// time): n = 1,000 in 0.028 ms with 1-row pieces on 8 CTAs against 0.037 ms with 4-row pieces on 2;
// n = 300 in 0.025 ms on one CTA against 0.028 ms on 3.
long long mid_f64_cta_rows(long long n, int sm_count) {
  const int ctas = std::min(sm_count, kMaxCtasMF);
  long long L = std::max<long long>(kTargetRowsMF, (n + (long long)ctas * kThreadsMF - 1) / ((long long)ctas * kThreadsMF));
  if (n <= kOneCtaMaxMF) L = (n + kThreadsMF - 1) / kThreadsMF;  // one CTA: the shortest pieces
  if (L * kThreadsMF > kMaxRowsBigMF) return 0;
  return L * kThreadsMF;
}

cudaError_t launch_mid_f64(const Inst *d_inst, const Inst *h_inst, long long n, void *exchange,
                           unsigned long long launch, int sm_count, unsigned fault, cudaStream_t stream) {
  if (!d_inst && !h_inst) return cudaErrorInvalidValue;
  const long long Lb = mid_f64_cta_rows(n, sm_count);
  if (Lb <= 0) return cudaErrorInvalidValue;
  const unsigned G = (unsigned)((n + Lb - 1) / Lb);
  const bool stage = Lb <= kMaxRowsMF;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev >= 0 && dev < kMaxDevMF && g_mid_ok[dev].load(std::memory_order_acquire))) {
    e = cudaFuncSetAttribute(mid_f64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mid_smem_bytes(kMaxRowsMF, true));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mid_f64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)mid_smem_bytes(kMaxRowsBigMF, false));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevMF) g_mid_ok[dev].store(1u, std::memory_order_release);
  }
  // cooperative: the CTAs wait for each other's maps, so all of them must be resident together
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kThreadsMF);
  cfg.dynamicSmemBytes = mid_smem_bytes(Lb, stage);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MidExchange *ex = reinterpret_cast<MidExchange *>(exchange);
  Inst one{};
  if (!d_inst) one = *h_inst;
  return stage ? cudaLaunchKernelEx(&cfg, mid_f64_kernel<true>, d_inst, one, ex, Lb, fault, launch)
               : cudaLaunchKernelEx(&cfg, mid_f64_kernel<false>, d_inst, one, ex, Lb, fault, launch);
}

}  // namespace spl
