// Plain FP64 fit + evaluation, fused, one thread per tile of knots.
//
// The fit is the tridiagonal system of eq. (init_val) ("Generating Second Derivatives")
// with the end rows of "Start and End Derivatives", solved by the Thomas recurrences of
// "Implementation"; the evaluation is the one-division form of "Fast Interpolation" at
// the uniform grid of "Curve Interpolation".
//
// Parallel decomposition (GB300 design, not in the paper).  The serial Thomas sweep is cut
// into tiles of L knots.  Every tile is solved independently by one thread:
//   * the forward elimination starts kHaloF rows before the tile with the guess
//     c' = d' = 0.  With b = 2(a + c) the multiplier a/(b - a c') is below 2/3 (c' <= 1/2),
//     so the error of the guess shrinks by at least that factor per row: after 96 rows it
//     is below 1.2e-17 of max|d'|;
//   * the back substitution of a segment of kSeg rows starts kHaloB rows past it with the
//     guess y'' = d'; its error shrinks by c' < 1/2 per row (below 6e-20 after 64 rows).
// Forward results (c', d', 1/h) of the last kSeg + kHaloB rows live in a per-thread ring in
// shared memory (192 KB for the CTA's 128 threads; lane-interleaved, conflict-free).  After
// each segment's back substitution the thread writes its y'' and evaluates the queries whose
// interval lies in the segment, walking the uniform grid and the knots together (the
// monotone sweep of "Quality Checks").  1/h_j computed by the fit is reused by the
// evaluation, so each knot costs two reciprocals; h_j is recomputed exactly.
//
// GB300 notes: FP64 runs at ~1.7 lanes/clk/SM here (one warp per SM sub-partition fills
// it), so the kernel is FP64-pipe bound: one persistent CTA of four warps per SM, the ring
// in shared memory so that no dependent load waits on L2, comparisons on integer keys and
// divisions as a MUFU seed + 3 DFMAs.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"

namespace spl {

constexpr int kThreads = 128;           // one CTA per SM, one warp per sub-partition
constexpr int kSeg = 16;                // rows per back-substitution segment
constexpr int kHaloB = 48;              // back-substitution halo: error <= 2^-48 of max|y''|
constexpr int kRing = kSeg + kHaloB;    // ring rows per thread (a power of two)
static_assert((kRing & (kRing - 1)) == 0, "ring size must be a power of two");
constexpr int kHaloF = 96;              // forward-elimination halo: error <= (2/3)^96
constexpr int kFields = 3;              // c', d' (then y''), 1/h
constexpr size_t kSmemBytes = (size_t)kRing * kFields * kThreads * sizeof(double);

struct Ring64 {
  double *base;  // shared memory of the CTA
  int tid;
  __device__ __forceinline__ double &at(int row, int f) const {
    return base[(row * kFields + f) * kThreads + tid];
  }
};

// State of the forward sweep after row r: the knot and value at r+1, h_r, s_r, c'_r, d'_r.
struct Fwd64 {
  double xn, yn, h, s, cp, dp;
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

__device__ __forceinline__ int slot_of(long long j, long long s0) { return (int)(j - s0) & (kRing - 1); }

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

__device__ void tile_f64(const Inst &I, long long tile, const Ring64 &ring) {
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = tile * (long long)I.tile_rows;
  const long long e0 = min(s0 + (long long)I.tile_rows, n);
  validate_rows(I, s0, e0);

  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  // ---- forward elimination up to row s0 (halo rows are not stored) ----
  long long r = max(s0 - kHaloF, 0LL);  // row whose (c', d') the state holds
  Fwd64 F;
  {
    double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    double h = x1 - x0, ih = rcp64(h), sl = quot64(y1 - y0, h, ih);
    F.xn = x1; F.yn = y1; F.h = h; F.s = sl;
    if (r == 0 && !nat0) {            // clamped start: c'_0 = 1/2, d'_0 = 3(s_0 - y'_0)/h_0
      F.cp = 0.5;
      F.dp = 3.0 * (sl - I.yp1) * ih;
    } else {                          // natural start, or the halo guess
      F.cp = 0.0;
      F.dp = 0.0;
    }
    if (r >= s0) {                    // r == s0 == 0: row 0 is this tile's first row
      ring.at(0, 0) = F.cp; ring.at(0, 1) = F.dp; ring.at(0, 2) = ih;
    }
  }
  // advance the forward sweep so that the state holds row `target`, storing rows >= s0
  auto forward_to = [&](long long target) {
    while (r < target) {
      const long long j = r + 1;
      double cpj, dpj, ihj = 0.0;
      if (j <= n - 2) {
        if (j + 17 < n) { prefetch_l1(x + j + 17); prefetch_l1(y + j + 17); }
        double x2 = x[j + 1], y2 = y[j + 1];
        double hj = x2 - F.xn;
        ihj = rcp64(hj);
        double sj = quot64(y2 - F.yn, hj, ihj);
        double den = twice(F.h + hj) - F.h * F.cp;
        double iden = rcp64(den);
        cpj = hj * iden;
        dpj = (6.0 * (sj - F.s) - F.h * F.dp) * iden;
        F.xn = x2; F.yn = y2; F.h = hj; F.s = sj;
      } else {  // j == n-1: last row
        cpj = 0.0;
        if (nat1) {
          dpj = 0.0;
        } else {
          double den = 2.0 * F.h - F.h * F.cp;
          dpj = (6.0 * (I.ypn - F.s) - F.h * F.dp) * rcp64(den);
        }
      }
      F.cp = cpj; F.dp = dpj;
      r = j;
      if (j >= s0) {
        const int slot = slot_of(j, s0);
        ring.at(slot, 0) = cpj; ring.at(slot, 1) = dpj; ring.at(slot, 2) = ihj;
      }
    }
  };
  if (s0 > 0) forward_to(s0);

  const Grid G = make_grid(x, n, m);
  long long k = first_query(G, x, s0);
  // ---- segments ----
  for (long long a = s0; a < e0; a += kSeg) {
    const long long b = min(a + kSeg, e0);
    const long long rlast = min(b + kHaloB, n) - 1;
    forward_to(rlast);
    // back substitution from rlast down to a; rows [a, b) get y'' in field 1
    double Y = ring.at(slot_of(rlast, s0), 1);  // y''_{rlast} := d'_{rlast} (exact when rlast == n-1)
    double Yb = Y;                              // y''_b (if b <= rlast)
    for (long long j = rlast - 1; j >= a; --j) {
      const int slot = slot_of(j, s0);
      Y = ring.at(slot, 1) - ring.at(slot, 0) * Y;
      if (j == b) Yb = Y;
      if (j < b) ring.at(slot, 1) = Y;
    }
    if (I.ypp) {
      for (long long j = a; j < b; ++j) I.ypp[j] = ring.at(slot_of(j, s0), 1);
    }
    // queries whose interval j lies in [a, b): x_k > x_a (guaranteed by k's position)
    // and x_k <= x_b when b <= n-2
    if (m > 0 && a <= n - 2) {
      const long long jmax = min(b, n - 1) - 1;  // last interval of the segment
      const bool bounded = (b <= n - 2);
      const long long kb = bounded ? dkey(x[b]) : 0;
      long long j = a;
      double xj = x[j], xj1 = x[j + 1], yj = y[j], yj1 = y[j + 1];
      double hj = xj1 - xj;
      long long kxj1 = dkey(xj1);
      while (k < m) {
        const double q = G.at(k);
        const long long kq = dkey(q);
        if (bounded && kq > kb) break;
        if (j < jmax && kxj1 < kq) {
          do {
            ++j;
            if (j + 17 < n) { prefetch_l1(x + j + 17); prefetch_l1(y + j + 17); }
            xj = xj1; yj = yj1;
            xj1 = x[j + 1]; yj1 = y[j + 1];
            kxj1 = dkey(xj1);
          } while (j < jmax && kxj1 < kq);
          hj = xj1 - xj;
        }
        const int slot = slot_of(j, s0);
        const double ppj = ring.at(slot, 1);
        const double ppj1 = (j + 1 == b) ? Yb : ring.at(slot_of(j + 1, s0), 1);
        I.yq[k] = newint64(q, xj, xj1, yj, yj1, ppj, ppj1, hj, ring.at(slot, 2));
        if (I.jq) I.jq[k] = (int32_t)j;
        ++k;
      }
    }
  }
}

// Persistent CTAs; each warp fetches 32 tiles at a time from a counter zeroed before the
// launch, so tiles of uneven length (ragged tails, small instances) balance across SMs.
__global__ void __launch_bounds__(kThreads, 1) fused_f64_kernel(const Inst *__restrict__ insts, int ninst,
                                                                long long total_tiles,
                                                                unsigned long long *__restrict__ counter) {
  extern __shared__ double smem_ring[];
  Ring64 ring{smem_ring, (int)threadIdx.x};
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total_tiles) break;
    const long long t = (long long)base + lane;
    if (t < total_tiles) {
      const int i = find_inst(insts, ninst, t);
      const Inst I = insts[i];
      tile_f64(I, t - I.tile_begin, ring);
    }
    __syncwarp();
  }
}

size_t ring_bytes_f64(long long) { return 0; }  // the ring lives in shared memory

int halo_rows_f64() { return kHaloF + kHaloB; }

long long threads_f64(int sm_count, long long total_tiles) {
  long long blocks = std::min<long long>((total_tiles + kThreads - 1) / kThreads, (long long)sm_count);
  return std::max<long long>(blocks, 1) * kThreads;
}

cudaError_t launch_fused_f64(const Inst *d_insts, int ninst, long long total_tiles, double *,
                             long long threads, unsigned long long *counter, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(fused_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  const long long grid = threads / kThreads;
  fused_f64_kernel<<<(unsigned)grid, kThreads, kSmemBytes, stream>>>(d_insts, ninst, total_tiles, counter);
  return cudaGetLastError();
}

}  // namespace spl
