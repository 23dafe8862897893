// Evaluation of a fitted spline at a batch of queries, lane-parallel over queries: explicit query
// positions in any order (or the uniform grid of section "Curve Interpolation"), each
// bracketed by bisection (or by galloping from the interval of the lane's previous query when
// that lies below it), then one of the three forms of section "Fast Interpolation" that the
// paper benchmarks (section "Curve Interpolation": newint orig / noinv / vol).
//
// Bracketing is the definition the monotone sweep of section "Quality Checks" implements for
// sorted queries: the largest i in [0, n-2] with x_i < q, or 0 when there is none.  It runs on
// the order-preserving integer keys of the binary64 values, so the index is bit-identical to a
// binary64 comparison; a query equal to a knot takes the interval on its left.  Each probe is a
// dependent load: launches on the uniform grid (ascending queries) run eval_runs_kernel, whose
// lanes gallop a few knots from their previous query; launches with explicit positions run
// eval_bisect_kernel, one query per thread paying about log2(n) latencies, hidden by many
// threads per SM.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_numeric.h"

namespace spl {

constexpr int kThreadsE = 256;
// CTAs per SM: all resident at once within the register limit this imposes (51 per thread, no
// spills), so a launch is one wave (8 CTAs at the 48-56 registers the kernels take unbounded
// ran as a wave and a partial one: ~9 % slower on unsorted queries)
constexpr int kBlocksPerSmE = 5;

// count = the number of knots x_0..x_{n-2} whose key is below kq; the bracket is count - 1 (0 when
// count is 0).  With a coarse table T[i] = key(x_{16 i}) (built by coarse_keys_kernel for large
// instances) the first levels run on T, which stays in L2: the entries below kq number
// cc = ceil(count / 16), so count lies in [16 (cc - 1) + 1, min(16 cc, n - 1)], a window of one
// 128-byte run of knots that four probes of x finish.  The comparisons are the same key
// comparisons, so the bracket is the same as the plain bisection's.  (Every 4th, 8th, 16th or
// 32nd knot measured at 1e7 unsorted queries: 0.81, 0.72, 0.70, 0.73 ms.)
__device__ __forceinline__ long long bracket_bisect(const double *__restrict__ x, long long n, long long kq,
                                                    const long long *__restrict__ ktab) {
  long long lo = 0, hi = n - 1;  // knots x_0..x_{n-2} below q: a count in [lo, hi]
  if (ktab) {
    long long a = 0, b = coarse_key_entries(n);
    while (a < b) {
      const long long mid = a + ((b - a) >> 1);
      if (ktab[mid] < kq) a = mid + 1; else b = mid;
    }
    if (a == 0) return 0;
    lo = (long long)kCoarseKeys * (a - 1) + 1;
    hi = min((long long)kCoarseKeys * a, n - 1);
  }
  while (lo < hi) {
    const long long mid = lo + ((hi - lo) >> 1);
    if (dkey(x[mid]) < kq) lo = mid + 1; else hi = mid;
  }
  return lo > 0 ? lo - 1 : 0;
}

// The coarse key tables of the instances that have one (blockIdx.y strides the instances).
__global__ void coarse_keys_kernel(const Inst *__restrict__ insts, int ninst) {
  for (int i = blockIdx.y; i < ninst; i += gridDim.y) {
    const Inst &I = insts[i];
    if (!I.ktab) continue;
    long long *t = const_cast<long long *>(I.ktab);
    const long long nt = coarse_key_entries(I.n);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (long long)gridDim.x * blockDim.x)
      t[e] = dkey(I.x[e * kCoarseKeys]);
  }
}

// The one-division form, with ba = x_{j+1}-x_j, xa = x-x_j, bx = x_{j+1}-x:
//   y = (xa y_{j+1} + bx y_j + (1/6)((xa^2-ba^2) xa y''_{j+1} + (bx^2-ba^2) bx y''_j)) / ba.
// kVariant 0 (orig): inv_ba = 1/ba formed first, the sum multiplied by it.
// kVariant 1 (noinv): the sum divided by ba.
// kVariant 2 (vol): orig with inv_ba held in a volatile local, whose store and reload pin the
// division ahead of the cubic.
// kVariant 3 (noop): the paper's control loop of section "Curve Interpolation" (query generation
// and bracketing without the evaluation): the bracket's left knot x_j is written in place of the
// value, so the output traffic is the same and the bracket cannot be optimised away.
template <int kVariant>
__device__ __forceinline__ double newint_variant(double q, double xj, double xj1, double yj, double yj1, double ppj,
                                                 double ppj1) {
  if (kVariant == 3) return xj;
  const double ba = xj1 - xj;
  double inv_ba = 0.0;
  volatile double inv_pinned;
  if (kVariant == 0) inv_ba = 1.0 / ba;
  if (kVariant == 2) inv_pinned = 1.0 / ba;
  const double xa = q - xj;
  const double bx = xj1 - q;
  const double ba2 = ba * ba;
  const double lower = xa * yj1 + bx * yj;
  const double C = (xa * xa - ba2) * xa * ppj1;
  const double D = (bx * bx - ba2) * bx * ppj;
  const double sum = lower + (1.0 / 6.0) * (C + D);
  if (kVariant == 1) return sum / ba;
  if (kVariant == 2) return sum * inv_pinned;
  return sum * inv_ba;
}

// The binary32 form (mixed-precision plans): the differences of binary64 positions are formed
// exactly and rounded once (one FP64 subtraction for operands of one sign and exponent field,
// which is exact; a binary32 rounding of the FP64 difference otherwise), values and y'' are
// rounded to binary32, and the cubic runs in binary32 with the variant's division.
__device__ __forceinline__ float near_diff32(double b, double a) {
  const unsigned hb = (unsigned)(bits64(b) >> 32), ha = (unsigned)(bits64(a) >> 32);
  if (((hb ^ ha) >> 20) == 0u) return (float)(b - a);
  float v;
  if (diff_f32(b, a, &v)) return v;
  return (float)(b - a);
}

template <int kVariant>
__device__ __forceinline__ double newint_variant32(double q, double xj, double xj1, double yj, double yj1,
                                                   double ppj, double ppj1) {
  if (kVariant == 3) return xj;
  const float ba = near_diff32(xj1, xj);
  const float xa = near_diff32(q, xj);
  const float bx = ba - xa;
  float inv_ba = 0.0f;
  volatile float inv_pinned;
  if (kVariant == 0) inv_ba = 1.0f / ba;
  if (kVariant == 2) inv_pinned = 1.0f / ba;
  const float ba2 = ba * ba;
  const float lower = xa * (float)yj1 + bx * (float)yj;
  const float C = (xa * xa - ba2) * xa * (float)ppj1;
  const float D = (bx * bx - ba2) * bx * (float)ppj;
  const float sum = lower + (1.0f / 6.0f) * (C + D);
  if (kVariant == 1) return (double)(sum / ba);
  if (kVariant == 2) return (double)(sum * inv_pinned);
  return (double)(sum * inv_ba);
}

// Bracket of q given a knot x_{j0} < q (the previous query's interval): galloping steps of 1, 2,
// 4, ... knots from j0 (at most kGallopE of them; beyond, `far` is set and the rest of the
// instance is bisected), then bisection of the last step; the same index as bracket_bisect.
constexpr int kGallopE = 8;

__device__ __forceinline__ long long bracket_from(const double *__restrict__ x, long long n, long long j0,
                                                  long long kq, bool &far) {
  long long lo = j0, hi, step = 1;  // x_lo < q throughout
  far = false;
  for (int s = 0;; ++s) {
    hi = lo + step;
    if (hi > n - 2) {
      hi = n - 1;
      break;
    }
    if (dkey(x[hi]) >= kq) break;
    lo = hi;
    step <<= 1;
    if (s + 1 == kGallopE) {
      hi = n - 1;
      far = true;
      break;
    }
  }
  while (hi - lo > 1) {  // largest i in [lo, hi) with x_i < q
    const long long mid = lo + ((hi - lo) >> 1);
    if (dkey(x[mid]) < kq) lo = mid; else hi = mid;
  }
  return lo;
}

// Each warp takes runs of 32 kRunE consecutive queries, lane l the queries run + l + 32 i: every
// access of a step is contiguous across the warp, and a lane's successive queries lie 32 apart,
// so sorted queries find their interval by galloping from the previous one (~2 log2 32 probes
// near it instead of log2 n across the instance); a lane whose query lies below its previous one,
// or far above it, bisects for the rest of the run, so any order gives the same brackets.
constexpr int kRunE = 8;

template <int kVariant, bool kF32>
__global__ void __launch_bounds__(kThreadsE, kBlocksPerSmE)
    eval_runs_kernel(const Inst *__restrict__ insts, int ninst, long long total_q) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  constexpr long long kSpan = 32LL * kRunE;
  int cur = -1;  // instance of the previous query of this lane, whose grid is cached
  long long qb = 0, qe = 0;
  Grid G{};
  for (long long run = warp * kSpan; run < total_q; run += nwarps * kSpan) {
    long long jprev = -1;  // interval of the lane's previous query in this run
    bool gallop = true;    // the lane's queries have been ascending and close so far
#pragma unroll 1
    for (int i = 0; i < kRunE; ++i) {
      const long long g = run + lane + 32LL * i;
      if (g >= total_q) break;
      if (cur < 0 || g < qb || g >= qe) {  // the instance owning query g: last with q_begin <= g
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (insts[mid].q_begin <= g) lo = mid; else hi = mid - 1;
        }
        cur = lo;
        qb = insts[lo].q_begin;
        qe = qb + insts[lo].mq;
        G = insts[lo].xq ? Grid{} : make_grid(insts[lo].x, insts[lo].n, insts[lo].mq);
        jprev = -1;
      }
      const Inst &I = insts[cur];
      const long long n = I.n, k = g - qb;
      const double *__restrict__ x = I.x;
      double q;
      if (I.xq) {
        q = I.xq[k];
        if (!finite64(q)) {
          atomicOr(I.status, kStNonFinite);
          continue;
        }
      } else {
        q = G.at(k);
      }
      const long long kq = dkey(q);
      long long j;
      if (gallop && jprev >= 0 && dkey(x[jprev]) < kq) {
        bool far;
        j = bracket_from(x, n, jprev, kq, far);
        if (far) gallop = false;
      } else {
        if (jprev >= 0) gallop = false;
        j = bracket_bisect(x, n, kq, nullptr);
      }
      jprev = j;
      const double *__restrict__ y = I.y;
      const double *__restrict__ ypp = I.ypp;
      if (kVariant == 3)
        I.yq[k] = x[j];
      else
        I.yq[k] = kF32 ? newint_variant32<kVariant>(q, x[j], x[j + 1], y[j], y[j + 1], ypp[j], ypp[j + 1])
                       : newint_variant<kVariant>(q, x[j], x[j + 1], y[j], y[j + 1], ypp[j], ypp[j + 1]);
      if (I.jq) I.jq[k] = (int32_t)j;
    }
  }
}

// Queries in any order (explicit positions): one query per thread, grid-stride, bisection.
template <int kVariant, bool kF32>
__global__ void __launch_bounds__(kThreadsE, kBlocksPerSmE)
    eval_bisect_kernel(const Inst *__restrict__ insts, int ninst, long long total_q) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  int cur = -1;  // instance whose grid is cached
  Grid G{};
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total_q; g += stride) {
    int lo = 0, hi = ninst - 1;  // the instance owning query g: last with q_begin <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].q_begin <= g) lo = mid; else hi = mid - 1;
    }
    const Inst &I = insts[lo];
    const long long n = I.n, k = g - I.q_begin;
    const double *__restrict__ x = I.x;
    double q;
    if (I.xq) {
      q = I.xq[k];
      if (!finite64(q)) {
        atomicOr(I.status, kStNonFinite);
        continue;
      }
    } else {
      if (lo != cur) {
        G = make_grid(x, n, I.mq);
        cur = lo;
      }
      q = G.at(k);
    }
    const long long j = bracket_bisect(x, n, dkey(q), I.ktab);
    const double *__restrict__ y = I.y;
    const double *__restrict__ ypp = I.ypp;
    if (kVariant == 3)
      I.yq[k] = x[j];
    else
      I.yq[k] = kF32 ? newint_variant32<kVariant>(q, x[j], x[j + 1], y[j], y[j + 1], ypp[j], ypp[j + 1])
                     : newint_variant<kVariant>(q, x[j], x[j + 1], y[j], y[j + 1], ypp[j], ypp[j + 1]);
    if (I.jq) I.jq[k] = (int32_t)j;
  }
}

cudaError_t launch_eval(const Inst *d_insts, int ninst, long long total_q, int variant, bool f32, bool uniform,
                        long long max_coarse_entries, int sm_count, cudaStream_t stream) {
  if (total_q <= 0) return cudaSuccess;
  if (!uniform && max_coarse_entries > 0) {  // coarse key tables first (instances that have one)
    const long long bx = std::min<long long>((max_coarse_entries + kThreadsE - 1) / kThreadsE, 4LL * sm_count);
    const dim3 g((unsigned)std::max<long long>(bx, 1), (unsigned)std::min(ninst, 65535));
    coarse_keys_kernel<<<g, kThreadsE, 0, stream>>>(d_insts, ninst);
  }
  // uniform grids (ascending by construction): runs of queries per lane with galloping brackets;
  // explicit positions (any order): one query per thread with bisection
  const long long per_block = uniform ? (long long)kThreadsE * kRunE : (long long)kThreadsE;
  const long long blocks =
      std::min<long long>((total_q + per_block - 1) / per_block, (long long)sm_count * kBlocksPerSmE);
  const unsigned grid = (unsigned)std::max<long long>(blocks, 1);
#define SPL_EVAL_LAUNCH(V, F)                                                                         \
  (uniform ? (eval_runs_kernel<V, F><<<grid, kThreadsE, 0, stream>>>(d_insts, ninst, total_q), 0) \
           : (eval_bisect_kernel<V, F><<<grid, kThreadsE, 0, stream>>>(d_insts, ninst, total_q), 0))
  switch (variant * 2 + (f32 ? 1 : 0)) {
    case 2: SPL_EVAL_LAUNCH(1, false); break;
    case 3: SPL_EVAL_LAUNCH(1, true); break;
    case 4: SPL_EVAL_LAUNCH(2, false); break;
    case 5: SPL_EVAL_LAUNCH(2, true); break;
    case 6: SPL_EVAL_LAUNCH(3, false); break;
    case 7: SPL_EVAL_LAUNCH(3, true); break;
    case 1: SPL_EVAL_LAUNCH(0, true); break;
    default: SPL_EVAL_LAUNCH(0, false); break;
  }
#undef SPL_EVAL_LAUNCH
  return cudaGetLastError();
}

}  // namespace spl
