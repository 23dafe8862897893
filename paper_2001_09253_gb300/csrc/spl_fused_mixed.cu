// Mixed-precision fit + evaluation, one thread per tile of knots: the kernel of launches of many
// small instances and of the no-allocation entry point (long instances and the serving loop use
// the warp-cooperative tiles of spl_mixed_scan.cu).
//
// Same method and tiling as the plain FP64 kernel (tridiagonal system of eq. (init_val) with
// the end rows of "Start and End Derivatives", Thomas recurrences of "Implementation",
// evaluation by the form of "Fast Interpolation" on the grid of "Curve Interpolation"), but:
//   * the bulk arithmetic (Thomas recurrences, slopes, the cubic) runs in binary32;
//   * every difference of binary64 inputs that feeds it (knot widths h_j, value differences
//     y_{j+1}-y_j, query offsets x - x_j) is formed exactly on the integer pipe from the
//     encodings (spl_numeric.h) and rounded once to binary32, so large knots with tiny gaps
//     lose nothing before the binary32 arithmetic starts;
//   * the query positions x_k = x_0 + k*step stay binary64 (two FP64 instructions per query)
//     so that the bracket indices are bit-identical to the FP64 sweep;
//   * binary32 <-> binary64 conversions of values and outputs run on the integer pipe; the
//     rare operands the integer routes do not cover go through out-of-line FP64 helpers, so
//     the compiler cannot evaluate them speculatively on the slow FP64 pipe.
// The halos shrink with the binary32 target: the forward guess error falls below (2/3)^48
// (3.6e-9) and the backward one below 2^-24 (6e-8) of the solution's magnitude.
//
// Optional refinement (two launches): the first pass stores the binary32 y'' (Z) in scratch;
// the second forms the residual r = d - A Z of the system in double-float arithmetic from
// exact double-float widths and value differences, solves A delta = r with the same binary32
// tiling, outputs y'' = Z + delta and evaluates with it.
//
// Tiles are fetched dynamically, 32 at a time per warp, from a counter zeroed before the
// launch, so instances of very different sizes balance across SMs.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_mixed_math.cuh"
#include "spl_numeric.h"

namespace spl {

constexpr int kThreadsM = 512;            // one CTA per SM, four warps per sub-partition
constexpr int kSegM = 24;
constexpr int kHaloBM = 24;
constexpr int kRingM = kSegM + kHaloBM;
constexpr int kHaloFM = 48;
constexpr int kFieldsM = 2;               // c', d' (then y'')
constexpr int kPrefetchM = 32;            // rows between an L2 prefetch of x, y and their load
constexpr size_t kSmemM = (size_t)kRingM * kFieldsM * kThreadsM * sizeof(float);

struct RingM {
  float *base;
  int tid;
  __device__ __forceinline__ float &at(int row, int f) const { return base[(row * kFieldsM + f) * kThreadsM + tid]; }
};

// Queries of intervals [a, b) (local rows ta..tb of the tile), with y'' of the segment in
// ring field 1 and y''_b in Yb; returns the next query index.  Knots and values come from
// global memory (L2: the forward sweep touched them a segment earlier); the right end of the
// next interval is loaded one interval ahead.
__device__ __forceinline__ long long eval_segment(const Inst &I, const Grid &G, const RingM &ring, long long s0,
                                                  int ta, int tb, float Yb, long long k) {
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long a = s0 + ta, b = s0 + tb;
  if (m == 0 || a > n - 2) return k;
  const long long jmax = min(b, n - 1) - 1;
  const bool bounded = (b <= n - 2);
  const long long kb = bounded ? dkey(x[b]) : 0;
  long long j = a;
  int slot = ta % kRingM;
  double xj = x[j], xj1 = x[j + 1], yj = y[j], yj1 = y[j + 1];
  double xj2 = 0.0, yj2 = 0.0;  // x_{j+2}, y_{j+2}
  if (j + 2 < n) { xj2 = x[j + 2]; yj2 = y[j + 2]; }
  long long kxj1 = dkey(xj1);
  float ba = dif32_near(xj1, xj), iba = rcp32(ba);
  float fy0 = to_f32(yj), fy1 = to_f32(yj1);
  while (k < m) {
    const double q = G.at(k);
    const long long kq = dkey(q);
    if (bounded && kq > kb) break;
    if (j < jmax && kxj1 < kq) {
      const long long j_old = j;
      do {
        ++j;
        xj = xj1; yj = yj1;
        xj1 = xj2; yj1 = yj2;
        if (j + 2 < n) { xj2 = x[j + 2]; yj2 = y[j + 2]; }
        kxj1 = dkey(xj1);
      } while (j < jmax && kxj1 < kq);
      slot = (int)(j - s0) % kRingM;
      ba = dif32_near(xj1, xj);
      iba = rcp32(ba);
      fy0 = (j == j_old + 1) ? fy1 : to_f32(yj);
      fy1 = to_f32(yj1);
    }
    const int slot1 = (slot + 1 == kRingM) ? 0 : slot + 1;
    const float xa = dif32_near(q, xj);
    const float bx = ba - xa;
    const float ppj = ring.at(slot, 1);
    const float ppj1 = (j + 1 == b) ? Yb : ring.at(slot1, 1);
    I.yq[k] = to_f64(newint32(xa, bx, fy0, fy1, ppj, ppj1, ba, iba));
    if (I.jq) I.jq[k] = (int32_t)j;
    ++k;
  }
  return k;
}

// Forward state at row r: (c'_r, d'_r), h_r, s_r, the knot and value of row r+1 and the
// loads of rows r+2 and r+3 already in flight.
struct FwdM {
  double xn, yn;  // x_{r+1}, y_{r+1}
  double xa, ya;  // x_{r+2}, y_{r+2}
  double xb, yb;  // x_{r+3}, y_{r+3}
  float h, s, cp, dp;
};

// kFitOnly: first pass of the refined path; y'' (binary32) goes to the scratch I.z and no
// query is evaluated.
template <bool kFitOnly>
__device__ void tile_mixed(const Inst &I, long long tile, const RingM &ring) {
  const long long n = I.n;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = tile * (long long)I.tile_rows;
  const long long e0 = min(s0 + (long long)I.tile_rows, n);

  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  unsigned bad = 0;
  long long r = max(s0 - kHaloFM, 0LL);
  FwdM F;
  {
    const double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    F.xa = F.ya = F.xb = F.yb = 0.0;
    if (r + 2 < n) { F.xa = x[r + 2]; F.ya = y[r + 2]; }
    if (r + 3 < n) { F.xb = x[r + 3]; F.yb = y[r + 3]; }
    const float h = dif32_near(x1, x0), ih = rcp32(h), sl = quot32(dy32(y1, y0), h, ih);
    F.xn = x1; F.yn = y1; F.h = h; F.s = sl;
    if (r == 0 && !nat0) {
      F.cp = 0.5f;
      F.dp = 3.0f * (sl - to_f32(I.yp1)) * ih;
    } else {
      F.cp = 0.0f;
      F.dp = 0.0f;
    }
    if (r >= s0) {
      ring.at(0, 0) = F.cp; ring.at(0, 1) = F.dp;
      bad |= row_check(x0, y0, true, x1);
    }
  }
  int slot_r = (int)(r - s0);  // only meaningful once r >= s0
  auto forward_to = [&](long long target) {
    while (r < target) {
      const long long j = r + 1;
      float cpj, dpj;
      const bool owned = (j >= s0 && j < e0);
      if (j <= n - 2) {
        const double x2 = F.xa, y2 = F.ya;
        F.xa = F.xb; F.ya = F.yb;
        if (j + 3 < n) { F.xb = x[j + 3]; F.yb = y[j + 3]; }
        if (j + 3 + kPrefetchM < n) {
          if (first_in_block(x + j + 3 + kPrefetchM)) prefetch_l2m(x + j + 3 + kPrefetchM);
          if (first_in_block(y + j + 3 + kPrefetchM)) prefetch_l2m(y + j + 3 + kPrefetchM);
        }
        if (owned) bad |= row_check(F.xn, F.yn, true, x2);
        const float hj = dif32_near(x2, F.xn);
        const float ihj = rcp32(hj);
        const float sj = quot32(dy32(y2, F.yn), hj, ihj);
        const float den = 2.0f * (F.h + hj) - F.h * F.cp;
        const float iden = rcp32(den);
        cpj = hj * iden;
        dpj = (6.0f * (sj - F.s) - F.h * F.dp) * iden;
        F.xn = x2; F.yn = y2; F.h = hj; F.s = sj;
      } else {
        if (owned) bad |= row_check(F.xn, F.yn, false, 0.0);
        cpj = 0.0f;
        if (nat1) {
          dpj = 0.0f;
        } else {
          const float den = 2.0f * F.h - F.h * F.cp;
          dpj = (6.0f * (to_f32(I.ypn) - F.s) - F.h * F.dp) * rcp32(den);
        }
      }
      F.cp = cpj; F.dp = dpj;
      r = j;
      if (j >= s0) {
        slot_r = (j == s0) ? 0 : ((slot_r + 1 == kRingM) ? 0 : slot_r + 1);
        ring.at(slot_r, 0) = cpj; ring.at(slot_r, 1) = dpj;
      }
    }
  };
  if (s0 > 0) forward_to(s0);

  const Grid G = make_grid(x, n, I.m);
  long long k = kFitOnly ? 0 : first_query(G, x, s0);
  const int len = (int)(e0 - s0);
  for (int ta = 0; ta < len; ta += kSegM) {
    const int tb = min(ta + kSegM, len);
    const long long rlast = min(s0 + tb + kHaloBM, n) - 1;
    forward_to(rlast);
    const int tl = (int)(rlast - s0);
    int slot = tl % kRingM;
    float Y = ring.at(slot, 1);
    float Yb = Y;
    for (int t = tl - 1; t >= ta; --t) {
      slot = (slot == 0) ? kRingM - 1 : slot - 1;
      Y = ring.at(slot, 1) - ring.at(slot, 0) * Y;
      if (t == tb) Yb = Y;
      if (t < tb) ring.at(slot, 1) = Y;
    }
    if (kFitOnly) {
      for (int t = ta; t < tb; ++t) I.z[s0 + t] = ring.at(t % kRingM, 1);
      continue;
    }
    if (I.ypp) {
      for (int t = ta; t < tb; ++t) I.ypp[s0 + t] = to_f64(ring.at(t % kRingM, 1));
    }
    k = eval_segment(I, G, ring, s0, ta, tb, Yb, k);
  }
  if (bad) atomicOr(I.status, bad);
}

// ---- refinement pass ----
struct FwdR {
  double xn, yn;  // x_{r+1}, y_{r+1}
  double xa, ya;  // x_{r+2}, y_{r+2} (loaded one step early)
  F2 h, s;        // h_r, s_r
  float zr, zn;   // Z_r, Z_{r+1}
  float za;       // Z_{r+2}
  float cp, dp;   // Thomas state of the correction system at row r
};

__device__ void tile_refine(const Inst &I, long long tile, const RingM &ring) {
  const long long n = I.n;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const float *__restrict__ z = I.z;
  const long long s0 = tile * (long long)I.tile_rows;
  const long long e0 = min(s0 + (long long)I.tile_rows, n);
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  long long r = max(s0 - kHaloFM, 0LL);
  FwdR F;
  {
    const double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    const float z0 = z[r], z1 = z[r + 1];
    F.xa = F.ya = 0.0;
    F.za = 0.0f;
    if (r + 2 < n) { F.xa = x[r + 2]; F.ya = y[r + 2]; F.za = z[r + 2]; }
    const F2 h = dif2(x1, x0);
    const float ih = rcp32(h.hi);
    const F2 sl = df_div(dif2(y1, y0), h, ih);
    F.xn = x1; F.yn = y1; F.h = h; F.s = sl; F.zr = z0; F.zn = z1;
    if (r == 0 && !nat0) {
      // clamped first row: 6(s_0 - y'_0) - (2 h_0 Z_0 + h_0 Z_1), divided by b = 2 h_0
      const F2 d = df_mul_f(df_add(sl, df_neg(f2_of(I.yp1))), 6.0f);
      const F2 az = df_add(df_mul_f(h, 2.0f * z0), df_mul_f(h, z1));
      const F2 res = df_add(d, df_neg(az));
      F.cp = 0.5f;
      F.dp = (res.hi + res.lo) * 0.5f * ih;
    } else if (r == 0) {
      F.cp = 0.0f;
      F.dp = -z0;  // natural first row: y''_0 = 0
    } else {
      F.cp = 0.0f;
      F.dp = 0.0f;
    }
    if (r >= s0) { ring.at(0, 0) = F.cp; ring.at(0, 1) = F.dp; }
  }
  int slot_r = (int)(r - s0);
  auto forward_to = [&](long long target) {
    while (r < target) {
      const long long j = r + 1;
      float cpj, dpj;
      if (j <= n - 2) {
        const double x2 = F.xa, y2 = F.ya;
        const float z2 = F.za;
        if (j + 2 < n) { F.xa = x[j + 2]; F.ya = y[j + 2]; F.za = z[j + 2]; }
        if (j + 2 + kPrefetchM < n) {
          if (first_in_block(x + j + 2 + kPrefetchM)) prefetch_l2m(x + j + 2 + kPrefetchM);
          if (first_in_block(y + j + 2 + kPrefetchM)) prefetch_l2m(y + j + 2 + kPrefetchM);
          if (first_in_block(z + j + 2 + kPrefetchM)) prefetch_l2m(z + j + 2 + kPrefetchM);
        }
        const F2 hj = dif2(x2, F.xn);
        const float ihj = rcp32(hj.hi);
        const F2 sj = df_div(dif2(y2, F.yn), hj, ihj);
        const F2 d = df_mul_f(df_add(sj, df_neg(F.s)), 6.0f);
        const F2 az = df_add(df_add(df_mul_f(F.h, F.zr), df_mul_f(df_add(F.h, hj), 2.0f * F.zn)), df_mul_f(hj, z2));
        const F2 res = df_add(d, df_neg(az));
        const float rf = res.hi + res.lo;
        const float hf = F.h.hi;
        const float den = 2.0f * (hf + hj.hi) - hf * F.cp;
        const float iden = rcp32(den);
        cpj = hj.hi * iden;
        dpj = (rf - hf * F.dp) * iden;
        F.xn = x2; F.yn = y2; F.h = hj; F.s = sj; F.zr = F.zn; F.zn = z2;
      } else {  // last row
        cpj = 0.0f;
        if (nat1) {
          dpj = -F.zn;  // y''_{n-1} = 0
        } else {
          const F2 d = df_mul_f(df_add(f2_of(I.ypn), df_neg(F.s)), 6.0f);
          const F2 az = df_add(df_mul_f(F.h, F.zr), df_mul_f(F.h, 2.0f * F.zn));
          const F2 res = df_add(d, df_neg(az));
          const float hf = F.h.hi;
          const float den = 2.0f * hf - hf * F.cp;
          dpj = ((res.hi + res.lo) - hf * F.dp) * rcp32(den);
        }
      }
      F.cp = cpj; F.dp = dpj;
      r = j;
      if (j >= s0) {
        slot_r = (j == s0) ? 0 : ((slot_r + 1 == kRingM) ? 0 : slot_r + 1);
        ring.at(slot_r, 0) = cpj; ring.at(slot_r, 1) = dpj;
      }
    }
  };
  if (s0 > 0) forward_to(s0);

  const Grid G = make_grid(x, n, I.m);
  long long k = first_query(G, x, s0);
  const int len = (int)(e0 - s0);
  for (int ta = 0; ta < len; ta += kSegM) {
    const int tb = min(ta + kSegM, len);
    const long long rlast = min(s0 + tb + kHaloBM, n) - 1;
    forward_to(rlast);
    const int tl = (int)(rlast - s0);
    int slot = tl % kRingM;
    float D = ring.at(slot, 1);  // delta_{rlast} guess (exact at the last row)
    float Db = D;
    for (int t = tl - 1; t >= ta; --t) {
      slot = (slot == 0) ? kRingM - 1 : slot - 1;
      D = ring.at(slot, 1) - ring.at(slot, 0) * D;
      if (t == tb) Db = D;
      if (t < tb) ring.at(slot, 1) = D;
    }
    // y'' = Z + delta; field 1 then holds y'' for the evaluation
    const float Yb = (tb <= tl) ? z[s0 + tb] + Db : 0.0f;
    for (int t = ta; t < tb; ++t) {
      const int sl = t % kRingM;
      const float zj = z[s0 + t], dj = ring.at(sl, 1);
      if (I.ypp) I.ypp[s0 + t] = to_f64(zj) + to_f64(dj);
      ring.at(sl, 1) = zj + dj;
    }
    k = eval_segment(I, G, ring, s0, ta, tb, Yb, k);
  }
}

// ---- kernels: persistent CTAs, tiles fetched 32 at a time per warp ----
template <int kMode>  // 0: fit + eval, 1: fit only (refined path), 2: refine + eval
__global__ void __launch_bounds__(kThreadsM, 1) mixed_kernel(const Inst *__restrict__ insts, int ninst,
                                                             long long total_tiles,
                                                             unsigned long long *__restrict__ counter) {
  extern __shared__ float smem_ring_m[];
  RingM ring{smem_ring_m, (int)threadIdx.x};
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
      if (kMode == 0) tile_mixed<false>(I, t - I.tile_begin, ring);
      if (kMode == 1) tile_mixed<true>(I, t - I.tile_begin, ring);
      if (kMode == 2) tile_refine(I, t - I.tile_begin, ring);
    }
    __syncwarp();
  }
}

int mixed_threads_per_sm() { return kThreadsM; }

long long threads_mixed(int sm_count, long long total_tiles) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles, kThreadsM, &blocks, &bt);
  return (long long)blocks * bt;
}

// The ring is laid out for kThreadsM threads; a smaller CTA (few tiles spread over the SMs)
// uses the first blockDim.x columns of it.
template <int kMode>
static cudaError_t launch_mode(const Inst *d_insts, int ninst, long long total_tiles, int sm_count,
                               unsigned long long *counter, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(mixed_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemM);
  if (e != cudaSuccess) return e;
  int blocks, bt;
  spread_grid(sm_count, total_tiles, kThreadsM, &blocks, &bt);
  mixed_kernel<kMode><<<(unsigned)blocks, (unsigned)bt, kSmemM, stream>>>(d_insts, ninst, total_tiles, counter);
  return cudaGetLastError();
}

cudaError_t launch_fused_mixed(const Inst *d_insts, int ninst, long long total_tiles, int sm_count,
                               unsigned long long *counter, cudaStream_t stream, bool fit_only) {
  return fit_only ? launch_mode<1>(d_insts, ninst, total_tiles, sm_count, counter, stream)
                  : launch_mode<0>(d_insts, ninst, total_tiles, sm_count, counter, stream);
}

cudaError_t launch_refine_mixed(const Inst *d_insts, int ninst, long long total_tiles, int sm_count,
                                unsigned long long *counter, cudaStream_t stream) {
  return launch_mode<2>(d_insts, ninst, total_tiles, sm_count, counter, stream);
}

}  // namespace spl
