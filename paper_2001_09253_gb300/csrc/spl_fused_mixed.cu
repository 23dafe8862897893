// Mixed-precision fit + evaluation, fused, one thread per tile of knots.
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
//   * binary32 <-> binary64 conversions of values and outputs run on the integer pipe.
// The halos shrink with the binary32 target: the forward guess error falls below (2/3)^48
// (3.6e-9) and the backward one below 2^-24 (6e-8) of the solution's magnitude, i.e. to
// binary32 resolution.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_numeric.h"

namespace spl {

constexpr int kThreadsM = 256;            // one CTA per SM, two warps per sub-partition
constexpr int kSegM = 8;
constexpr int kHaloBM = 24;
constexpr int kRingM = kSegM + kHaloBM;   // a power of two
constexpr int kHaloFM = 48;
static_assert((kRingM & (kRingM - 1)) == 0, "ring size must be a power of two");
constexpr int kFieldsM = 4;               // c', d' (then y''), h, 1/h
constexpr size_t kSmemM = (size_t)kRingM * kFieldsM * kThreadsM * sizeof(float);

struct RingM {
  float *base;
  int tid;
  __device__ __forceinline__ float &at(int row, int f) const { return base[(row * kFieldsM + f) * kThreadsM + tid]; }
};

// b - a in binary32 from the integer route, or through FP64 when it does not apply
// (zero or subnormal operands, results outside binary32's normal range).
__device__ __forceinline__ float dif32(double b, double a) {
  float v;
  if (!diff_f32(b, a, &v)) v = (float)(b - a);
  return v;
}

__device__ __forceinline__ float quot32(float num, float den, float r) {
  float q = num * r;
  float rem = fmaf(-den, q, num);
  return fmaf(rem, r, q);
}

struct FwdM {
  double xn, yn;   // knot and value at r+1 (binary64)
  float h, s, cp, dp;
};

// "Fast Interpolation" in binary32, with xa = x - x_j and bx = x_{j+1} - x.
__device__ __forceinline__ float newint32(float xa, float bx, float yj, float yj1, float ppj, float ppj1,
                                          float ba, float inv_ba) {
  float ba2 = ba * ba;
  float lower = xa * yj1 + bx * yj;
  float C = (xa * xa - ba2) * xa * ppj1;
  float D = (bx * bx - ba2) * bx * ppj;
  return (lower + (1.0f / 6.0f) * (C + D)) * inv_ba;
}

__device__ __forceinline__ int slot_m(long long j, long long s0) { return (int)(j - s0) & (kRingM - 1); }

__device__ __forceinline__ void prefetch_l1m(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// kFitOnly: first pass of the refined path; y'' (binary32) goes to the scratch I.z and no
// query is evaluated.
template <bool kFitOnly>
__device__ void tile_mixed(const Inst &I, long long tile, const RingM &ring) {
  const long long n = I.n, m = I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = tile * (long long)I.tile_rows;
  const long long e0 = min(s0 + (long long)I.tile_rows, n);
  validate_rows(I, s0, e0);

  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  long long r = max(s0 - kHaloFM, 0LL);
  FwdM F;
  {
    double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    float h = dif32(x1, x0), ih = rcp32(h), sl = quot32(dif32(y1, y0), h, ih);
    F.xn = x1; F.yn = y1; F.h = h; F.s = sl;
    if (r == 0 && !nat0) {
      F.cp = 0.5f;
      F.dp = 3.0f * (sl - f64_to_f32(I.yp1)) * ih;
    } else {
      F.cp = 0.0f;
      F.dp = 0.0f;
    }
    if (r >= s0) {
      ring.at(0, 0) = F.cp; ring.at(0, 1) = F.dp; ring.at(0, 2) = h; ring.at(0, 3) = ih;
    }
  }
  auto forward_to = [&](long long target) {
    while (r < target) {
      const long long j = r + 1;
      float cpj, dpj, hj = 0.0f, ihj = 0.0f;
      if (j <= n - 2) {
        if (j + 17 < n) { prefetch_l1m(x + j + 17); prefetch_l1m(y + j + 17); }
        double x2 = x[j + 1], y2 = y[j + 1];
        hj = dif32(x2, F.xn);
        ihj = rcp32(hj);
        float sj = quot32(dif32(y2, F.yn), hj, ihj);
        float den = 2.0f * (F.h + hj) - F.h * F.cp;
        float iden = rcp32(den);
        cpj = hj * iden;
        dpj = (6.0f * (sj - F.s) - F.h * F.dp) * iden;
        F.xn = x2; F.yn = y2; F.h = hj; F.s = sj;
      } else {
        cpj = 0.0f;
        if (nat1) {
          dpj = 0.0f;
        } else {
          float den = 2.0f * F.h - F.h * F.cp;
          dpj = (6.0f * (f64_to_f32(I.ypn) - F.s) - F.h * F.dp) * rcp32(den);
        }
      }
      F.cp = cpj; F.dp = dpj;
      r = j;
      if (j >= s0) {
        const int slot = slot_m(j, s0);
        ring.at(slot, 0) = cpj; ring.at(slot, 1) = dpj; ring.at(slot, 2) = hj; ring.at(slot, 3) = ihj;
      }
    }
  };
  if (s0 > 0) forward_to(s0);

  const Grid G = make_grid(x, n, m);
  long long k = kFitOnly ? 0 : first_query(G, x, s0);
  for (long long a = s0; a < e0; a += kSegM) {
    const long long b = min(a + kSegM, e0);
    const long long rlast = min(b + kHaloBM, n) - 1;
    forward_to(rlast);
    float Y = ring.at(slot_m(rlast, s0), 1);
    float Yb = Y;
    for (long long j = rlast - 1; j >= a; --j) {
      const int slot = slot_m(j, s0);
      Y = ring.at(slot, 1) - ring.at(slot, 0) * Y;
      if (j == b) Yb = Y;
      if (j < b) ring.at(slot, 1) = Y;
    }
    if (kFitOnly) {
      for (long long j = a; j < b; ++j) I.z[j] = ring.at(slot_m(j, s0), 1);
      continue;
    }
    if (I.ypp) {
      for (long long j = a; j < b; ++j) I.ypp[j] = f32_to_f64(ring.at(slot_m(j, s0), 1));
    }
    if (m > 0 && a <= n - 2) {
      const long long jmax = min(b, n - 1) - 1;
      const bool bounded = (b <= n - 2);
      const long long kb = bounded ? dkey(x[b]) : 0;
      long long j = a;
      double xj = x[j], xj1 = x[j + 1];
      float yj = f64_to_f32(y[j]), yj1 = f64_to_f32(y[j + 1]);
      long long kxj1 = dkey(xj1);
      while (k < m) {
        const double q = G.at(k);
        const long long kq = dkey(q);
        if (bounded && kq > kb) break;
        if (j < jmax && kxj1 < kq) {
          do {
            ++j;
            xj = xj1;
            xj1 = x[j + 1];
            kxj1 = dkey(xj1);
          } while (j < jmax && kxj1 < kq);
          yj = f64_to_f32(y[j]);
          yj1 = f64_to_f32(y[j + 1]);
        }
        const int slot = slot_m(j, s0);
        const float ba = ring.at(slot, 2), iba = ring.at(slot, 3);
        const float xa = dif32(q, xj);
        const float bx = ba - xa;
        const float ppj = ring.at(slot, 1);
        const float ppj1 = (j + 1 == b) ? Yb : ring.at(slot_m(j + 1, s0), 1);
        I.yq[k] = f32_to_f64(newint32(xa, bx, yj, yj1, ppj, ppj1, ba, iba));
        if (I.jq) I.jq[k] = (int32_t)j;
        ++k;
      }
    }
  }
}

template <bool kFitOnly>
__global__ void __launch_bounds__(kThreadsM, 1) fused_mixed_kernel(const Inst *__restrict__ insts, int ninst,
                                                                   long long total_tiles) {
  extern __shared__ float smem_ring_m[];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  RingM ring{smem_ring_m, (int)threadIdx.x};
  for (long long t = tid; t < total_tiles; t += nthreads) {
    const int i = find_inst(insts, ninst, t);
    const Inst I = insts[i];
    tile_mixed<kFitOnly>(I, t - I.tile_begin, ring);
  }
}

// ---------------------------------------------------------------------------------------
// Second pass of the refined path: one step of iterative refinement of y'' followed by the
// evaluation.  With Z the binary32 solution of the first pass, the residual r = d - A Z of
// the system of eq. (init_val) (and of the end rows) is formed in double-float arithmetic
// from exact double-float knot widths and value differences, so it is accurate far below
// binary32 resolution; the correction A delta = r is solved with the same binary32 Thomas
// tiling, and y'' = Z + delta (accumulated in binary64 for the output) carries about twice
// the correct digits of Z.
constexpr int kFieldsR = 5;  // c', d' (then delta, then y''), h, 1/h, Z
constexpr size_t kSmemR = (size_t)kRingM * kFieldsR * kThreadsM * sizeof(float);

struct RingR {
  float *base;
  int tid;
  __device__ __forceinline__ float &at(int row, int f) const { return base[(row * kFieldsR + f) * kThreadsM + tid]; }
};

__device__ __forceinline__ F2 dif2(double b, double a) {
  F2 v;
  if (!diff_f2(b, a, &v)) {
    const double d = b - a;
    const float hi = (float)d;
    v = F2{hi, (float)(d - (double)hi)};
  }
  return v;
}

__device__ __forceinline__ F2 f2_of(double v) {
  const float hi = f64_to_f32(v);
  return F2{hi, (float)(v - (double)hi)};
}

struct FwdR {
  double xn, yn;  // x_{r+1}, y_{r+1}
  F2 h, s;        // h_r, s_r
  float zr, zn;   // Z_r, Z_{r+1}
  float cp, dp;   // Thomas state of the correction system at row r
};

__device__ void tile_refine(const Inst &I, long long tile, const RingR &ring) {
  const long long n = I.n, m = I.m;
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
    if (r >= s0) {
      ring.at(0, 0) = F.cp; ring.at(0, 1) = F.dp; ring.at(0, 2) = h.hi; ring.at(0, 3) = ih; ring.at(0, 4) = z0;
    }
  }
  auto forward_to = [&](long long target) {
    while (r < target) {
      const long long j = r + 1;
      float cpj, dpj, hst = 0.0f, ihst = 0.0f;
      const float zj = F.zn;
      if (j <= n - 2) {
        if (j + 17 < n) { prefetch_l1m(x + j + 17); prefetch_l1m(y + j + 17); prefetch_l1m(z + j + 33); }
        const double x2 = x[j + 1], y2 = y[j + 1];
        const float z2 = z[j + 1];
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
        hst = hj.hi;
        ihst = ihj;
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
        const int slot = slot_m(j, s0);
        ring.at(slot, 0) = cpj; ring.at(slot, 1) = dpj; ring.at(slot, 2) = hst; ring.at(slot, 3) = ihst;
        ring.at(slot, 4) = zj;
      }
    }
  };
  if (s0 > 0) forward_to(s0);

  const Grid G = make_grid(x, n, m);
  long long k = first_query(G, x, s0);
  for (long long a = s0; a < e0; a += kSegM) {
    const long long b = min(a + kSegM, e0);
    const long long rlast = min(b + kHaloBM, n) - 1;
    forward_to(rlast);
    float D = ring.at(slot_m(rlast, s0), 1);  // delta_{rlast} guess (exact at the last row)
    float Db = D;
    for (long long j = rlast - 1; j >= a; --j) {
      const int slot = slot_m(j, s0);
      D = ring.at(slot, 1) - ring.at(slot, 0) * D;
      if (j == b) Db = D;
      if (j < b) ring.at(slot, 1) = D;
    }
    for (long long j = a; j < b; ++j) {
      const int slot = slot_m(j, s0);
      const float zj = ring.at(slot, 4), dj = ring.at(slot, 1);
      if (I.ypp) I.ypp[j] = f32_to_f64(zj) + f32_to_f64(dj);
      ring.at(slot, 1) = zj + dj;
    }
    const float Yb = (b <= rlast) ? ring.at(slot_m(b, s0), 4) + Db : 0.0f;
    if (m > 0 && a <= n - 2) {
      const long long jmax = min(b, n - 1) - 1;
      const bool bounded = (b <= n - 2);
      const long long kb = bounded ? dkey(x[b]) : 0;
      long long j = a;
      double xj = x[j], xj1 = x[j + 1];
      float yj = f64_to_f32(y[j]), yj1 = f64_to_f32(y[j + 1]);
      long long kxj1 = dkey(xj1);
      while (k < m) {
        const double q = G.at(k);
        const long long kq = dkey(q);
        if (bounded && kq > kb) break;
        if (j < jmax && kxj1 < kq) {
          do {
            ++j;
            xj = xj1;
            xj1 = x[j + 1];
            kxj1 = dkey(xj1);
          } while (j < jmax && kxj1 < kq);
          yj = f64_to_f32(y[j]);
          yj1 = f64_to_f32(y[j + 1]);
        }
        const int slot = slot_m(j, s0);
        const float ba = ring.at(slot, 2), iba = ring.at(slot, 3);
        const float xa = dif32(q, xj);
        const float bx = ba - xa;
        const float ppj = ring.at(slot, 1);
        const float ppj1 = (j + 1 == b) ? Yb : ring.at(slot_m(j + 1, s0), 1);
        I.yq[k] = f32_to_f64(newint32(xa, bx, yj, yj1, ppj, ppj1, ba, iba));
        if (I.jq) I.jq[k] = (int32_t)j;
        ++k;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreadsM, 1) refine_mixed_kernel(const Inst *__restrict__ insts, int ninst,
                                                                    long long total_tiles) {
  extern __shared__ float smem_ring_r[];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  RingR ring{smem_ring_r, (int)threadIdx.x};
  for (long long t = tid; t < total_tiles; t += nthreads) {
    const int i = find_inst(insts, ninst, t);
    const Inst I = insts[i];
    tile_refine(I, t - I.tile_begin, ring);
  }
}

long long threads_mixed(int sm_count, long long total_tiles) {
  long long blocks = std::min<long long>((total_tiles + kThreadsM - 1) / kThreadsM, (long long)sm_count);
  return std::max<long long>(blocks, 1) * kThreadsM;
}

cudaError_t launch_fused_mixed(const Inst *d_insts, int ninst, long long total_tiles, long long threads,
                               cudaStream_t stream, bool fit_only) {
  const unsigned grid = (unsigned)(threads / kThreadsM);
  cudaError_t e;
  if (fit_only) {
    e = cudaFuncSetAttribute(fused_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemM);
    if (e != cudaSuccess) return e;
    fused_mixed_kernel<true><<<grid, kThreadsM, kSmemM, stream>>>(d_insts, ninst, total_tiles);
  } else {
    e = cudaFuncSetAttribute(fused_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemM);
    if (e != cudaSuccess) return e;
    fused_mixed_kernel<false><<<grid, kThreadsM, kSmemM, stream>>>(d_insts, ninst, total_tiles);
  }
  return cudaGetLastError();
}

cudaError_t launch_refine_mixed(const Inst *d_insts, int ninst, long long total_tiles, long long threads,
                                cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(refine_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemR);
  if (e != cudaSuccess) return e;
  refine_mixed_kernel<<<(unsigned)(threads / kThreadsM), kThreadsM, kSmemR, stream>>>(d_insts, ninst, total_tiles);
  return cudaGetLastError();
}

}  // namespace spl
