// Mixed-precision fit + evaluation, one thread per tile of knots.
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

// ---------------------------------------------------------------------------------------
// Persistent serving loop (continuous batching).  Warp 0 of CTA 0 is the scheduler: it reads
// request entries that the host appends to a ring in mapped host memory, installs each in its
// device slot, maps the request's tiles into the device tile map and publishes them by
// advancing `published`.  Every other warp is a worker: it claims 32 consecutive tile tickets
// at a time and, once a ticket is published, solves that tile of that request with the same
// binary32 fit + evaluation as mixed_kernel<0>.  The lane finishing a request's last tile
// writes the request's status and sequence number to mapped host memory.  All waits are
// bounded: the scheduler leaves after `idle_ns` without work or at `deadline_ns`, and sets
// `stop`; workers leave once stop is set and every published tile is claimed.  The host
// relaunches the loop when new work arrives.  Launched cooperatively (one CTA per SM), so the
// scheduler and the workers are co-resident.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreadsM, 1) serve_kernel(ServeArgs a) {
  extern __shared__ float smem_ring_s[];
  RingM ring{smem_ring_s, (int)threadIdx.x};
  const int lane = threadIdx.x & 31;
  const bool scheduler = (blockIdx.x == 0 && threadIdx.x < 32);
  const unsigned long long t_start = globaltimer_ns();
  volatile unsigned long long *published = a.published;
  volatile unsigned *stop = a.stop;

  if (scheduler && (a.fault_flags & 1u)) return;  // failure-detection tests: no work is published
  if (scheduler) {
    unsigned long long consumed = *a.consumed;
    unsigned long long last_work = t_start;
    unsigned sleep_ns = 64;
    if (lane == 0) *a.h_alive = 1u;
    for (;;) {
      const unsigned long long tail = *a.h_tail;
      if (consumed < tail) {
        __threadfence_system();  // the entry was written before the tail: read it after
        const ServeEntry *e = a.h_ring + (consumed % a.rcap);
        // one 8-byte word of the entry per lane from mapped host memory, shared by shuffles
        constexpr int kWords = (int)(sizeof(ServeEntry) / 8);
        static_assert(kWords <= 32, "a serving entry must fit in one warp's loads");
        const volatile unsigned long long *src = reinterpret_cast<const volatile unsigned long long *>(e);
        const unsigned long long word = (lane < kWords) ? src[lane] : 0ull;
        ServeEntry ent;
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&ent);
        for (int w = 0; w < kWords; ++w) dst[w] = __shfl_sync(0xffffffffu, word, w);
        const unsigned slot = ent.slot;
        if (lane == 0) {
          ent.inst.status = a.slot_status + slot;
          ent.inst.z = nullptr;
          a.slot_inst[slot] = ent.inst;
          a.slot_first[slot] = ent.first_tile;
          a.slot_done[slot] = 0u;
          a.slot_status[slot] = 0u;
          a.slot_seq[slot] = ent.seq;
        }
        const unsigned long long nt = (unsigned long long)ent.inst.ntiles;
        for (unsigned long long i = lane; i < nt; i += 32) a.tile_slot[(ent.first_tile + i) % a.tile_cap] = slot;
        __threadfence();
        __syncwarp();
        if (lane == 0) *published = ent.first_tile + nt;
        ++consumed;
        if (lane == 0) {
          *a.consumed = consumed;
          *a.h_consumed = consumed;
          __threadfence_system();
        }
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

  // workers
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.claimed, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    const unsigned long long t = base + lane;
    bool have = false;
    unsigned sleep_ns = 64;
    for (;;) {
      if (*published > t) {
        have = true;
        break;
      }
      if (*stop) {
        __threadfence();
        have = *published > t;
        break;
      }
      if (globaltimer_ns() - t_start > a.deadline_ns + 1000000000ull) {  // the scheduler stops first
        atomicOr(a.err, 1u);
        break;
      }
      __nanosleep(sleep_ns);
      if (sleep_ns < 4096) sleep_ns <<= 1;
    }
    if (have) {
      __threadfence();
      const unsigned slot = a.tile_slot[t % a.tile_cap];
      const Inst I = a.slot_inst[slot];
      tile_mixed<false>(I, (long long)(t - a.slot_first[slot]), ring);
      __threadfence();
      const unsigned done = atomicAdd(a.slot_done + slot, 1u) + 1u;
      if (done == (unsigned)I.ntiles) {
        __threadfence();
        const unsigned st = *(volatile unsigned *)(a.slot_status + slot);
        a.h_done[2 * slot] = st;
        __threadfence_system();
        a.h_done[2 * slot + 1] = a.slot_seq[slot];
        __threadfence_system();
      }
    }
    if (__all_sync(0xffffffffu, !have)) break;
  }
}

cudaError_t launch_serve(const ServeArgs &args, int sm_count, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemM);
  if (e != cudaSuccess) return e;
  ServeArgs copy = args;
  void *params[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)serve_kernel, dim3((unsigned)sm_count), dim3(kThreadsM), params,
                                     kSmemM, stream);
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

// ---------------------------------------------------------------------------------------
// Tiled binary32 fit + evaluation (no refinement): the decomposition of the plain FP64 kernel
// (spl_fused_f64.cu) with the binary32 arithmetic above.  One thread per tile, a warp's 32
// tiles grouped (instances of >= 32 tiles):
//   * only the first lane of a group runs a forward halo (48 rows, (2/3)^48 < 2^-28); its tile
//     is kLane0ShortT rows shorter;
//   * the other lanes are chained: the exact c'_{s0-1} from 8 rows of the c' recurrence alone
//     (error factor <= 1/12 per row), the guess d'_{s0-1} = 0, and the sensitivity M_i of
//     their d'_i to the true d'_{s0-1}, kept while |M_i| >= 2^-100; a warp scan over the lanes'
//     affine maps then gives every lane its d'_{s0-1} and the kept rows are corrected;
//   * the back substitution starts 24 rows past a tile (error x c' < 1/2 per row: 2^-24),
//     taken from the next lane's forward sweep (the last lane's tile is 24 rows shorter);
//   * the back substitution is fused with the evaluation, one query per iteration, the rows
//     walked down as far as the query needs.
// (c', d') live in per-warp scratch in global memory (binary32, lane-interleaved).
constexpr int kThreadsT = 512;          // one CTA per SM, four warps per sub-partition
constexpr int kOvT = 24;                // back-substitution start past a tile
constexpr int kLane0ShortT = 48;        // the first lane's forward halo
constexpr int kHaloCT = 8;              // c'-only rows before a chained tile
constexpr int kMRowsT = 192;            // sensitivities kept per lane: (2/3)^192 < 2^-112
constexpr float kMStopT = 0x1p-100f;    // far below binary32 resolution: d'_{s0-1} may exceed the
                                        // tile's values by many orders of magnitude (tiny gaps)

struct ScrT {
  float *base;  // rows x {c', d'} x 32 lanes
  float *mb;    // kMRowsT x 32 lanes
  int lane;
  __device__ __forceinline__ float &at(long long row, int f) const { return base[(((size_t)row * 2 + f) << 5) + lane]; }
  __device__ __forceinline__ float &m(int row) const { return mb[(row << 5) + lane]; }
};

struct RowsT {
  long long s0, e0;
  bool succ, chain;
};

__device__ __forceinline__ RowsT rows_of_t(const Inst &I, long long tile) {
  const long long n = I.n, L = I.tile_rows;
  RowsT T;
  if (I.pad & 1) {
    const long long lane = tile & 31;
    const long long g0 = (tile >> 5) * (32 * L - kOvT - kLane0ShortT);
    T.s0 = lane == 0 ? g0 : g0 + lane * L - kLane0ShortT;
    const long long len = lane == 0 ? L - kLane0ShortT : (lane == 31 ? L - kOvT : L);
    T.e0 = min(T.s0 + len, n);
    T.succ = lane < 31 && T.e0 < n;
    T.chain = lane > 0;
  } else {
    T.s0 = tile * L;
    T.e0 = min(T.s0 + L, n);
    T.succ = T.chain = false;
  }
  return T;
}

struct FwdOutT {
  long long rlast;
  float A, B;
  int K;
  unsigned bad;
};

__device__ FwdOutT tile_forward_t(const Inst &I, const RowsT &T, const ScrT &S) {
  const long long n = I.n;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const long long s0 = T.s0, e0 = T.e0;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  unsigned bad = 0;
  long long r;
  float cp_start = 0.0f;
  if (T.chain) {
    const long long i0 = max(s0 - 1 - kHaloCT, 0LL);
    float c = (i0 == 0 && !nat0) ? 0.5f : 0.0f;  // exact at row 0, a guess elsewhere
    double xb = x[i0 + 1];
    float hp = dif32_near(xb, x[i0]);
    for (long long i = i0 + 1; i <= s0 - 1; ++i) {
      const double xc = x[i + 1];
      const float hi = dif32_near(xc, xb);
      c = hi * rcp32(2.0f * (hp + hi) - hp * c);
      hp = hi;
      xb = xc;
    }
    cp_start = c;
    r = s0 - 1;
  } else {
    r = max(s0 - kLane0ShortT, 0LL);
  }
  FwdM F;
  {
    const double x0 = x[r], x1 = x[r + 1], y0 = y[r], y1 = y[r + 1];
    F.xa = F.ya = F.xb = F.yb = 0.0;
    if (r + 2 < n) { F.xa = x[r + 2]; F.ya = y[r + 2]; }
    if (r + 3 < n) { F.xb = x[r + 3]; F.yb = y[r + 3]; }
    const float h = dif32_near(x1, x0), ih = rcp32(h), sl = quot32(dy32(y1, y0), h, ih);
    F.xn = x1; F.yn = y1; F.h = h; F.s = sl;
    if (T.chain) {
      F.cp = cp_start;
      F.dp = 0.0f;
    } else if (r == 0 && !nat0) {
      F.cp = 0.5f;
      F.dp = 3.0f * (sl - to_f32(I.yp1)) * ih;
    } else {
      F.cp = 0.0f;
      F.dp = 0.0f;
    }
    if (r >= s0) {
      S.at(0, 0) = F.cp; S.at(0, 1) = F.dp;
      bad |= row_check(x0, y0, true, x1);
    }
  }
  FwdOutT out;
  out.A = out.B = 0.0f;
  float M = 1.0f;
  int K = 0;
  bool track = T.chain;
  const long long rlast = T.succ ? e0 - 1 : min(e0 + kOvT, n) - 1;
  while (r < rlast) {
    const long long j = r + 1;
    const bool owned = (j >= s0 && j < e0);
    const float a = F.h;
    float cpj, dpj, iden;
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
      iden = rcp32(2.0f * (F.h + hj) - F.h * F.cp);
      cpj = hj * iden;
      dpj = (6.0f * (sj - F.s) - F.h * F.dp) * iden;
      F.xn = x2; F.yn = y2; F.h = hj; F.s = sj;
    } else {
      if (owned) bad |= row_check(F.xn, F.yn, false, 0.0);
      cpj = 0.0f;
      iden = rcp32(2.0f * F.h - F.h * F.cp);
      dpj = nat1 ? 0.0f : (6.0f * (to_f32(I.ypn) - F.s) - F.h * F.dp) * iden;
    }
    F.cp = cpj; F.dp = dpj;
    r = j;
    if (j >= s0) { S.at(j - s0, 0) = cpj; S.at(j - s0, 1) = dpj; }
    if (track) {  // d'_j = (r_j - a_j d'_{j-1}) / den_j: the sensitivity picks up -a_j / den_j
      M *= (j == n - 1 && nat1) ? 0.0f : -a * iden;
      S.m(K++) = M;
      if (!(fabsf(M) >= kMStopT) || K == kMRowsT) track = false;
    }
    if (j == e0 - 1) {
      out.A = dpj;
      out.B = track ? M : 0.0f;
    }
  }
  out.rlast = rlast;
  out.K = K;
  out.bad = bad;
  return out;
}

// Forward sweep of the refinement's correction system A delta = r, r = d - A Z (the residual of
// the stored binary32 Z in double-float arithmetic from exact double-float widths and value
// differences), with the binary32 matrix of the first pass; the tile's start as in
// tile_forward_t (halo, or chained with the same sensitivities: the matrix is the same).
struct FwdRT {
  double xn, yn;  // x_{r+1}, y_{r+1}
  double xa, ya;  // x_{r+2}, y_{r+2}
  F2 h, s;        // h_r, s_r
  float zr, zn, za;  // Z_r, Z_{r+1}, Z_{r+2}
  float cp, dp;
};

__device__ FwdOutT tile_forward_rt(const Inst &I, const RowsT &T, const ScrT &S) {
  const long long n = I.n;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const float *__restrict__ z = I.z;
  const long long s0 = T.s0, e0 = T.e0;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  long long r;
  float cp_start = 0.0f;
  if (T.chain) {
    const long long i0 = max(s0 - 1 - kHaloCT, 0LL);
    float c = (i0 == 0 && !nat0) ? 0.5f : 0.0f;
    double xb = x[i0 + 1];
    float hp = dif32_near(xb, x[i0]);
    for (long long i = i0 + 1; i <= s0 - 1; ++i) {
      const double xc = x[i + 1];
      const float hi = dif32_near(xc, xb);
      c = hi * rcp32(2.0f * (hp + hi) - hp * c);
      hp = hi;
      xb = xc;
    }
    cp_start = c;
    r = s0 - 1;
  } else {
    r = max(s0 - kLane0ShortT, 0LL);
  }
  FwdRT F;
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
    if (T.chain) {
      F.cp = cp_start;
      F.dp = 0.0f;
    } else if (r == 0 && !nat0) {
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
    if (r >= s0) { S.at(0, 0) = F.cp; S.at(0, 1) = F.dp; }
  }
  FwdOutT out;
  out.A = out.B = 0.0f;
  out.bad = 0;
  float M = 1.0f;
  int K = 0;
  bool track = T.chain;
  const long long rlast = T.succ ? e0 - 1 : min(e0 + kOvT, n) - 1;
  while (r < rlast) {
    const long long j = r + 1;
    const float hf = F.h.hi;
    float cpj, dpj, iden;
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
      iden = rcp32(2.0f * (hf + hj.hi) - hf * F.cp);
      cpj = hj.hi * iden;
      dpj = ((res.hi + res.lo) - hf * F.dp) * iden;
      F.xn = x2; F.yn = y2; F.h = hj; F.s = sj; F.zr = F.zn; F.zn = z2;
    } else {  // last row
      cpj = 0.0f;
      iden = rcp32(2.0f * hf - hf * F.cp);
      if (nat1) {
        dpj = -F.zn;  // y''_{n-1} = 0
      } else {
        const F2 d = df_mul_f(df_add(f2_of(I.ypn), df_neg(F.s)), 6.0f);
        const F2 az = df_add(df_mul_f(F.h, F.zr), df_mul_f(F.h, 2.0f * F.zn));
        const F2 res = df_add(d, df_neg(az));
        dpj = ((res.hi + res.lo) - hf * F.dp) * iden;
      }
    }
    F.cp = cpj; F.dp = dpj;
    r = j;
    if (j >= s0) { S.at(j - s0, 0) = cpj; S.at(j - s0, 1) = dpj; }
    if (track) {
      M *= (j == n - 1 && nat1) ? 0.0f : -hf * iden;
      S.m(K++) = M;
      if (!(fabsf(M) >= kMStopT) || K == kMRowsT) track = false;
    }
    if (j == e0 - 1) {
      out.A = dpj;
      out.B = track ? M : 0.0f;
    }
  }
  out.rlast = rlast;
  out.K = K;
  return out;
}

// Back substitution from the tile's top, fused with the evaluation.  kMode 0: the recurrence
// gives y''; output y'' and S(x_k).  kMode 1 (first pass of the refined path): output y'' in
// binary32 to the scratch I.z, no evaluation.  kMode 2 (refinement): the recurrence gives the
// correction delta of the stored binary32 Z; y'' = Z + delta is output (the sum in binary64) and
// evaluated.
template <int kMode>
__device__ void tile_bwd_eval_t(const Inst &I, const RowsT &T, long long rlast, const ScrT &S) {
  const long long n = I.n, m = kMode == 1 ? 0 : I.m;
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const float *__restrict__ z = I.z;
  const long long s0 = T.s0, e0 = T.e0;
  const long long te = e0 - 1 - s0;
  float Y;
  long long t;
  if (T.succ) {
    const ScrT Sn{S.base, S.mb, S.lane + 1};
    long long u = min(e0 + kOvT, n) - 1 - e0;
    Y = Sn.at(u, 1);
    for (--u; u >= 0; --u) Y = Sn.at(u, 1) - Sn.at(u, 0) * Y;
    t = te;
  } else {
    t = rlast - s0;
    Y = S.at(t, 1);
    for (--t; t > te; --t) Y = S.at(t, 1) - S.at(t, 0) * Y;
  }
  // a row's outputs from its recurrence value v; returns the row's binary32 y''
  auto out_row = [&](long long row, float v) -> float {
    if (kMode == 1) {
      I.z[row] = v;
      return v;
    }
    if (kMode == 2) {
      const float zr = z[row];
      if (I.ypp) I.ypp[row] = to_f64(zr) + to_f64(v);
      return zr + v;
    }
    if (I.ypp) I.ypp[row] = to_f64(v);
    return v;
  };
  if (t == te - 1) out_row(n - 1, Y);
  if (t < 0) return;
  if (kMode == 1) {  // no evaluation: the back substitution alone, loads one row ahead
    float c = S.at(t, 0), d = S.at(t, 1);
    for (; t >= 0; --t) {
      const float cc = c, dd = d;
      if (t > 0) { c = S.at(t - 1, 0); d = S.at(t - 1, 1); }
      Y = dd - cc * Y;
      out_row(s0 + t, Y);
    }
    return;
  }
  const bool evaluate = (m > 0 && s0 <= n - 2);
  const Grid G = make_grid(x, n, m);
  const long long klo = evaluate ? first_query(G, x, s0) : 0;
  long long k = evaluate ? ((e0 <= n - 2) ? first_query(G, x, e0) - 1 : m - 1) : -1;
  // current row t: recurrence values (Yt, Yt1) and binary32 y'' (Pt, Pt1) of rows t and t+1,
  // knots and values, and the interval's binary32 width, reciprocal and values; the next row
  // down is loaded one step ahead
  float Yt1 = Y;
  float Pt1 = kMode == 2 ? z[s0 + t + 1] + Y : Y;
  double xt1 = x[s0 + t + 1], xt = x[s0 + t];
  double ytd1 = y[s0 + t + 1], ytd = y[s0 + t];
  float Yt = S.at(t, 1) - S.at(t, 0) * Yt1;
  float Pt = out_row(s0 + t, Yt);
  float fy1 = to_f32(ytd1), fy0 = to_f32(ytd);
  float ba = dif32_near(xt1, xt), iba = rcp32(ba);
  float c_n = 0.0f, d_n = 0.0f;
  double x_n = 0.0, y_n = 0.0;
  auto load_next = [&](long long row) {
    if (row >= 0) {
      if (row >= 8) {
        prefetch_l1m(&S.at(row - 8, 0));
        if (first_in_block(x + s0 + row - 8)) prefetch_l1m(x + s0 + row - 8);
        if (first_in_block(y + s0 + row - 8)) prefetch_l1m(y + s0 + row - 8);
      }
      c_n = S.at(row, 0); d_n = S.at(row, 1);
      x_n = x[s0 + row]; y_n = y[s0 + row];
    }
  };
  load_next(t - 1);
  auto step_down = [&]() {
    --t;
    Yt1 = Yt; Pt1 = Pt; xt1 = xt; fy1 = fy0;
    xt = x_n; ytd = y_n;
    Yt = d_n - c_n * Yt1;
    Pt = out_row(s0 + t, Yt);
    load_next(t - 1);
    fy0 = to_f32(ytd);
    ba = dif32_near(xt1, xt);
    iba = rcp32(ba);
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
    const float xa = dif32_near(q, xt);
    I.yq[k] = to_f64(newint32(xa, ba - xa, fy0, fy1, Pt, Pt1, ba, iba));
    if (I.jq) I.jq[k] = (int32_t)(s0 + t);
    q = qn;
  }
  while (t > 0) step_down();
}

__device__ __forceinline__ void tile_correct_t(const FwdOutT &o, float delta, const ScrT &S) {
  for (int k = 0; k < o.K; ++k) S.at(k, 1) = fmaf(S.m(k), delta, S.at(k, 1));
}

template <int kMode>  // 0: fit + eval, 1: fit only (refined path), 2: refine + eval
__global__ void __launch_bounds__(kThreadsT, 1)
    mixed_tiled_kernel(const Inst *__restrict__ insts, int ninst, long long total_tiles,
                       unsigned long long *__restrict__ counter, float *__restrict__ scratch, long long rows_cap) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  float *wbase = scratch + (size_t)warp * (rows_cap * 2 + kMRowsT) * 32;
  const ScrT S{wbase, wbase + (size_t)rows_cap * 2 * 32, lane};
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total_tiles) break;
    const long long t = (long long)base + lane;
    Inst I;
    RowsT T;
    T.s0 = T.e0 = 0;
    T.succ = T.chain = false;
    FwdOutT o;
    o.rlast = -1;
    o.A = o.B = 0.0f;
    o.K = 0;
    o.bad = 0;
    if (t < total_tiles) {
      const int i = find_inst(insts, ninst, t);
      I = insts[i];
      T = rows_of_t(I, t - I.tile_begin);
      if (T.s0 < I.n) o = kMode == 2 ? tile_forward_rt(I, T, S) : tile_forward_t(I, T, S);
    }
    float sa = o.A, sb = o.B;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float pa = __shfl_up_sync(0xffffffffu, sa, off), pb = __shfl_up_sync(0xffffffffu, sb, off);
      if (lane >= off) {
        sa = fmaf(sb, pa, sa);
        sb *= pb;
      }
    }
    const float delta = __shfl_up_sync(0xffffffffu, sa, 1);
    if (o.rlast >= 0 && T.chain) tile_correct_t(o, delta, S);
    __syncwarp();
    if (o.rlast >= 0) {
      tile_bwd_eval_t<kMode>(I, T, o.rlast, S);
      if (o.bad) atomicOr(I.status, o.bad);
    }
    __syncwarp();
  }
}

int tiled_mixed_overhang_rows() { return kOvT; }
int tiled_mixed_threads_per_sm() { return kThreadsT; }

long long threads_tiled_mixed(int sm_count, long long total_tiles) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles, kThreadsT, &blocks, &bt);
  return (long long)blocks * bt;
}
int tiled_mixed_lane0_short_rows() { return kLane0ShortT; }

size_t scratch_bytes_tiled_mixed(long long threads, int tile_rows) {
  const long long warps = (threads + 31) / 32;
  return (size_t)warps * (((size_t)tile_rows + kOvT) * 2 + kMRowsT) * 32 * sizeof(float);
}

cudaError_t launch_tiled_mixed(const Inst *d_insts, int ninst, long long total_tiles, float *scratch, int tile_rows,
                               int sm_count, unsigned long long *counter, cudaStream_t stream, int mode) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles, kThreadsT, &blocks, &bt);
  const unsigned grid = (unsigned)blocks, block = (unsigned)bt;
  const long long rows_cap = (long long)tile_rows + kOvT;
  switch (mode) {
    case 1: mixed_tiled_kernel<1><<<grid, block, 0, stream>>>(d_insts, ninst, total_tiles, counter, scratch, rows_cap); break;
    case 2: mixed_tiled_kernel<2><<<grid, block, 0, stream>>>(d_insts, ninst, total_tiles, counter, scratch, rows_cap); break;
    default: mixed_tiled_kernel<0><<<grid, block, 0, stream>>>(d_insts, ninst, total_tiles, counter, scratch, rows_cap); break;
  }
  return cudaGetLastError();
}

}  // namespace spl
