// Warp-cooperative binary32 fit + evaluation ("scan" form of the mixed-precision path).
//
// The same system and arithmetic as the binary32 ring kernel (spl_fused_mixed.cu: tridiagonal system of eq.
// (init_val) with the end rows of "Start and End Derivatives", Thomas recurrences of
// "Implementation", the one-division form of "Fast Interpolation" on the grid of "Curve
// Interpolation"; binary32 arithmetic on exact, once-rounded differences of the binary64
// inputs), laid out the other way round: a warp solves one tile of rows, 32 consecutive rows
// at a time, lane l holding row R + l.  Every global access of a warp is then one contiguous
// run (coalesced), and the recurrences become warp scans:
//   * c'_j = c_j / (b_j - a_j c'_{j-1}) contracts errors in c'_{j-1} by 1/12 or more per row
//     (diagonal dominance), so a few relaxation sweeps across the lanes reach the sequential
//     values;
//   * d'_j = (d_j - a_j d'_{j-1}) / den_j and the back substitution y''_j = d'_j - c'_j y''_{j+1}
//     are affine maps, composed by an inclusive scan (the second one from the top down);
//   * the queries of a chunk's 32 intervals are evaluated 32 at a time, lane-parallel: each finds
//     its interval among the lanes' knots by a 5-step search on the order-preserving keys (so
//     brackets stay bit-identical to the sequential sweep) and gathers the interval's data by
//     shuffles.
// A tile starts its forward sweep 64 rows early from a guessed state (the guess error decays by
// <= 2/3 per row for d' and <= 1/12 for c') and its back substitution 32 rows past its end (the
// error decays by c' < 1/2 per row).  (c', d') of the tile's rows, with the binary32 width and
// value the evaluation needs, go to a per-warp scratch (16 bytes per row, a few tens of MB for
// all warps: L2-resident between the two sweeps), so the back substitution re-reads only the
// knots.
// Exact differences of neighbouring knots take the integer/FP32 route: with 16 warps per SM
// the kernel is bound by instruction throughput, where the FP64 pipe (~1/64 of the FP32 rate)
// is the scarce unit.
#include <algorithm>

#include "spl_device.cuh"
#include "spl_internal.h"
#include "spl_mixed_math.cuh"
#include "spl_numeric.h"

namespace spl {

constexpr int kThreadsS = 1024;  // one CTA per SM (more warps hide the scans' shuffle latency)
constexpr int kHaloS = 64;      // forward rows before a tile (a multiple of 32)
constexpr int kOvS = 32;        // back-substitution start past a tile
constexpr unsigned kFullS = 0xffffffffu;
constexpr int kRelaxS = 8;     // relaxation sweeps of the c' recurrence in a chunk

__device__ __forceinline__ double shfl_f64(double v, int src) {
  return __longlong_as_double(__shfl_sync(kFullS, __double_as_longlong(v), src));
}
__device__ __forceinline__ long long shfl_i64(long long v, int src) { return __shfl_sync(kFullS, v, src); }

// Least k in [0, m] with x_k > v on the uniform grid (x_0 <= v): an estimate from the grid step,
// corrected on the exact grid points.
__device__ __forceinline__ long long first_above(const Grid &G, double v, double inv_step) {
  if (G.m <= 1) return (G.m == 1 && dkey(G.x0) <= dkey(v)) ? 1 : 0;
  const double e = (v - G.x0) * inv_step;
  long long k = !(e >= 0.0) ? 0 : (e >= (double)G.m ? G.m : (long long)e + 1);
  const long long kv = dkey(v);
  while (k > 0 && dkey(G.at(k - 1)) > kv) --k;
  while (k < G.m && dkey(G.at(k)) <= kv) ++k;
  return k;
}

// One tile: rows [s0, e0) of instance I.  kMode 0: fit + evaluation; 1: fit only, the binary32
// y'' to I.z (first pass of the refined path); 2: one refinement step of I.z (the residual
// r = d - A Z in double-float arithmetic from exact double-float widths and value differences,
// A delta = r solved with the binary32 matrix), y'' = Z + delta, and the evaluation.
template <int kMode>
__device__ void scan_tile(const Inst &I, long long tile, float4 *__restrict__ W, int lane) {
  const long long n = I.n, TR = I.tile_rows;
  const long long s0 = tile * TR, e0 = min(s0 + TR, n);
  const long long f0 = max(s0 - kHaloS, 0LL), f1 = min(e0 + kOvS, n);
  const double *__restrict__ x = I.x;
  const double *__restrict__ y = I.y;
  const float *__restrict__ z = I.z;
  const bool nat0 = is_natural(I.yp1), nat1 = is_natural(I.ypn);
  const float yp1f = nat0 ? 0.0f : to_f32(I.yp1), ypnf = nat1 ? 0.0f : to_f32(I.ypn);
  unsigned bad = 0;

  // ---- forward sweep, rows f0 .. f1-1 ----
  // row R-1 (a guess at a tile's start): c', d', width, slope (double-float in the refinement), Z
  float cp = 0.0f, dp = 0.0f, zp = 0.0f;
  F2 hp{0.0f, 0.0f}, sp{0.0f, 0.0f};
  // rows of the next chunk are loaded one chunk ahead (rows up to f1, the row past the sweep
  // giving the last row's width and slope)
  const long long lim = min(f1 + 1, n);
  double xn = (f0 + lane < lim) ? x[f0 + lane] : 0.0, yn = (f0 + lane < lim) ? y[f0 + lane] : 0.0;
  float zn = (kMode == 2 && f0 + lane < lim) ? z[f0 + lane] : 0.0f;
  for (long long R = f0; R < f1; R += 32) {
    const long long j = R + lane;
    const bool act = j < f1, hasn = act && j <= n - 2;
    const double x0 = xn, y0 = yn;
    const float z0 = zn;
    xn = (j + 32 < lim) ? x[j + 32] : 0.0;
    yn = (j + 32 < lim) ? y[j + 32] : 0.0;
    if (kMode == 2) zn = (j + 32 < lim) ? z[j + 32] : 0.0f;
    const double xf = shfl_f64(xn, 0), yf = shfl_f64(yn, 0);  // row R+32
    double x1 = shfl_f64(x0, (lane + 1) & 31), y1 = shfl_f64(y0, (lane + 1) & 31);
    if (lane == 31) {
      x1 = xf;
      y1 = yf;
    }
    F2 hF{0.0f, 0.0f}, sF{0.0f, 0.0f};
    if (hasn) {
      if (kMode == 2) {
        hF = dif2(x1, x0);
        sF = df_div(dif2(y1, y0), hF, rcp32(hF.hi));
      } else {
        hF.hi = dif32_up(x1, x0);
        sF.hi = quot32(dy32(y1, y0), hF.hi, rcp32(hF.hi));
      }
    }
    const float h = hF.hi;
    if (kMode != 2 && act && j >= s0 && j < e0) bad |= row_check(x0, y0, j <= n - 2, x1);
    F2 hm{__shfl_up_sync(kFullS, hF.hi, 1), 0.0f}, sm{__shfl_up_sync(kFullS, sF.hi, 1), 0.0f};
    if (kMode == 2) {
      hm.lo = __shfl_up_sync(kFullS, hF.lo, 1);
      sm.lo = __shfl_up_sync(kFullS, sF.lo, 1);
    }
    if (lane == 0) {
      hm = hp;
      sm = sp;
    }
    // row j: a y''_{j-1} + b y''_j + c y''_{j+1} = d (the refinement: the same matrix, d the residual)
    float a = hm.hi, b = 2.0f * (hm.hi + h), c = h, d;
    if (kMode == 2) {
      float zm = __shfl_up_sync(kFullS, z0, 1);
      const float zf = __shfl_sync(kFullS, zn, 0);
      float z1 = __shfl_down_sync(kFullS, z0, 1);
      if (lane == 0) zm = zp;
      if (lane == 31) z1 = zf;
      F2 res;
      if (j == 0) {
        a = 0.0f;
        if (nat0) {
          b = 1.0f; c = 0.0f;
          res = F2{-z0, 0.0f};  // natural first row: y''_0 = 0
        } else {
          b = 2.0f * h;
          const F2 dd = df_mul_f(df_add(sF, df_neg(f2_of(I.yp1))), 6.0f);
          res = df_add(dd, df_neg(df_add(df_mul_f(hF, 2.0f * z0), df_mul_f(hF, z1))));
        }
      } else if (j == n - 1) {
        c = 0.0f;
        if (nat1) {
          a = 0.0f; b = 1.0f;
          res = F2{-z0, 0.0f};  // y''_{n-1} = 0
        } else {
          b = 2.0f * hm.hi;
          const F2 dd = df_mul_f(df_add(f2_of(I.ypn), df_neg(sm)), 6.0f);
          res = df_add(dd, df_neg(df_add(df_mul_f(hm, zm), df_mul_f(hm, 2.0f * z0))));
        }
      } else {
        const F2 dd = df_mul_f(df_add(sF, df_neg(sm)), 6.0f);
        const F2 az = df_add(df_add(df_mul_f(hm, zm), df_mul_f(df_add(hm, hF), 2.0f * z0)), df_mul_f(hF, z1));
        res = df_add(dd, df_neg(az));
      }
      d = res.hi + res.lo;
      zp = __shfl_sync(kFullS, z0, (int)min(31LL, f1 - 1 - R));
    } else {
      d = 6.0f * (sF.hi - sm.hi);
      if (j == 0) {
        a = 0.0f;
        if (nat0) { b = 1.0f; c = 0.0f; d = 0.0f; }
        else { b = 2.0f * h; d = 6.0f * (sF.hi - yp1f); }
      } else if (j == n - 1) {
        c = 0.0f;
        if (nat1) { a = 0.0f; b = 1.0f; d = 0.0f; }
        else { b = 2.0f * hm.hi; d = 6.0f * (ypnf - sm.hi); }
      }
    }
    if (!act) { a = 0.0f; b = 1.0f; c = 0.0f; d = 0.0f; }
    // c'_j = c_j / (b_j - a_j c'_{j-1}): relaxation across the lanes from the guess c'_{j-1} = 0.
    // The map contracts errors in c'_{j-1} by at most h_j h_{j-1} / (1.5 h_{j-1} + 2 h_j)^2 <= 1/12,
    // so after kRelaxS sweeps every lane is within 12^-8 / 2 (< 2^-29) of the sequential value; lane 0
    // starts from the carried c'_{R-1}.
    // The sweeps before the last use the MUFU reciprocal alone (~1 ulp): they only move the
    // guess, the last one forms the refined 1/den that the d' step uses.
    float cj = c * rcp_approx32(b - a * (lane == 0 ? cp : 0.0f)), iden = 0.0f;
#pragma unroll
    for (int it = 0; it < kRelaxS; ++it) {
      float cm = __shfl_up_sync(kFullS, cj, 1);
      if (lane == 0) cm = cp;
      iden = it + 1 < kRelaxS ? rcp_approx32(b - a * cm) : rcp32(b - a * cm);
      cj = c * iden;
    }
    // d': scan of the affine maps t -> (-a/den) t + d/den, applied to d'_{R-1}
    float A = -a * iden, B = d * iden;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float A2 = __shfl_up_sync(kFullS, A, off), B2 = __shfl_up_sync(kFullS, B, off);
      if (lane >= off) {
        B = fmaf(A, B2, B);
        A *= A2;
      }
    }
    const float dj = fmaf(A, dp, B);
    if (act) W[j - f0] = make_float4(cj, dj, h, kMode == 1 ? 0.0f : to_f32(y0));
    const int last = (int)min(31LL, f1 - 1 - R);
    cp = __shfl_sync(kFullS, cj, last);
    dp = __shfl_sync(kFullS, dj, last);
    hp.hi = __shfl_sync(kFullS, hF.hi, last);
    sp.hi = __shfl_sync(kFullS, sF.hi, last);
    if (kMode == 2) {
      hp.lo = __shfl_sync(kFullS, hF.lo, last);
      sp.lo = __shfl_sync(kFullS, sF.lo, last);
    }
  }

  // ---- back substitution from row f1-1 down to s0, fused with the evaluation ----
  const long long rt = f1 - 1;
  const long long m = I.m;
  const bool evaluate = kMode != 1 && m > 0 && s0 <= n - 2;
  const Grid G = make_grid(x, n, m);
  const double inv_step = (m >= 2) ? 1.0 / G.step : 0.0;
  // queries of the tile's intervals s0 .. min(e0, n-1)-1: klo .. khi-1, taken from the top down
  // in batches of 32 (lane l: the l-th next one); a chunk takes the leading queries of a batch
  // that lie above its lowest knot, the rest go to the chunks below
  long long khi = 0, klo = 0;
  if (evaluate) {
    khi = (e0 >= n - 1) ? m : (finite64(x[e0]) ? first_above(G, x[e0], inv_step) : 0);
    klo = (s0 == 0) ? 0 : (finite64(x[s0]) ? min(first_above(G, x[s0], inv_step), khi) : khi);
  }
  float ycarry = 0.0f;  // recurrence value of row R+32 (a guess above the top row)
  float pcarry = 0.0f;  // binary32 y'' of row R+32
  float fytop = 0.0f;   // binary32 y_{R+32}
  // the next chunk down (scratch, knots, stored Z) is loaded one chunk ahead
  const long long Rtop = f0 + ((rt - f0) >> 5 << 5);
  float4 cdn = (Rtop + lane <= rt) ? W[Rtop + lane - f0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  double xjn = (evaluate && Rtop + lane <= rt) ? x[Rtop + lane] : 0.0;
  float zjn = (kMode == 2 && Rtop + lane <= rt) ? z[Rtop + lane] : 0.0f;
  for (long long R = Rtop; R >= s0; R -= 32) {
    const long long j = R + lane;
    const bool act = j <= rt;
    const float4 cd = cdn;
    const double xj = xjn;
    const float zj = zjn;
    if (R - 32 >= s0) {  // rows below R are all inside the forward range
      cdn = W[j - 32 - f0];
      if (evaluate) xjn = x[j - 32];
      if (kMode == 2) zjn = z[j - 32];
    }
    float A = act ? -cd.x : 1.0f, B = act ? cd.y : 0.0f;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float A2 = __shfl_down_sync(kFullS, A, off), B2 = __shfl_down_sync(kFullS, B, off);
      if (lane + off < 32) {
        B = fmaf(A, B2, B);
        A *= A2;
      }
    }
    const float v = fmaf(A, ycarry, B);  // y''_j, or the correction delta_j of the refinement
    const float ypp = kMode == 2 ? zj + v : v;
    const bool own = j >= s0 && j < e0;
    if (kMode == 1) {
      if (own) I.z[j] = v;
    } else if (own && I.ypp) {
      I.ypp[j] = kMode == 2 ? to_f64(zj) + to_f64(v) : to_f64(v);
    }
    if (evaluate) {
      const float fy = cd.w;
      float fy1 = __shfl_down_sync(kFullS, fy, 1), yp1 = __shfl_down_sync(kFullS, ypp, 1);
      if (lane == 31) {
        fy1 = fytop;
        yp1 = pcarry;
      }
      const int hi = (int)(min(min(R + 31, e0 - 1), n - 2) - R);
      if (R < e0 && hi >= 0) {  // the chunk holds intervals of the tile: R .. R+hi
        float ba = 1.0f, iba = 1.0f;
        if (lane <= hi) {
          ba = cd.z;
          iba = rcp32(ba);
        }
        const long long key = dkey(xj);
        const long long keyR = shfl_i64(key, 0);
        while (khi > klo) {
          const long long k = khi - 1 - lane;
          const bool qa = k >= klo;
          const double q = qa ? G.at(k) : xj;
          const long long kq = dkey(q);
          const bool in = qa && (R == s0 || kq > keyR);
          const int cnt = __popc(__ballot_sync(kFullS, in));
          // the interval: largest l in [0, hi] with x_{R+l} < q (0 when none: the first interval)
          int l = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = l + step;
            const long long kc = shfl_i64(key, cand & 31);
            if (cand <= hi && kc < kq) l = cand;
          }
          const double xl = shfl_f64(xj, l);
          const float fl = __shfl_sync(kFullS, fy, l), fl1 = __shfl_sync(kFullS, fy1, l);
          const float pl = __shfl_sync(kFullS, ypp, l), pl1 = __shfl_sync(kFullS, yp1, l);
          const float bl = __shfl_sync(kFullS, ba, l), ibl = __shfl_sync(kFullS, iba, l);
          if (in) {
            const float xa = dif32_up(q, xl);
            I.yq[k] = to_f64(newint32(xa, bl - xa, fl, fl1, pl, pl1, bl, ibl));
            if (I.jq) I.jq[k] = (int32_t)(R + l);
          }
          khi -= cnt;
          if (cnt < 32) break;
        }
      }
      fytop = __shfl_sync(kFullS, fy, 0);
    }
    ycarry = __shfl_sync(kFullS, v, 0);
    pcarry = __shfl_sync(kFullS, ypp, 0);
  }
  if (bad) atomicOr(I.status, bad);
}

template <int kMode>
__global__ void __launch_bounds__(kThreadsS, 1)
    mixed_scan_kernel(const Inst *__restrict__ insts, int ninst, long long total_tiles,
                      unsigned long long *__restrict__ counter, float4 *__restrict__ scratch, long long rows_cap) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float4 *W = scratch + (size_t)warp * rows_cap;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(counter, 1ull);
    t = __shfl_sync(kFullS, t, 0);
    if ((long long)t >= total_tiles) break;
    const int i = find_inst(insts, ninst, (long long)t);
    const Inst I = insts[i];
    scan_tile<kMode>(I, (long long)t - I.tile_begin, W, lane);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// Persistent serving loop (continuous batching).  Warp 0 of CTA 0 is the scheduler: it reads
// request entries that the host appends to a ring in mapped host memory, installs each in its
// device slot, maps the request's tiles into the device tile map and publishes them by
// advancing `published`.  Every other warp is a worker: it claims one tile ticket at a time and,
// once the ticket is published, solves that tile of that request with the warp-cooperative
// binary32 fit + evaluation above (scan_tile<0>, in the warp's own scratch).  The warp finishing
// a request's last tile writes the request's status and sequence number to mapped host memory.
// All waits are
// bounded: the scheduler leaves after `idle_ns` without work or at `deadline_ns`, and sets
// `stop`; workers leave once stop is set and every published tile is claimed.  The host
// relaunches the loop when new work arrives.  Launched cooperatively (one CTA per SM), so the
// scheduler and the workers are co-resident.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreadsS, 1) serve_kernel(ServeArgs a) {
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

  // workers: one ticket per warp; lane 0 waits for it (bounded) and the warp solves the tile
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float4 *W = a.scan_scratch + (size_t)warp * a.scan_rows_cap;
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
    scan_tile<0>(I, (long long)(t - __ldcg(a.slot_first + slot)), W, lane);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
      const unsigned done = atomicAdd(a.slot_done + slot, 1u) + 1u;
      if (done == (unsigned)I.ntiles) {
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

cudaError_t launch_serve(const ServeArgs &args, int sm_count, cudaStream_t stream) {
  ServeArgs copy = args;
  void *params[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)serve_kernel, dim3((unsigned)sm_count), dim3(kThreadsS), params, 0,
                                     stream);
}

int serve_tile_rows(int tile_rows) { return std::max(32, (tile_rows + 31) / 32 * 32); }
long long serve_rows_cap(int tile_rows) { return (long long)serve_tile_rows(tile_rows) + kHaloS + kOvS; }
size_t serve_scratch_bytes(int sm_count, int tile_rows) {
  return (size_t)sm_count * (kThreadsS / 32) * (size_t)serve_rows_cap(tile_rows) * sizeof(float4);
}


int scan_mixed_threads_per_sm() { return kThreadsS; }

// rows of one tile: a multiple of 32, about two tiles per resident warp for one instance
int scan_mixed_tile_rows(long long total_points, int sm_count, int count) {
  const long long warps = (long long)sm_count * (kThreadsS / 32);
  long long L = count > 1 ? 1024 : (total_points + 2 * warps - 1) / (2 * warps);
  L = (L + 31) / 32 * 32;
  return (int)std::max<long long>(std::min<long long>(L, 1 << 20), 256);
}

long long threads_scan_mixed(int sm_count, long long total_tiles) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles * 32, kThreadsS, &blocks, &bt);
  return (long long)blocks * bt;
}

size_t scratch_bytes_scan_mixed(long long threads, int tile_rows) {
  const long long warps = (threads + 31) / 32;
  return (size_t)warps * ((size_t)tile_rows + kHaloS + kOvS) * sizeof(float4);
}

cudaError_t launch_scan_mixed(const Inst *d_insts, int ninst, long long total_tiles, float *scratch, int tile_rows,
                              int sm_count, unsigned long long *counter, cudaStream_t stream, int mode) {
  int blocks, bt;
  spread_grid(sm_count, total_tiles * 32, kThreadsS, &blocks, &bt);
  const long long rows_cap = (long long)tile_rows + kHaloS + kOvS;
  float4 *W = reinterpret_cast<float4 *>(scratch);
  switch (mode) {
    case 1: mixed_scan_kernel<1><<<(unsigned)blocks, (unsigned)bt, 0, stream>>>(d_insts, ninst, total_tiles, counter, W, rows_cap); break;
    case 2: mixed_scan_kernel<2><<<(unsigned)blocks, (unsigned)bt, 0, stream>>>(d_insts, ninst, total_tiles, counter, W, rows_cap); break;
    default: mixed_scan_kernel<0><<<(unsigned)blocks, (unsigned)bt, 0, stream>>>(d_insts, ninst, total_tiles, counter, W, rows_cap); break;
  }
  return cudaGetLastError();
}

}  // namespace spl
