// Host runtime behind include/spl.h: contexts, plans, the arena sub-allocator, request
// submission / completion tracking and reusable graph-captured batches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/spl.h"
#include "spl_internal.h"

using spl::Inst;

namespace {

constexpr uint64_t kAlign = 256;

uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// Per-launch status block: one status word per instance, then two tile counters (one per
// kernel of the launch), all zeroed before the launch.  Direct launches (LaunchPlan::direct) use
// none: their status word is pinned host memory and their counter and exchange area the context's.
uint64_t status_words_bytes(uint64_t count) { return round_up(4 * count, 16); }
// (a single instance's block also holds the exchange area of the multi-CTA FP64 kernel)
uint64_t status_block_bytes(uint64_t count) {
  return status_words_bytes(count) + 16 + (count == 1 ? spl::mid_f64_exchange_bytes() : 0);
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit free-list allocator over [0, cap) with coalescing; offsets are kAlign-aligned.
class Pool {
 public:
  void init(uint64_t cap) {
    free_.clear();
    cap_ = cap / kAlign * kAlign;
    if (cap_) free_[0] = cap_;
    used_ = high_ = 0;
  }
  uint64_t capacity() const { return cap_; }
  uint64_t high_water() const { return high_; }
  bool alloc(uint64_t size, uint64_t *off) {
    size = round_up(std::max<uint64_t>(size, 1), kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= size) {
        *off = it->first;
        uint64_t rest = it->second - size;
        uint64_t at = it->first + size;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += size;
        high_ = std::max(high_, used_);
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t size) {
    size = round_up(std::max<uint64_t>(size, 1), kAlign);
    used_ -= size;
    auto it = free_.emplace(off, size).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t cap_ = 0, used_ = 0, high_ = 0;
};

struct Block {
  uint64_t off = 0, size = 0;
};

}  // namespace

struct spl_plan {
  spl_ctx *ctx;
  uint64_t max_n;
  int precision;
  int refine_steps;
  int tile_rows;
  int query_mode;
  int eval_variant;
  unsigned fault_flags;
};

struct Job;

struct Ticket {
  Job *job;
  int index;
  double t_submit;
};

struct Job {
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  cudaEvent_t ev_in = nullptr, ev_kernel = nullptr;  // host-memory requests: copies pipelined
  std::vector<Block> dev_blocks;   // arena blocks, released once the GPU is done
  Block pin_block;                 // pinned staging block
  int count = 0;
  int slots_base = -1;
  int remaining = 0;               // tickets not collected yet
  bool done = false;
  float ms = 0.f;
  unsigned *h_status = nullptr;    // pinned, count words
};

struct spl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t s_in = nullptr, s_out = nullptr;  // copy streams of host-memory requests (lazy)
  char *arena = nullptr;
  bool own_arena = false;
  int max_slots = 1;
  int sm_count = 0;
  std::mutex mu;
  Pool dev;
  Pool pin;
  char *pinned = nullptr;          // pinned staging (descriptors, statuses)
  char *pinned_dev = nullptr;      // the same memory as the device addresses it
  uint64_t pinned_bytes = 0;
  // Direct launches (one instance in device memory on a latency kernel; see LaunchPlan::direct):
  // possible when the device's atomics on host memory are native.  Their arena area: the
  // multi-CTA FP64 kernel's exchange area, then the binary32 kernel's tile counter (which that
  // kernel leaves at zero); and the last launch number written into the exchange area.
  bool direct_ok = false;
  uint64_t direct_off = 0;
  unsigned long long xchg_launch = 0;
  int slots_used = 0;
  uint64_t next_ticket = 1;
  std::unordered_map<uint64_t, Ticket> tickets;
  spl_stats stats{};
};

struct spl_batch {
  spl_ctx *ctx = nullptr;
  int count = 0;
  std::vector<Block> dev_blocks;
  Block pin_block;
  unsigned *h_status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_done = nullptr;
  bool launched = false;
  int launches_per_replay = 0;
};

namespace {

spl_status cuda_fail(cudaError_t e) { return e == cudaSuccess ? SPL_OK : SPL_ERR_CUDA; }

spl_status map_status_bits(unsigned bits) {
  if (bits & spl::kStBadTile) return SPL_ERR_INVALID_ARG;
  if (bits & spl::kStNonFinite) return SPL_ERR_NONFINITE;
  if (bits & spl::kStNotIncreasing) return SPL_ERR_NOT_INCREASING;
  if (bits & spl::kStWaitTimeout) return SPL_ERR_TIMEOUT;
  return SPL_OK;
}

bool slope_ok(double s) { return !std::isnan(s) && !(std::isinf(s) && s < 0); }

// Plan options that spl_plan_create accepts.
bool plan_desc_ok(const spl_plan_desc *d) {
  if (d->max_n < 3) return false;
  if (d->precision != SPL_PREC_F64 && d->precision != SPL_PREC_F32_REFINE) return false;
  if (d->refine_steps < 0 || d->refine_steps > 1) return false;
  if (d->precision == SPL_PREC_F64 && d->refine_steps != 0) return false;
  if (d->tile_rows != 0 && d->tile_rows < 16) return false;
  if (d->query_mode != SPL_QUERY_UNIFORM && d->query_mode != SPL_QUERY_EXPLICIT) return false;
  if (d->eval_variant < SPL_EVAL_ORIG || d->eval_variant > SPL_EVAL_NOOP) return false;
  if (d->fault_flags & ~1u) return false;
  return true;
}

spl_status check_request(const spl_plan *plan, const spl_request *r) {
  if (!r) return SPL_ERR_INVALID_ARG;
  if (r->n < 3 || r->n > plan->max_n) return SPL_ERR_INVALID_ARG;
  if (r->n > (1ull << 40) || r->m > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  if (!r->x || !r->y) return SPL_ERR_INVALID_ARG;
  if (r->m > 0 && !r->yq_out) return SPL_ERR_INVALID_ARG;
  if (!slope_ok(r->yp1) || !slope_ok(r->ypn)) return SPL_ERR_INVALID_ARG;
  if (r->mem != SPL_MEM_DEVICE && r->mem != SPL_MEM_HOST) return SPL_ERR_INVALID_ARG;
  if (plan->query_mode == SPL_QUERY_EXPLICIT) {
    if (r->m > 0 && !r->xq) return SPL_ERR_INVALID_ARG;
  } else if (r->xq) {
    return SPL_ERR_INVALID_ARG;
  }
  return SPL_OK;
}

// Launch geometry: persistent CTAs, tiles fetched dynamically.  The FP64 kernel runs 448
// threads per SM, one tile per thread (its measured best between FP64-pipe latency hiding and
// the per-tile work more tiles bring); the warp-cooperative binary32 kernel 640, one tile per
// warp.
long long threads_for(const spl_ctx *c, int precision, long long total_tiles) {
  return precision == SPL_PREC_F64 ? spl::threads_f64(c->sm_count, total_tiles)
                                   : spl::threads_scan_mixed(c->sm_count, total_tiles);
}

// Tile length (one tile per thread) for the tiled FP64 kernel, so that one instance of
// total_points fills every thread of one wave; never shorter than a few halos.  FP64 tiles come
// in warp groups of 32L - overhang - lane0_short rows, so L is chosen for the group count to
// match the warps.
int auto_tile_rows(int sm_count, uint64_t total_points, uint32_t count) {
  // several instances: short tiles, fetched dynamically, balance instances of uneven sizes
  // (one wave of long tiles waits on the longest; 4,096 log-uniform instances run ~1.4x faster)
  if (count > 1) return 128;
  // One instance too small to keep the GPU's FP64 pipes busy with long tiles (an explicit tile
  // length or a stored fit keeps it on this kernel; otherwise it takes the multi-CTA kernel):
  // its time is then one tile's serial dependency chain (halo, tile, back-substitution start,
  // one thread), so short tiles spread it over more warps.  Measured on GB300 for n = 1e3..1e5:
  // 16-row tiles halve the time (0.36-0.41 -> 0.17 ms); past a few 1e5 points the halo work that
  // every short tile repeats outweighs the shorter chain, and from ~1e6 the grouped long tiles
  // below win.
  const uint64_t upto16 = (uint64_t)sm_count * 2000ull;
  const uint64_t upto32 = (uint64_t)sm_count * 8000ull;
  if (total_points <= upto16) return 16;
  if (total_points <= upto32) return 32;
  const long long target = (long long)sm_count * spl::f64_threads_per_sm();
  const long long warps = std::max<long long>(target / 32, 1);
  const long long per_warp = (long long)((total_points + warps - 1) / warps);
  long long L = (per_warp + spl::overhang_rows_f64() + spl::lane0_short_rows_f64() + 31) / 32;
  L = std::max<long long>(L, 128);
  L = std::min<long long>(L, 1 << 20);
  return (int)L;
}

// The launch shape of a submission: which kernel fits it and with what tiling, as a pure function
// of the plan's options, the instances' sizes, where their arrays live and the SM count (no
// device state).  prepare() builds the launch from it; spl_launch_geometry reports it.
struct PathChoice {
  int fit_kernel = SPL_KERNEL_NONE;  // spl_kernel
  bool separate_eval = false;        // explicit queries or a stored fit: the evaluation kernel
  int tile_rows = 0;                 // knots per tile in the descriptors
  long long cta_rows = 0, ctas = 0;  // the multi-CTA FP64 kernel's grid
  bool direct = false;               // a direct launch where the device allows it (LaunchPlan::direct)
};

PathChoice choose_path(int precision, int plan_tile_rows, int query_mode, bool fit, bool device_mem,
                       const uint64_t *ns, uint32_t count, int sm_count) {
  PathChoice pc;
  uint64_t total_points = 0;
  for (uint32_t i = 0; i < count; ++i) total_points += ns[i];
  pc.separate_eval = query_mode == SPL_QUERY_EXPLICIT || !fit;
  if (precision == SPL_PREC_F32_REFINE) {
    // the warp-cooperative kernel for every binary32 launch (one thread per tile was 2-6x slower
    // even on batches of instances of a few hundred knots): tiles of whole 32-row chunks, no
    // longer than its shared memory holds
    pc.tile_rows = plan_tile_rows > 0 ? std::min((plan_tile_rows + 31) / 32 * 32, spl::scan_mixed_tile_max())
                                      : spl::scan_mixed_tile_rows((long long)total_points, sm_count, (int)count);
  } else {
    pc.tile_rows = plan_tile_rows > 0 ? plan_tile_rows : auto_tile_rows(sm_count, total_points, count);
  }
  if (!fit) return pc;
  if (precision == SPL_PREC_F32_REFINE) {
    pc.fit_kernel = SPL_KERNEL_SCAN_MIXED;
  } else {
    pc.fit_kernel = SPL_KERNEL_FUSED_F64;
    if (plan_tile_rows == 0 && !pc.separate_eval) {
      // one instance up to SMs x 9,600 knots: the multi-CTA kernel (its latency is a piece's FP64
      // chain); up to two waves of instances of at most 4,096 knots (two CTAs fit an SM): one CTA
      // each.  More instances go to the tiled kernel, whose throughput then wins (4,096 instances
      // of 3..4,096 knots: 0.98 ms against 1.24 ms; 512 of 1,000..4,096: 0.43 ms against 0.27 ms).
      const long long cr = count == 1 ? spl::mid_f64_cta_rows((long long)ns[0], sm_count) : 0;
      if (cr > 0) {
        pc.fit_kernel = SPL_KERNEL_MID_F64;
        pc.cta_rows = cr;
        pc.ctas = ((long long)ns[0] + cr - 1) / cr;
      } else {
        bool small = count <= 4u * (uint32_t)sm_count;
        for (uint32_t i = 0; i < count; ++i) small = small && ns[i] <= (uint64_t)spl::small_f64_max_rows();
        if (small) pc.fit_kernel = SPL_KERNEL_SMALL_F64;
      }
    }
  }
  pc.direct = count == 1 && device_mem && !pc.separate_eval &&
              (pc.fit_kernel == SPL_KERNEL_MID_F64 || pc.fit_kernel == SPL_KERNEL_SCAN_MIXED);
  return pc;
}

// Instances from this many knots up get a coarse key table for the bisection of explicit query
// positions (below it the whole knot array stays in L2 anyway).
constexpr uint64_t kCoarseMinKnots = 1ull << 16;

struct Staged {
  std::vector<Block> dev;
  Block pin;
  bool ok = true;
};

// Everything one launch needs, carved from the arena and the pinned pool.
struct LaunchPlan {
  int precision = SPL_PREC_F64;
  int refine_steps = 0;
  int tile_rows = 0;
  std::vector<Inst> insts;
  long long total_tiles = 0;
  long long threads = 0;
  uint64_t ring_bytes = 0;
  bool fit = true;             // run the fit kernel(s)
  bool small_f64 = false;      // FP64: every instance small enough for one CTA (latency path)
  bool mid_f64 = false;        // FP64: one instance on a cooperative grid of CTAs (latency path)
  unsigned fault_flags = 0;    // failure-detection tests (the plan's)
  bool separate_eval = false;  // evaluate with the separate kernel (explicit queries, stored y'')
  // Direct launch: one instance in device memory, fit + evaluation on the multi-CTA FP64 kernel or
  // the binary32 kernel.  The descriptor goes as a kernel parameter, the kernel ORs its status bits
  // straight into the job's pinned status word (zeroed by the host), the FP64 kernel's exchange
  // flags carry a launch number and the binary32 kernel's tile counter resets itself: no memset,
  // upload or status copy around the kernel (~13 us less per request on GB300).
  bool direct = false;
  int eval_variant = 0;
  long long total_queries = 0;
  // host-memory staging: device copies of inputs/outputs
  struct HostIO {
    const double *hx, *hy, *hxq, *hyppin;
    double *hypp, *hyq;
    int32_t *hjq;
    uint64_t n, m;
    uint64_t off_x, off_y, off_ypp, off_yq, off_jq, off_xq, off_yppin;
  };
  std::vector<HostIO> hio;
};

void release_blocks(spl_ctx *c, std::vector<Block> &blocks) {
  for (auto &b : blocks) c->dev.release(b.off, b.size);
  blocks.clear();
}

bool dev_alloc(spl_ctx *c, uint64_t size, std::vector<Block> &blocks, uint64_t *off) {
  uint64_t o;
  if (!c->dev.alloc(size, &o)) return false;
  blocks.push_back({o, round_up(std::max<uint64_t>(size, 1), kAlign)});
  *off = o;
  return true;
}

// Build descriptors, allocate the arena blocks and pinned staging for `count` requests.
// Returns SPL_OK, SPL_ERR_BUDGET (can never fit) or SPL_ERR_QUEUE_FULL (not now).
spl_status prepare(spl_ctx *c, spl_plan *p, const spl_request *reqs, uint32_t count, LaunchPlan &lp,
                   std::vector<Block> &dev_blocks, Block &pin_block, uint64_t *d_insts_off,
                   uint64_t *d_status_off, uint64_t *d_ring_off, bool allow_direct) {
  uint64_t total_points = 0;
  std::vector<uint64_t> ns(count);
  for (uint32_t i = 0; i < count; ++i) {
    ns[i] = reqs[i].n;
    total_points += reqs[i].n;
  }
  lp.precision = p->precision;
  lp.refine_steps = p->precision == SPL_PREC_F64 ? 0 : p->refine_steps;
  lp.fit = reqs[0].ypp_in == nullptr;
  const PathChoice pc = choose_path(p->precision, p->tile_rows, p->query_mode, lp.fit,
                                    reqs[0].mem == SPL_MEM_DEVICE, ns.data(), count, c->sm_count);
  lp.separate_eval = pc.separate_eval;
  const int L = pc.tile_rows;
  lp.eval_variant = p->eval_variant;
  lp.fault_flags = p->fault_flags;
  lp.mid_f64 = pc.fit_kernel == SPL_KERNEL_MID_F64;
  lp.small_f64 = pc.fit_kernel == SPL_KERNEL_SMALL_F64;
  lp.direct = allow_direct && c->direct_ok && pc.direct;
  lp.insts.resize(count);
  // Instances of 32 tiles or more of the FP64 kernel use the grouped geometry: their tiles
  // start on a warp boundary, and each warp's 32 tiles cover 32L - overhang - lane0_short rows
  // (the lanes take the rows past their tile from the next lane and, but for the first, their
  // start state from the previous one)
  const long long ov = p->precision == SPL_PREC_F64 ? spl::overhang_rows_f64() : 0;
  const long long l0s = p->precision == SPL_PREC_F64 ? spl::lane0_short_rows_f64() : 0;
  long long tiles = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const spl_request &r = reqs[i];
    Inst &I = lp.insts[i];
    std::memset(&I, 0, sizeof(I));
    I.x = r.x; I.y = r.y; I.ypp = r.ypp_out; I.yq = r.yq_out; I.jq = r.jq_out;
    I.n = (long long)r.n; I.m = (long long)r.m;
    I.yp1 = r.yp1; I.ypn = r.ypn;
    I.tile_rows = L;
    I.ntiles = ((long long)r.n + L - 1) / L;
    if (ov > 0 && I.ntiles >= 32 && L > ov + l0s &&
        8 * 32 * (((long long)r.n + 32LL * L - ov - l0s - 1) / (32LL * L - ov - l0s)) <= 9 * I.ntiles) {
      const long long G = 32LL * L - ov - l0s;
      tiles = (tiles + 31) / 32 * 32;
      I.ntiles = 32 * (((long long)r.n + G - 1) / G);
      I.pad = 1;
    }
    I.tile_begin = tiles;
    tiles += I.ntiles;
    if (lp.separate_eval) {  // the fit kernel sees no queries; the evaluation kernel takes them
      I.xq = r.xq;
      I.mq = I.m;
      I.m = 0;
      I.q_begin = lp.total_queries;
      lp.total_queries += I.mq;
      if (!lp.fit) I.ypp = const_cast<double *>(r.ypp_in);
    }
  }
  lp.total_tiles = tiles;
  lp.threads = threads_for(c, p->precision, tiles);
  lp.tile_rows = L;
  lp.ring_bytes = (lp.fit && p->precision == SPL_PREC_F64 && !lp.small_f64 && !lp.mid_f64)
                      ? spl::ring_bytes_f64(lp.threads, L)
                      : 0;

  // footprint check against the whole budget first
  uint64_t need = round_up(sizeof(Inst) * count, kAlign) + round_up(status_block_bytes(count), kAlign) +
                  round_up(lp.ring_bytes, kAlign);
  // a fit feeding the separate evaluation needs y'' somewhere: the caller's ypp_out or scratch
  auto needs_ypp_scratch = [&](const spl_request &r) {
    return lp.separate_eval && lp.fit && r.m > 0 && (!r.ypp_out || r.mem == SPL_MEM_HOST);
  };
  for (uint32_t i = 0; i < count; ++i) {
    const spl_request &r = reqs[i];
    if (r.mem == SPL_MEM_HOST) {
      need += round_up(8 * r.n, kAlign) * 2;
      if (r.ypp_out && lp.fit) need += round_up(8 * r.n, kAlign);
      if (r.m) need += round_up(8 * r.m, kAlign);
      if (r.jq_out && r.m) need += round_up(4 * r.m, kAlign);
      if (r.xq && r.m) need += round_up(8 * r.m, kAlign);
      if (r.ypp_in) need += round_up(8 * r.n, kAlign);
    } else if (needs_ypp_scratch(r)) {
      need += round_up(8 * r.n, kAlign);
    }
  }
  // explicit query positions on a large instance: the coarse key table of its bisection (scratch)
  auto coarse_bytes = [&](const spl_request &r) -> uint64_t {
    return (lp.separate_eval && r.xq && r.m > 0 && r.n >= kCoarseMinKnots)
               ? 8ull * (uint64_t)spl::coarse_key_entries((long long)r.n)
               : 0;
  };
  for (uint32_t i = 0; i < count; ++i) need += round_up(coarse_bytes(reqs[i]), kAlign);
  // refined mixed path: binary32 y'' of the first pass, one float per knot (scratch)
  const uint64_t z_bytes = lp.refine_steps > 0 ? 4 * total_points : 0;
  need += round_up(z_bytes, kAlign);
  if (need > c->dev.capacity()) return SPL_ERR_BUDGET;
  uint64_t pin_need = sizeof(Inst) * count + 4ull * count + 64;
  if (pin_need > c->pin.capacity()) return SPL_ERR_BUDGET;

  *d_insts_off = *d_status_off = 0;
  bool ok = lp.direct || (dev_alloc(c, sizeof(Inst) * count, dev_blocks, d_insts_off) &&
                          dev_alloc(c, status_block_bytes(count), dev_blocks, d_status_off));
  ok = ok && dev_alloc(c, lp.ring_bytes, dev_blocks, d_ring_off);
  if (ok && z_bytes) {
    uint64_t zoff = 0;
    ok = dev_alloc(c, z_bytes, dev_blocks, &zoff);
    uint64_t acc = 0;
    for (uint32_t i = 0; ok && i < count; ++i) {
      lp.insts[i].z = reinterpret_cast<float *>(c->arena + zoff) + acc;
      acc += reqs[i].n;
    }
  }
  for (uint32_t i = 0; ok && i < count; ++i) {
    const spl_request &r = reqs[i];
    if (r.mem != SPL_MEM_HOST) {
      if (needs_ypp_scratch(r)) {  // device request: y'' for the evaluation, not returned
        uint64_t off = 0;
        ok = dev_alloc(c, 8 * r.n, dev_blocks, &off);
        if (ok) lp.insts[i].ypp = reinterpret_cast<double *>(c->arena + off);
      }
      continue;
    }
    LaunchPlan::HostIO h{};
    h.hx = r.x; h.hy = r.y; h.hyq = r.yq_out; h.hjq = r.jq_out;
    h.hypp = lp.fit ? r.ypp_out : nullptr;
    h.hxq = (r.xq && r.m) ? r.xq : nullptr;
    h.hyppin = r.ypp_in;
    h.n = r.n; h.m = r.m;
    ok = dev_alloc(c, 8 * r.n, dev_blocks, &h.off_x) && dev_alloc(c, 8 * r.n, dev_blocks, &h.off_y);
    const bool dev_ypp = (lp.fit && r.ypp_out) || needs_ypp_scratch(r) || r.ypp_in;
    if (ok && dev_ypp) ok = dev_alloc(c, 8 * r.n, dev_blocks, &h.off_ypp);
    if (ok && r.m) ok = dev_alloc(c, 8 * r.m, dev_blocks, &h.off_yq);
    if (ok && r.jq_out && r.m) ok = dev_alloc(c, 4 * r.m, dev_blocks, &h.off_jq);
    if (ok && h.hxq) ok = dev_alloc(c, 8 * r.m, dev_blocks, &h.off_xq);
    h.off_yppin = h.off_ypp;
    if (ok) {
      Inst &I = lp.insts[i];
      I.x = reinterpret_cast<const double *>(c->arena + h.off_x);
      I.y = reinterpret_cast<const double *>(c->arena + h.off_y);
      I.ypp = dev_ypp ? reinterpret_cast<double *>(c->arena + h.off_ypp) : nullptr;
      I.yq = r.m ? reinterpret_cast<double *>(c->arena + h.off_yq) : nullptr;
      I.jq = (r.jq_out && r.m) ? reinterpret_cast<int32_t *>(c->arena + h.off_jq) : nullptr;
      if (h.hxq) I.xq = reinterpret_cast<const double *>(c->arena + h.off_xq);
      lp.hio.push_back(h);
    }
  }
  for (uint32_t i = 0; ok && i < count; ++i) {
    const uint64_t cb = coarse_bytes(reqs[i]);
    if (!cb) continue;
    uint64_t off = 0;
    ok = dev_alloc(c, cb, dev_blocks, &off);
    if (ok) lp.insts[i].ktab = reinterpret_cast<const long long *>(c->arena + off);
  }
  uint64_t poff = 0;
  if (ok) ok = c->pin.alloc(pin_need, &poff);
  if (!ok) {
    release_blocks(c, dev_blocks);
    return SPL_ERR_QUEUE_FULL;
  }
  pin_block = {poff, round_up(pin_need, kAlign)};
  // status words: the launch's status block, or for a direct launch the job's pinned words (at the
  // offset where the job keeps them, after the descriptors)
  unsigned *status0 = lp.direct ? reinterpret_cast<unsigned *>(c->pinned_dev + poff + round_up(sizeof(Inst) * count, 64))
                                : reinterpret_cast<unsigned *>(c->arena + *d_status_off);
  for (uint32_t i = 0; i < count; ++i) lp.insts[i].status = status0 + i;
  return SPL_OK;
}

// The kernel(s) of the hot path for the plan's precision.
cudaError_t launch_path(spl_ctx *c, const LaunchPlan &lp, uint64_t d_insts_off, uint64_t d_ring_off,
                        uint64_t d_status_off, cudaStream_t st, int *launches) {
  const Inst *insts = reinterpret_cast<const Inst *>(c->arena + d_insts_off);
  const int count = (int)lp.insts.size();
  unsigned long long *counters =
      reinterpret_cast<unsigned long long *>(c->arena + d_status_off + status_words_bytes(count));
  cudaError_t e = cudaSuccess;
  if (!lp.fit) {
    // stored y'': evaluation only
  } else if (lp.precision == SPL_PREC_F64 && lp.mid_f64) {
    e = spl::launch_mid_f64(insts, nullptr, lp.insts[0].n, counters + 2, 0, c->sm_count, lp.fault_flags, st);
    if (launches) *launches += 1;
  } else if (lp.precision == SPL_PREC_F64 && lp.small_f64) {
    e = spl::launch_small_f64(insts, count, st);
    if (launches) *launches += 1;
  } else if (lp.precision == SPL_PREC_F64) {
    e = spl::launch_fused_f64(insts, count, lp.total_tiles, reinterpret_cast<double *>(c->arena + d_ring_off),
                              lp.tile_rows, c->sm_count, counters, st);
    if (launches) *launches += 1;
  } else if (lp.refine_steps == 0) {
    e = spl::launch_scan_mixed(insts, nullptr, count, lp.total_tiles, c->sm_count, counters, st, 0);
    if (launches) *launches += 1;
  } else {
    e = spl::launch_scan_mixed(insts, nullptr, count, lp.total_tiles, c->sm_count, counters, st, 1);
    if (e == cudaSuccess)
      e = spl::launch_scan_mixed(insts, nullptr, count, lp.total_tiles, c->sm_count, counters + 1, st, 2);
    if (launches) *launches += 2;
  }
  if (e == cudaSuccess && lp.separate_eval && lp.total_queries > 0) {
    bool uniform = true;
    long long coarse = 0;
    for (const Inst &I : lp.insts) {
      uniform = uniform && I.xq == nullptr;
      if (I.ktab) coarse = std::max(coarse, spl::coarse_key_entries(I.n));
    }
    e = spl::launch_eval(insts, count, lp.total_queries, lp.eval_variant, lp.precision != SPL_PREC_F64, uniform,
                         coarse, c->sm_count, st);
    if (launches) *launches += coarse > 0 ? 2 : 1;
  }
  return e;
}

// Enqueue the launch described by lp: statuses cleared, descriptors uploaded, host inputs
// copied in, the fused kernel, outputs and statuses copied back.  Device-memory requests run
// everything on the context's stream.  Host-memory requests put their input copies on the
// context's input-copy stream and their output copies (and the status words) on its
// output-copy stream, ordered against the kernels by events, so that the copies of one request
// overlap the kernels of its neighbours; the job is then complete when its output copies are.
cudaError_t enqueue(spl_ctx *c, const LaunchPlan &lp, char *pin_base, unsigned *h_status, uint64_t d_insts_off,
                    uint64_t d_status_off, uint64_t d_ring_off, cudaStream_t st, int *launches, Job *job) {
  const int count = (int)lp.insts.size();
  if (lp.direct) {  // the kernel(s) alone, on the context's stream
    const Inst &I = lp.insts[0];
    h_status[0] = 0u;  // the kernel ORs its status bits into this word
    cudaError_t e;
    char *area = c->arena + c->direct_off;
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(area + spl::mid_f64_exchange_bytes());
    if (lp.mid_f64) {
      e = spl::launch_mid_f64(nullptr, &I, I.n, area, ++c->xchg_launch, c->sm_count, lp.fault_flags, st);
      if (launches) *launches += 1;
    } else if (lp.refine_steps == 0) {
      e = spl::launch_scan_mixed(nullptr, &I, 1, lp.total_tiles, c->sm_count, counter, st, 0);
      if (launches) *launches += 1;
    } else {
      e = spl::launch_scan_mixed(nullptr, &I, 1, lp.total_tiles, c->sm_count, counter, st, 1);
      if (e == cudaSuccess) e = spl::launch_scan_mixed(nullptr, &I, 1, lp.total_tiles, c->sm_count, counter, st, 2);
      if (launches) *launches += 2;
    }
    return e;
  }
  const bool piped = !lp.hio.empty() && job && c->s_in && c->s_out;
  cudaStream_t s_in = piped ? c->s_in : st, s_out = piped ? c->s_out : st;
  std::memcpy(pin_base, lp.insts.data(), sizeof(Inst) * count);
  // statuses and descriptors go with the inputs: on the input stream when the copies are
  // pipelined, so that the kernel waits on one event and no small copy of the kernel's stream
  // queues behind a neighbour's large input copy on the copy engine
  cudaError_t e = cudaMemsetAsync(c->arena + d_status_off, 0, status_block_bytes(count), s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->arena + d_insts_off, pin_base, sizeof(Inst) * count, cudaMemcpyHostToDevice, s_in);
  for (const auto &h : lp.hio) {
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(c->arena + h.off_x, h.hx, 8 * h.n, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->arena + h.off_y, h.hy, 8 * h.n, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess && h.hxq)
      e = cudaMemcpyAsync(c->arena + h.off_xq, h.hxq, 8 * h.m, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess && h.hyppin)
      e = cudaMemcpyAsync(c->arena + h.off_yppin, h.hyppin, 8 * h.n, cudaMemcpyHostToDevice, s_in);
  }
  if (piped) {
    if (e == cudaSuccess) e = cudaEventRecord(job->ev_in, s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, job->ev_in, 0);
  }
  if (e == cudaSuccess) e = launch_path(c, lp, d_insts_off, d_ring_off, d_status_off, st, launches);
  if (piped) {
    if (e == cudaSuccess) e = cudaEventRecord(job->ev_kernel, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, job->ev_kernel, 0);
  }
  for (const auto &h : lp.hio) {
    if (e != cudaSuccess) break;
    if (h.hypp) e = cudaMemcpyAsync(h.hypp, c->arena + h.off_ypp, 8 * h.n, cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess && h.m)
      e = cudaMemcpyAsync(h.hyq, c->arena + h.off_yq, 8 * h.m, cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess && h.hjq && h.m)
      e = cudaMemcpyAsync(h.hjq, c->arena + h.off_jq, 4 * h.m, cudaMemcpyDeviceToHost, s_out);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_status, c->arena + d_status_off, 4ull * count, cudaMemcpyDeviceToHost, s_out);
  return e;
}

void finish_job(spl_ctx *c, Job *j) {
  // the GPU is done with everything the job used
  release_blocks(c, j->dev_blocks);
  cudaEventElapsedTime(&j->ms, j->ev_start, j->ev_done);
  j->done = true;
}

void free_job(spl_ctx *c, Job *j) {
  if (!j->done) release_blocks(c, j->dev_blocks);
  c->pin.release(j->pin_block.off, j->pin_block.size);
  c->slots_used -= j->count;
  if (j->ev_start) cudaEventDestroy(j->ev_start);
  if (j->ev_done) cudaEventDestroy(j->ev_done);
  if (j->ev_in) cudaEventDestroy(j->ev_in);
  if (j->ev_kernel) cudaEventDestroy(j->ev_kernel);
  delete j;
}

}  // namespace

int spl_ctx_device(spl_ctx *c) { return c->device; }
int spl_ctx_sms(spl_ctx *c) { return c->sm_count; }
char *spl_ctx_arena_base(spl_ctx *c) { return c->arena; }
bool spl_ctx_arena_alloc(spl_ctx *c, uint64_t bytes, uint64_t *off) {
  std::lock_guard<std::mutex> lk(c->mu);
  return c->dev.alloc(bytes, off);
}
void spl_ctx_arena_release(spl_ctx *c, uint64_t off, uint64_t bytes) {
  std::lock_guard<std::mutex> lk(c->mu);
  c->dev.release(off, bytes);
}
void spl_ctx_count_launch(spl_ctx *c, int n) {
  std::lock_guard<std::mutex> lk(c->mu);
  c->stats.kernel_launches += (uint64_t)n;
}

extern "C" {

const char *spl_status_str(int32_t s) {
  switch (s) {
    case SPL_OK: return "ok";
    case SPL_PENDING: return "pending";
    case SPL_ERR_INVALID_ARG: return "invalid argument";
    case SPL_ERR_NOT_INCREASING: return "knots not strictly increasing";
    case SPL_ERR_NONFINITE: return "non-finite knot or value";
    case SPL_ERR_BUDGET: return "request exceeds the memory budget";
    case SPL_ERR_QUEUE_FULL: return "no free slot or memory now";
    case SPL_ERR_TIMEOUT: return "timed out";
    case SPL_ERR_CUDA: return "CUDA error";
    case SPL_ERR_UNKNOWN_TICKET: return "unknown ticket";
    case SPL_ERR_STATE: return "invalid in the current state";
    default: return "unknown status";
  }
}

spl_status spl_create(spl_ctx **out, const spl_ctx_desc *d) {
  if (!out || !d || d->max_slots < 1 || d->arena_bytes < (1u << 20)) return SPL_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev) return SPL_ERR_CUDA;
  if (cudaSetDevice(d->device) != cudaSuccess) return SPL_ERR_CUDA;
  std::unique_ptr<spl_ctx> c(new (std::nothrow) spl_ctx());
  if (!c) return SPL_ERR_CUDA;
  c->device = d->device;
  c->stream = static_cast<cudaStream_t>(d->stream);
  c->max_slots = d->max_slots;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess)
    return SPL_ERR_CUDA;
  if (d->arena) {
    c->arena = static_cast<char *>(d->arena);
    if (reinterpret_cast<uintptr_t>(c->arena) % kAlign) return SPL_ERR_INVALID_ARG;
  } else {
    if (cudaMalloc(&c->arena, d->arena_bytes) != cudaSuccess) return SPL_ERR_CUDA;
    c->own_arena = true;
  }
  c->dev.init(d->arena_bytes);
  c->pinned_bytes = round_up((uint64_t)d->max_slots * (sizeof(Inst) + 8) + 4096, kAlign) * 2;
  if (cudaHostAlloc(&c->pinned, c->pinned_bytes, cudaHostAllocMapped) != cudaSuccess) {
    if (c->own_arena) cudaFree(c->arena);
    return SPL_ERR_CUDA;
  }
  c->pin.init(c->pinned_bytes);
  // direct launches: the pinned memory's device address, native atomics on host memory (the
  // kernels OR status bits into it), and their arena area, zeroed once here on the context's
  // stream, which every later launch follows (launch numbers start at 1)
  int native = 0;
  void *pdev = nullptr;
  const uint64_t area = spl::mid_f64_exchange_bytes() + 16;
  bool ok = cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, d->device) == cudaSuccess &&
            cudaHostGetDevicePointer(&pdev, c->pinned, 0) == cudaSuccess && pdev &&
            c->dev.alloc(area, &c->direct_off) &&
            cudaMemsetAsync(c->arena + c->direct_off, 0, area, c->stream) == cudaSuccess;
  if (!ok) {
    cudaFreeHost(c->pinned);
    if (c->own_arena) cudaFree(c->arena);
    return SPL_ERR_CUDA;
  }
  c->pinned_dev = static_cast<char *>(pdev);
  c->direct_ok = native != 0;
  *out = c.release();
  return SPL_OK;
}

void spl_destroy(spl_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->s_in) cudaStreamSynchronize(c->s_in);
  if (c->s_out) cudaStreamSynchronize(c->s_out);
  std::vector<Job *> jobs;
  for (auto &kv : c->tickets) jobs.push_back(kv.second.job);
  std::sort(jobs.begin(), jobs.end());
  jobs.erase(std::unique(jobs.begin(), jobs.end()), jobs.end());
  for (Job *j : jobs) {
    if (!j->done) finish_job(c, j);
    free_job(c, j);
  }
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->own_arena) cudaFree(c->arena);
  if (c->s_in) cudaStreamDestroy(c->s_in);
  if (c->s_out) cudaStreamDestroy(c->s_out);
  delete c;
}

spl_status spl_plan_create(spl_ctx *c, const spl_plan_desc *d, spl_plan **out) {
  if (!c || !d || !out) return SPL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!plan_desc_ok(d)) return SPL_ERR_INVALID_ARG;
  spl_plan *p = new (std::nothrow) spl_plan();
  if (!p) return SPL_ERR_CUDA;
  p->ctx = c;
  p->max_n = d->max_n;
  p->precision = d->precision;
  p->refine_steps = d->refine_steps;
  p->tile_rows = d->tile_rows;
  p->query_mode = d->query_mode;
  p->eval_variant = d->eval_variant;
  p->fault_flags = d->fault_flags;
  *out = p;
  return SPL_OK;
}

void spl_plan_destroy(spl_plan *p) { delete p; }

spl_status spl_submit_batch(spl_ctx *c, spl_plan *p, const spl_request *reqs, uint32_t count, uint64_t *tickets) {
  if (!c || !p || !reqs || !tickets || count == 0 || p->ctx != c) return SPL_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    spl_status s = check_request(p, &reqs[i]);
    if (s != SPL_OK) return s;
    if (reqs[i].mem != reqs[0].mem) return SPL_ERR_INVALID_ARG;
    if ((reqs[i].ypp_in == nullptr) != (reqs[0].ypp_in == nullptr)) return SPL_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  if ((int)count > c->max_slots) return SPL_ERR_BUDGET;
  if (c->slots_used + (int)count > c->max_slots) return SPL_ERR_QUEUE_FULL;
  if (cudaSetDevice(c->device) != cudaSuccess) return SPL_ERR_CUDA;
  LaunchPlan lp;
  std::vector<Block> blocks;
  Block pb;
  uint64_t oi = 0, os = 0, orr = 0;
  spl_status s = prepare(c, p, reqs, count, lp, blocks, pb, &oi, &os, &orr, true);
  if (s != SPL_OK) return s;
  Job *j = new (std::nothrow) Job();
  if (!j) {
    release_blocks(c, blocks);
    c->pin.release(pb.off, pb.size);
    return SPL_ERR_CUDA;
  }
  j->dev_blocks = std::move(blocks);
  j->pin_block = pb;
  j->count = (int)count;
  j->remaining = (int)count;
  c->slots_used += (int)count;
  char *pin_base = c->pinned + pb.off;
  j->h_status = reinterpret_cast<unsigned *>(pin_base + round_up(sizeof(Inst) * count, 64));
  cudaError_t e = cudaEventCreate(&j->ev_start);
  if (e == cudaSuccess) e = cudaEventCreate(&j->ev_done);
  const bool host_io = !lp.hio.empty();
  if (host_io && e == cudaSuccess && !c->s_in) e = cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking);
  if (host_io && e == cudaSuccess && !c->s_out) e = cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking);
  if (host_io && e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev_in, cudaEventDisableTiming);
  if (host_io && e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev_kernel, cudaEventDisableTiming);
  cudaStream_t s_first = host_io ? c->s_in : c->stream, s_last = host_io ? c->s_out : c->stream;
  if (e == cudaSuccess) e = cudaEventRecord(j->ev_start, s_first);
  int launches = 0;
  if (e == cudaSuccess) e = enqueue(c, lp, pin_base, j->h_status, oi, os, orr, c->stream, &launches, j);
  if (e == cudaSuccess) e = cudaEventRecord(j->ev_done, s_last);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(c->stream);
    if (c->s_in) cudaStreamSynchronize(c->s_in);
    if (c->s_out) cudaStreamSynchronize(c->s_out);
    free_job(c, j);
    return SPL_ERR_CUDA;
  }
  c->stats.kernel_launches += launches;
  const double t = now_ms();
  for (uint32_t i = 0; i < count; ++i) {
    uint64_t tk = c->next_ticket++;
    c->tickets[tk] = Ticket{j, (int)i, t};
    tickets[i] = tk;
  }
  return SPL_OK;
}

spl_status spl_submit(spl_ctx *c, spl_plan *p, const spl_request *r, uint64_t *ticket) {
  return spl_submit_batch(c, p, r, 1, ticket);
}

spl_status spl_poll(spl_ctx *c, uint64_t ticket, spl_result *res) {
  if (!c) return SPL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->tickets.find(ticket);
  if (it == c->tickets.end()) return SPL_ERR_UNKNOWN_TICKET;
  Ticket &t = it->second;
  Job *j = t.job;
  if (!j->done) {
    cudaError_t q = cudaEventQuery(j->ev_done);
    if (q == cudaErrorNotReady) {
      if (res) { res->status = SPL_PENDING; res->device_ms = 0; res->latency_ms = now_ms() - t.t_submit; }
      return SPL_PENDING;
    }
    if (q != cudaSuccess) return SPL_ERR_CUDA;
    finish_job(c, j);
  }
  spl_status st = map_status_bits(j->h_status[t.index]);
  if (res) { res->status = st; res->device_ms = j->ms; res->latency_ms = now_ms() - t.t_submit; }
  c->tickets.erase(it);
  c->stats.requests_done++;
  if (--j->remaining == 0) free_job(c, j);
  return st;
}

spl_status spl_wait(spl_ctx *c, uint64_t ticket, uint64_t timeout_ns, spl_result *res) {
  // Polls with yields for the first 2 ms (a sleep overshoots by tens of microseconds, which a
  // request of a few hundred microseconds would see), then sleeps between polls.
  const double t0 = now_ms();
  const double limit = (double)timeout_ns * 1e-6;
  for (;;) {
    spl_status s = spl_poll(c, ticket, res);
    if (s != SPL_PENDING) return s;
    const double waited = now_ms() - t0;
    if (waited >= limit) return SPL_ERR_TIMEOUT;
    if (waited > 2.0) std::this_thread::sleep_for(std::chrono::microseconds(20));
    else std::this_thread::yield();
  }
}

spl_status spl_launch_geometry(const spl_plan_desc *plan, const uint64_t *n, uint32_t count, int32_t mem,
                               int32_t stored_fit, int32_t sm_count, spl_geometry *out) {
  if (!plan || !n || !out || count == 0 || sm_count < 1 || !plan_desc_ok(plan)) return SPL_ERR_INVALID_ARG;
  if (mem != SPL_MEM_DEVICE && mem != SPL_MEM_HOST) return SPL_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i)
    if (n[i] < 3 || n[i] > plan->max_n || n[i] > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  const PathChoice pc = choose_path(plan->precision, plan->tile_rows, plan->query_mode, stored_fit == 0,
                                    mem == SPL_MEM_DEVICE, n, count, sm_count);
  out->fit_kernel = pc.fit_kernel;
  out->separate_eval = pc.separate_eval ? 1 : 0;
  out->tile_rows = pc.tile_rows;
  out->direct = pc.direct ? 1 : 0;
  out->cta_rows = pc.cta_rows;
  out->ctas = pc.ctas;
  return SPL_OK;
}

spl_status spl_get_stats(spl_ctx *c, spl_stats *out) {
  if (!c || !out) return SPL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->stats.arena_high_water = c->dev.high_water();
  *out = c->stats;
  return SPL_OK;
}

spl_status spl_batch_create(spl_ctx *c, spl_plan *p, const spl_request *reqs, uint32_t count, spl_batch **out) {
  if (!c || !p || !reqs || !out || count == 0 || p->ctx != c) return SPL_ERR_INVALID_ARG;
  *out = nullptr;
  for (uint32_t i = 0; i < count; ++i) {
    spl_status s = check_request(p, &reqs[i]);
    if (s != SPL_OK) return s;
    if (reqs[i].mem != SPL_MEM_DEVICE) return SPL_ERR_INVALID_ARG;
    if ((reqs[i].ypp_in == nullptr) != (reqs[0].ypp_in == nullptr)) return SPL_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  if (cudaSetDevice(c->device) != cudaSuccess) return SPL_ERR_CUDA;
  std::unique_ptr<spl_batch> b(new (std::nothrow) spl_batch());
  if (!b) return SPL_ERR_CUDA;
  b->ctx = c;
  b->count = (int)count;
  LaunchPlan lp;
  uint64_t oi = 0, os = 0, orr = 0;
  spl_status s = prepare(c, p, reqs, count, lp, b->dev_blocks, b->pin_block, &oi, &os, &orr, false);
  if (s != SPL_OK) return s;
  char *pin_base = c->pinned + b->pin_block.off;
  b->h_status = reinterpret_cast<unsigned *>(pin_base + round_up(sizeof(Inst) * count, 64));
  // descriptors are uploaded once, outside the graph
  std::memcpy(pin_base, lp.insts.data(), sizeof(Inst) * count);
  cudaError_t e = cudaMemcpyAsync(c->arena + oi, pin_base, sizeof(Inst) * count, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(c->arena + os, 0, status_block_bytes(count), cap);
    int nl = 0;
    if (e1 == cudaSuccess) e1 = launch_path(c, lp, oi, orr, os, cap, &nl);
    b->launches_per_replay = nl;
    if (e1 == cudaSuccess)
      e1 = cudaMemcpyAsync(b->h_status, c->arena + os, 4ull * count, cudaMemcpyDeviceToHost, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
    e = (e1 != cudaSuccess) ? e1 : e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev_done);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    release_blocks(c, b->dev_blocks);
    c->pin.release(b->pin_block.off, b->pin_block.size);
    return SPL_ERR_CUDA;
  }
  *out = b.release();
  return SPL_OK;
}

spl_status spl_batch_launch(spl_batch *b) {
  if (!b) return SPL_ERR_INVALID_ARG;
  spl_ctx *c = b->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaError_t e = cudaGraphLaunch(b->exec, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_done, c->stream);
  if (e != cudaSuccess) return SPL_ERR_CUDA;
  b->launched = true;
  c->stats.graph_launches++;
  c->stats.kernel_launches += b->launches_per_replay;
  return SPL_OK;
}

spl_status spl_batch_wait(spl_batch *b, uint64_t timeout_ns, int32_t *statuses) {
  if (!b) return SPL_ERR_INVALID_ARG;
  if (!b->launched) return SPL_ERR_STATE;
  const double t0 = now_ms();
  const double limit = (double)timeout_ns * 1e-6;
  for (;;) {  // the polling of spl_wait
    cudaError_t q = cudaEventQuery(b->ev_done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return SPL_ERR_CUDA;
    const double waited = now_ms() - t0;
    if (waited >= limit) return SPL_ERR_TIMEOUT;
    if (waited > 2.0) std::this_thread::sleep_for(std::chrono::microseconds(20));
    else std::this_thread::yield();
  }
  spl_status worst = SPL_OK;
  for (int i = 0; i < b->count; ++i) {
    spl_status s = map_status_bits(b->h_status[i]);
    if (statuses) statuses[i] = s;
    if (s != SPL_OK) worst = s;
  }
  return worst;
}

void spl_batch_destroy(spl_batch *b) {
  if (!b) return;
  spl_ctx *c = b->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  release_blocks(c, b->dev_blocks);
  c->pin.release(b->pin_block.off, b->pin_block.size);
  delete b;
}

uint64_t spl_generate_scratch_bytes(uint64_t n) { return spl::generate_scratch_bytes((long long)n); }

spl_status spl_generate_curve(uint64_t seed, uint64_t instance, uint64_t n, double *x, double *y, void *scratch,
                              uint64_t scratch_bytes, void *stream) {
  if (n == 0) return SPL_OK;
  if (!x || !y || !scratch || n > (1ull << 26)) return SPL_ERR_INVALID_ARG;
  if (scratch_bytes < spl::generate_scratch_bytes((long long)n)) return SPL_ERR_INVALID_ARG;
  return cuda_fail(spl::launch_generate_curve(seed, instance, (long long)n, x, y, scratch,
                                              static_cast<cudaStream_t>(stream), nullptr));
}

}  // extern "C"
