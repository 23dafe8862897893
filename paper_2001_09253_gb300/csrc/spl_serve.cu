// Host side of the serving loop (include/spl.h, spl_serve_*): continuous batching of
// independent instances onto the persistent device loop of spl_mixed_scan.cu (serve_kernel).
//
// A request is admitted when a slot is free, its tiles fit in the device tile map and its
// footprint (inputs and outputs) fits in the HBM budget; otherwise it waits in a host FIFO and
// is admitted by a later submit/poll/wait as earlier requests complete.  Admission writes one
// entry into a ring in mapped host memory and advances the ring's tail; the device loop picks
// it up while other requests are being solved, so work that arrives while the GPU is busy
// overlaps with it.  Completion is read from per-slot words the device writes into mapped host
// memory.  The device loop leaves after an idle period; the next admission relaunches it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
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
using spl::ServeArgs;
using spl::ServeEntry;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

uint64_t up256(uint64_t v) { return (v + 255) / 256 * 256; }

// Per-request tile length of a server created with tile_rows = 0: about 32 tiles (warps) per
// request, between 128 rows (a small request's latency: one short tile) and the longest tile the
// workers' shared memory holds (a large one's throughput: each tile repeats 96 rows of start-up).
constexpr int kServeTileMin = 128;
int serve_tile_for(uint64_t n) {
  const uint64_t L = (n + 32 * 32 - 1) / (32 * 32) * 32;
  return (int)std::min<uint64_t>(std::max<uint64_t>(L, kServeTileMin), (uint64_t)spl::serve_tile_max());
}

struct Req {
  int state = 0;  // 0 waiting on the host, 1 resident on the device, 2 done
  Inst inst{};
  uint64_t ntiles = 0, bytes = 0, first_tile = 0;  // ntiles: tile tickets (twice the tiles when refined)
  uint64_t z_off = 0, z_bytes = 0;                 // refinement: binary32 y'' in the context's arena
  unsigned slot = 0, seq = 0;
  double t_submit = 0, t_done = 0;
  int status = SPL_PENDING;
};

}  // namespace

struct spl_server {
  spl_ctx *ctx = nullptr;
  spl_serve_desc d{};
  int device = 0, sms = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_exit = nullptr;
  bool launched = false;
  std::vector<std::pair<uint64_t, uint64_t>> blocks;  // arena (offset, size)
  char *hblock = nullptr;
  ServeArgs args{};
  volatile unsigned long long *h_tail = nullptr;
  volatile unsigned *h_stop = nullptr;
  volatile unsigned long long *h_consumed = nullptr;
  volatile unsigned *h_done = nullptr;
  ServeEntry *h_ring = nullptr;
  std::mutex mu;
  uint64_t tail = 0, next_tile = 0;
  unsigned next_seq = 1;
  uint64_t bytes_inflight = 0;
  std::vector<unsigned> free_slots;
  std::vector<unsigned> resident;  // slots holding a request (only these are polled)
  std::vector<uint64_t> slot_ticket;
  std::map<uint64_t, int> live_first;  // first tiles of resident requests
  std::deque<uint64_t> waiting;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_ticket = 1;
  uint64_t launches = 0;
};

namespace {

// The request is finished with the device: its refinement buffer goes back to the arena.
void release_z(spl_server *s, Req &r) {
  if (r.z_bytes) spl_ctx_arena_release(s->ctx, r.z_off, r.z_bytes);
  r.z_bytes = 0;
}

spl_status relaunch(spl_server *s) {
  cudaError_t e = cudaSuccess;
  // tickets claimed past the last published tile by the previous loop are void
  e = cudaMemcpyAsync(s->args.claimed, s->args.published, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                      s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->args.stop, 0, sizeof(unsigned), s->stream);
  *s->h_stop = 0u;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (e == cudaSuccess) e = spl::launch_serve(s->args, s->sms, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_exit, s->stream);
  if (e != cudaSuccess) return SPL_ERR_CUDA;
  s->launched = true;
  s->launches++;
  spl_ctx_count_launch(s->ctx, 1);
  return SPL_OK;
}

// The loop has exited: if a worker gave up waiting (error flag), every request still resident
// on the device and not completed completes with SPL_ERR_TIMEOUT, and the device counters are
// moved past the dropped tiles and ring entries so that the next launch starts clean.
spl_status after_exit(spl_server *s) {
  unsigned err = 0;
  if (cudaMemcpy(&err, s->args.err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return SPL_ERR_CUDA;
  if (!err) return SPL_OK;
  const double t = now_s();
  std::atomic_thread_fence(std::memory_order_acquire);
  for (size_t ri = 0; ri < s->resident.size();) {
    const unsigned slot = s->resident[ri];
    Req &r = s->reqs[s->slot_ticket[slot]];
    if (s->h_done[2 * slot + 1] == r.seq) {  // finished before the failure: harvested as usual
      ++ri;
      continue;
    }
    r.status = SPL_ERR_TIMEOUT;
    r.state = 2;
    r.t_done = t;
    release_z(s, r);
    s->slot_ticket[slot] = 0;
    s->free_slots.push_back(slot);
    s->bytes_inflight -= r.bytes;
    auto it = s->live_first.find(r.first_tile);
    if (it != s->live_first.end() && --it->second == 0) s->live_first.erase(it);
    s->resident[ri] = s->resident.back();
    s->resident.pop_back();
  }
  const unsigned long long ctr[3] = {s->next_tile, s->next_tile, s->tail};  // published, claimed, consumed
  cudaError_t e = cudaMemcpy(s->args.published, ctr, sizeof(ctr), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->args.err, 0, sizeof(unsigned));
  *s->h_consumed = s->tail;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  return e == cudaSuccess ? SPL_OK : SPL_ERR_CUDA;
}

bool loop_running(spl_server *s, spl_status *st) {
  *st = SPL_OK;
  if (!s->launched) return false;
  cudaError_t q = cudaEventQuery(s->ev_exit);
  if (q == cudaErrorNotReady) return true;
  s->launched = false;
  *st = after_exit(s);
  return false;
}

// Completions, then admissions, then make sure the device loop runs if anything is resident.
spl_status pump(spl_server *s) {
  spl_status xs = SPL_OK;
  const bool running = loop_running(s, &xs);
  if (xs != SPL_OK) return xs;
  const double t = now_s();
  for (size_t ri = 0; ri < s->resident.size();) {
    const unsigned slot = s->resident[ri];
    const uint64_t tk = s->slot_ticket[slot];
    Req &r = s->reqs[tk];
    if (s->h_done[2 * slot + 1] != r.seq) {
      ++ri;
      continue;
    }
    s->resident[ri] = s->resident.back();
    s->resident.pop_back();
    std::atomic_thread_fence(std::memory_order_acquire);
    const unsigned bits = s->h_done[2 * slot];
    r.status = (bits & spl::kStBadTile)         ? SPL_ERR_INVALID_ARG
               : (bits & spl::kStNonFinite)     ? SPL_ERR_NONFINITE
               : (bits & spl::kStNotIncreasing) ? SPL_ERR_NOT_INCREASING
                                                : SPL_OK;
    r.state = 2;
    r.t_done = t;
    release_z(s, r);
    s->slot_ticket[slot] = 0;
    s->free_slots.push_back(slot);
    s->bytes_inflight -= r.bytes;
    auto it = s->live_first.find(r.first_tile);
    if (it != s->live_first.end() && --it->second == 0) s->live_first.erase(it);
  }
  bool admitted = false;
  while (!s->waiting.empty()) {
    const uint64_t tk = s->waiting.front();
    Req &r = s->reqs[tk];
    const uint64_t oldest = s->live_first.empty() ? s->next_tile : s->live_first.begin()->first;
    const bool fits = !s->free_slots.empty() && s->bytes_inflight + r.bytes <= s->d.budget_bytes &&
                      s->next_tile + r.ntiles - oldest <= s->args.tile_cap &&
                      s->tail - *s->h_consumed < s->args.rcap;
    if (!fits) break;
    if (r.inst.pad & spl::kServeRefined) {  // the first pass's binary32 y'', from the arena
      uint64_t off = 0;
      const uint64_t zb = (4ull * (uint64_t)r.inst.n + 255) / 256 * 256;
      if (!spl_ctx_arena_alloc(s->ctx, zb, &off)) break;  // waits for a completion to free memory
      r.z_off = off;
      r.z_bytes = zb;
      r.inst.z = reinterpret_cast<float *>(spl_ctx_arena_base(s->ctx) + off);
    }
    s->waiting.pop_front();
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    r.seq = s->next_seq++;
    if (s->next_seq == 0) s->next_seq = 1;
    r.first_tile = s->next_tile;
    s->next_tile += r.ntiles;
    s->bytes_inflight += r.bytes;
    s->live_first[r.first_tile]++;
    s->slot_ticket[r.slot] = tk;
    s->resident.push_back(r.slot);
    r.state = 1;
    ServeEntry &e = s->h_ring[s->tail % s->args.rcap];
    e.inst = r.inst;
    e.first_tile = r.first_tile;
    e.slot = r.slot;
    e.seq = r.seq;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *s->h_tail = ++s->tail;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    admitted = true;
  }
  if ((admitted || !s->resident.empty()) && !running) return relaunch(s);
  return SPL_OK;
}

void release_server(spl_server *s) {
  for (auto &b : s->blocks) spl_ctx_arena_release(s->ctx, b.first, b.second);
  if (s->hblock) cudaFreeHost(s->hblock);
  if (s->ev_exit) cudaEventDestroy(s->ev_exit);
  if (s->stream) cudaStreamDestroy(s->stream);
}

}  // namespace

extern "C" {

spl_status spl_serve_create(spl_ctx *c, const spl_serve_desc *d, spl_server **out) {
  if (!c || !d || !out) return SPL_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->max_inflight < 1 || d->max_inflight > 65536) return SPL_ERR_INVALID_ARG;
  if (d->tile_rows != 0 && d->tile_rows < 16) return SPL_ERR_INVALID_ARG;
  if (d->refine_steps > 1) return SPL_ERR_INVALID_ARG;
  std::unique_ptr<spl_server> s(new (std::nothrow) spl_server());
  if (!s) return SPL_ERR_CUDA;
  s->ctx = c;
  s->d = *d;
  // tile_rows 0: per request (serve_tile_for); otherwise one length, a whole number of chunks
  if (s->d.tile_rows)
    s->d.tile_rows = (uint32_t)spl::serve_tile_rows((int)std::min<uint32_t>(s->d.tile_rows, 1u << 20));
  if (!s->d.idle_timeout_ms) s->d.idle_timeout_ms = 200;
  s->device = spl_ctx_device(c);
  s->sms = spl_ctx_sms(c);
  if (cudaSetDevice(s->device) != cudaSuccess) return SPL_ERR_CUDA;
  const unsigned S = s->d.max_inflight;
  const uint64_t tile_cap = s->d.max_tiles ? s->d.max_tiles : std::max<uint64_t>(1ull << 20, 64ull * S);
  const uint64_t rcap = std::max<uint64_t>(256, 2ull * S);
  // device state, carved from the context's arena
  const uint64_t sz_ctr = 256, sz_inst = up256(sizeof(Inst) * S), sz_first = up256(8ull * S),
                 sz_u32 = up256(4ull * S), sz_map = up256(4ull * tile_cap);
  const uint64_t total = sz_ctr + sz_inst + sz_first + 3 * sz_u32 + sz_map;
  uint64_t off = 0;
  if (!spl_ctx_arena_alloc(c, total, &off)) return SPL_ERR_BUDGET;
  s->blocks.push_back({off, total});
  char *base = spl_ctx_arena_base(c) + off;
  ServeArgs &a = s->args;
  a.published = reinterpret_cast<unsigned long long *>(base);
  a.claimed = a.published + 1;
  a.consumed = a.published + 2;
  a.stop = reinterpret_cast<unsigned *>(base + 32);
  a.err = a.stop + 1;
  char *p = base + sz_ctr;
  a.slot_inst = reinterpret_cast<Inst *>(p);
  p += sz_inst;
  a.slot_first = reinterpret_cast<unsigned long long *>(p);
  p += sz_first;
  a.slot_done = reinterpret_cast<unsigned *>(p);
  p += sz_u32;
  a.slot_status = reinterpret_cast<unsigned *>(p);
  p += sz_u32;
  a.slot_seq = reinterpret_cast<unsigned *>(p);
  p += sz_u32;
  a.tile_slot = reinterpret_cast<unsigned *>(p);
  a.tile_cap = tile_cap;
  a.rcap = rcap;
  a.idle_ns = (unsigned long long)s->d.idle_timeout_ms * 1000000ull;
  // a single launch never runs longer than the deadline; the host relaunches
  a.deadline_ns = (unsigned long long)(s->d.deadline_ms ? s->d.deadline_ms : 30000u) * 1000000ull;
  a.fault_flags = s->d.fault_flags;
  // mapped host block: tail, stop, consumed, alive, done words, ring
  const uint64_t hbytes = 256 + up256(8ull * S) + sizeof(ServeEntry) * rcap;
  if (cudaHostAlloc(&s->hblock, hbytes, cudaHostAllocMapped) != cudaSuccess) {
    release_server(s.get());
    return SPL_ERR_CUDA;
  }
  std::memset(s->hblock, 0, hbytes);
  char *dh = nullptr;
  if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&dh), s->hblock, 0) != cudaSuccess) {
    release_server(s.get());
    return SPL_ERR_CUDA;
  }
  s->h_tail = reinterpret_cast<volatile unsigned long long *>(s->hblock);
  s->h_stop = reinterpret_cast<volatile unsigned *>(s->hblock + 8);
  s->h_consumed = reinterpret_cast<volatile unsigned long long *>(s->hblock + 16);
  s->h_done = reinterpret_cast<volatile unsigned *>(s->hblock + 256);
  s->h_ring = reinterpret_cast<ServeEntry *>(s->hblock + 256 + up256(8ull * S));
  a.h_tail = reinterpret_cast<const volatile unsigned long long *>(dh);
  a.h_stop = reinterpret_cast<const volatile unsigned *>(dh + 8);
  a.h_consumed = reinterpret_cast<volatile unsigned long long *>(dh + 16);
  a.h_alive = reinterpret_cast<volatile unsigned *>(dh + 24);
  a.h_done = reinterpret_cast<volatile unsigned *>(dh + 256);
  a.h_ring = reinterpret_cast<const ServeEntry *>(dh + 256 + up256(8ull * S));
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_exit, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, sz_ctr, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.slot_seq, 0, sz_u32, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    release_server(s.get());
    return SPL_ERR_CUDA;
  }
  s->slot_ticket.assign(S, 0);
  for (unsigned i = 0; i < S; ++i) s->free_slots.push_back(S - 1 - i);
  *out = s.release();
  return SPL_OK;
}

spl_status spl_serve_submit(spl_server *s, const spl_request *r, uint64_t *ticket) {
  if (!s || !r || !ticket) return SPL_ERR_INVALID_ARG;
  if (r->n < 3 || !r->x || !r->y || (r->m > 0 && !r->yq_out) || r->mem != SPL_MEM_DEVICE) return SPL_ERR_INVALID_ARG;
  if (r->n > (1ull << 40) || r->m > (1ull << 40)) return SPL_ERR_INVALID_ARG;
  if (r->xq || r->ypp_in) return SPL_ERR_INVALID_ARG;  // served requests: uniform queries, fit included
  if (std::isnan(r->yp1) || std::isnan(r->ypn) || (std::isinf(r->yp1) && r->yp1 < 0) ||
      (std::isinf(r->ypn) && r->ypn < 0))
    return SPL_ERR_INVALID_ARG;
  Req q;
  Inst &I = q.inst;
  I.x = r->x; I.y = r->y; I.ypp = r->ypp_out; I.yq = r->yq_out; I.jq = r->jq_out;
  I.n = (long long)r->n; I.m = (long long)r->m;
  I.yp1 = r->yp1; I.ypn = r->ypn;
  I.tile_rows = s->d.tile_rows ? (int)s->d.tile_rows : serve_tile_for(r->n);
  I.ntiles = ((long long)r->n + I.tile_rows - 1) / I.tile_rows;
  I.tile_begin = 0;
  q.ntiles = (uint64_t)I.ntiles;
  q.bytes = 16 * r->n + (r->ypp_out ? 8 * r->n : 0) + 8 * r->m + (r->jq_out ? 4 * r->m : 0);
  if (s->d.refine_steps) {  // two passes over the tiles, binary32 y'' of the first in between
    I.pad |= spl::kServeRefined;
    q.ntiles *= 2;
    q.bytes += 4 * r->n;
  }
  if (q.bytes > s->d.budget_bytes || q.ntiles > s->args.tile_cap) return SPL_ERR_BUDGET;
  std::lock_guard<std::mutex> lk(s->mu);
  if (cudaSetDevice(s->device) != cudaSuccess) return SPL_ERR_CUDA;
  q.t_submit = now_s();
  const uint64_t tk = s->next_ticket++;
  s->reqs[tk] = q;
  s->waiting.push_back(tk);
  *ticket = tk;
  return pump(s);
}

spl_status spl_serve_poll(spl_server *s, uint64_t ticket, spl_result *res) {
  if (!s) return SPL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SPL_ERR_UNKNOWN_TICKET;
  if (it->second.state != 2) {
    if (cudaSetDevice(s->device) != cudaSuccess) return SPL_ERR_CUDA;
    spl_status ps = pump(s);
    if (ps != SPL_OK) return ps;
  }
  Req &r = it->second;
  if (r.state != 2) {
    if (res) { res->status = SPL_PENDING; res->device_ms = 0; res->latency_ms = 1e3 * (now_s() - r.t_submit); }
    return SPL_PENDING;
  }
  const spl_status st = (spl_status)r.status;
  if (res) { res->status = st; res->device_ms = 0; res->latency_ms = 1e3 * (r.t_done - r.t_submit); }
  s->reqs.erase(it);
  return st;
}

spl_status spl_serve_wait(spl_server *s, uint64_t ticket, uint64_t timeout_ns, spl_result *res) {
  const double t0 = now_s(), limit = (double)timeout_ns * 1e-9;
  int spins = 0;
  for (;;) {
    spl_status st = spl_serve_poll(s, ticket, res);
    if (st != SPL_PENDING) return st;
    if (now_s() - t0 >= limit) return SPL_ERR_TIMEOUT;
    if (++spins > 256) std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
}

spl_status spl_serve_replay(spl_server *s, const spl_request *pool, uint32_t pool_count, const uint32_t *pick,
                            const double *arrival_s, uint64_t count, double *latency_ms, double *makespan_s) {
  if (!s || !pool || !pick || !arrival_s || !latency_ms || pool_count == 0) return SPL_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < count; ++i)
    if (pick[i] >= pool_count || (i && arrival_s[i] < arrival_s[i - 1])) return SPL_ERR_INVALID_ARG;
  std::vector<uint64_t> tk(count, 0);
  std::vector<char> done(count, 0);
  const double t0 = now_s();
  const double last = count ? arrival_s[count - 1] : 0.0;
  uint64_t next = 0, collected = 0, scan = 0;
  while (collected < count) {
    const double t = now_s() - t0;
    while (next < count && arrival_s[next] <= t) {
      spl_status st = spl_serve_submit(s, &pool[pick[next]], &tk[next]);
      if (st != SPL_OK) return st;
      ++next;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      spl_status ps = pump(s);
      if (ps != SPL_OK) return ps;
      for (uint64_t i = scan; i < next; ++i) {
        if (done[i]) continue;
        auto it = s->reqs.find(tk[i]);
        if (it == s->reqs.end() || it->second.state != 2) continue;
        if (it->second.status != SPL_OK) return (spl_status)it->second.status;
        latency_ms[i] = 1e3 * (it->second.t_done - (t0 + arrival_s[i]));
        s->reqs.erase(it);
        done[i] = 1;
        ++collected;
      }
      while (scan < next && done[scan]) ++scan;
    }
    if (now_s() - t0 > last + 60.0) return SPL_ERR_TIMEOUT;
  }
  if (makespan_s) *makespan_s = now_s() - t0;
  return SPL_OK;
}

spl_status spl_serve_stats(spl_server *s, uint64_t *loop_launches, uint64_t *waiting, uint64_t *resident) {
  if (!s) return SPL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (loop_launches) *loop_launches = s->launches;
  if (waiting) *waiting = s->waiting.size();
  if (resident) {
    uint64_t k = 0;
    for (auto t : s->slot_ticket) k += t != 0;
    *resident = k;
  }
  return SPL_OK;
}

void spl_serve_destroy(spl_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    cudaSetDevice(s->device);
    *s->h_stop = 1u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
  // the loop sees the stop word within microseconds; its own deadline bounds it regardless
  const double t0 = now_s();
  while (s->launched && cudaEventQuery(s->ev_exit) == cudaErrorNotReady && now_s() - t0 < 40.0)
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  cudaStreamSynchronize(s->stream);
  for (auto &kv : s->reqs) release_z(s, kv.second);
  release_server(s);
  delete s;
}

}  // extern "C"
