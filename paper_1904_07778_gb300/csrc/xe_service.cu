// Streaming service (declared in include/xengine.h): continuous batching of
// integration requests over the batched cross-multiply.
//
// Host side, in this file: an arena allocator that carves every admitted
// request's device state out of one allocation made at creation (first fit,
// neighbours coalesced on release), FIFO admission by that budget, slots
// that index the per-launch array descriptors, double-buffered ingest on a
// copy stream ordered by events, the composition of each tick (the oldest
// waiting block of every active request; one persistent launch per sample
// width, tasks spread over the SMs longest first), and completion times
// recorded by a host callback on the compute stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "xe_internal.h"
#include "xengine.h"

using namespace xe;

namespace {

constexpr int kMaxSlots = 64;        // concurrently active requests
constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator of offsets in [0, cap): free ranges by offset,
// coalesced with their neighbours on release.
struct Arena {
  size_t cap = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;
  void init(size_t c) {
    cap = c;
    free_.clear();
    if (c) free_[0] = c;
    used = peak = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used += bytes;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes);
    used -= bytes;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + bytes == nx->first) {  // merge with the next range
      bytes += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {  // merge into the previous range
        pv->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
};

struct Req {
  int64_t id = 0;
  corr_req r{};
  int state = CORR_REQ_QUEUED;
  int R = 0;                     // byte rows per channel
  size_t block_bytes = 0, acc_bytes = 0, turn_bytes = 0;
  bool has_turn = false;
  bool tci = false;  // blocks read in payload order (no corner turn)
  long long stride = 0;
  // arena offsets of the pieces (valid while admitted)
  size_t off_acc = 0, off_in[2] = {0, 0}, off_turn = 0;
  int slot = -1;
  int64_t pushed = 0, ticked = 0;
  std::vector<HerkTask> tasks;   // inst filled per tick
  int rpc = 0;
  CUtensorMap tmap[2];
  cudaEvent_t ev_copy[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  double t_submit = 0.0;
  std::atomic<double> t_done{0.0};
  std::atomic<int> done{0};
  bool latency_recorded = false;
};

void CUDART_CB mark_done(void* p) {
  Req* q = static_cast<Req*>(p);
  q->t_done.store(now_ms());
  q->done.store(1);
}

}  // namespace

struct corr_svc {
  bool dry = false;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  bool own_stream = false;
  uint8_t* base = nullptr;
  Arena arena;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::deque<int64_t> queue;
  int64_t next_id = 1;
  std::vector<int> free_slots;
  // per-tick launch descriptors, two sets (ticks alternate)
  HerkInst* d_insts[2] = {nullptr, nullptr};
  CUtensorMap* d_tmaps[2] = {nullptr, nullptr};
  HerkTask* d_tasks[2] = {nullptr, nullptr};
  int* d_first[2] = {nullptr, nullptr};
  size_t task_cap[2] = {0, 0}, first_cap[2] = {0, 0};
  HerkInst* h_insts[2] = {nullptr, nullptr};   // pinned staging
  CUtensorMap* h_tmaps[2] = {nullptr, nullptr};
  HerkTask* h_tasks[2] = {nullptr, nullptr};
  int* h_first[2] = {nullptr, nullptr};
  cudaEvent_t ev_tick[2] = {nullptr, nullptr};
  bool tick_used[2] = {false, false};
  int parity = 0;
  int* d_status = nullptr;
  int* h_status = nullptr;
  int2* scratch = nullptr;  // 8-bit: per-CTA partial sums (the tick's launches run in order)
  int scratch_ctas = 0;
  corr_svc_stats st{};
  std::vector<double> lat;
};

namespace {

int sm_count() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm > 0 ? nsm : 1;
}

bool valid_req(const corr_req& r) {
  const int chunk = r.bits == 8 ? kMaxChunk8 : kMaxChunk4;
  return r.n_inputs >= 1 && r.n_inputs <= 1024 && r.n_chans >= 1 && (r.bits == 4 || r.bits == 8) &&
         r.layout >= CORR_L_TCI && r.layout <= CORR_L_CIT && !(r.flags & ~CORR_F_LO_IS_REAL) &&
         !(r.bits == 8 && (r.flags & CORR_F_LO_IS_REAL)) && r.block_spectra >= 1 &&
         r.block_spectra <= chunk && r.n_blocks >= 1 &&
         (needs_turn(r.layout, r.bits) || r.block_spectra % 16 == 0);
}

size_t req_bytes(const Req& q) {
  return round_up(q.acc_bytes) + 2 * round_up(q.block_bytes) + (q.has_turn ? round_up(q.turn_bytes) : 0);
}

void release(corr_svc* s, Req& q) {
  s->arena.release(q.off_acc, q.acc_bytes);
  s->arena.release(q.off_in[0], q.block_bytes);
  s->arena.release(q.off_in[1], q.block_bytes);
  if (q.has_turn) s->arena.release(q.off_turn, q.turn_bytes);
  if (q.slot >= 0) s->free_slots.push_back(q.slot);
  q.slot = -1;
}

// Admit queued requests in arrival order while their state fits.
void admit(corr_svc* s) {
  while (!s->queue.empty() && !s->free_slots.empty()) {
    Req& q = *s->reqs[s->queue.front()];
    size_t a = 0, i0 = 0, i1 = 0, t = 0;
    if (!s->arena.alloc(q.acc_bytes, &a)) return;
    if (!s->arena.alloc(q.block_bytes, &i0)) { s->arena.release(a, q.acc_bytes); return; }
    if (!s->arena.alloc(q.block_bytes, &i1)) {
      s->arena.release(a, q.acc_bytes);
      s->arena.release(i0, q.block_bytes);
      return;
    }
    if (q.has_turn && !s->arena.alloc(q.turn_bytes, &t)) {
      s->arena.release(a, q.acc_bytes);
      s->arena.release(i0, q.block_bytes);
      s->arena.release(i1, q.block_bytes);
      return;
    }
    q.off_acc = a;
    q.off_in[0] = i0;
    q.off_in[1] = i1;
    q.off_turn = t;
    q.slot = s->free_slots.back();
    s->free_slots.pop_back();
    q.tasks = plan_tasks(q.r.n_inputs, q.r.n_chans, &q.rpc);
    if (!s->dry) {
      for (int b = 0; b < 2; ++b) {
        const uint8_t* x = q.has_turn ? s->base + q.off_turn : s->base + q.off_in[b];
        make_herk_tmap(&q.tmap[b], x, q.tci, q.r.bits, q.R, q.r.n_chans, q.r.block_spectra,
                       q.stride, q.rpc);
        if (!q.ev_copy[b]) cudaEventCreateWithFlags(&q.ev_copy[b], cudaEventDisableTiming);
        if (!q.ev_used[b]) cudaEventCreateWithFlags(&q.ev_used[b], cudaEventDisableTiming);
      }
    }
    q.state = CORR_REQ_ACTIVE;
    ++s->st.admitted;
    s->queue.pop_front();
  }
}

int refresh(Req& q) {
  if (q.state == CORR_REQ_ACTIVE && q.ticked == q.r.n_blocks && q.done.load()) q.state = CORR_REQ_DONE;
  return q.state;
}

void record_latency(corr_svc* s, Req& q) {
  if (q.latency_recorded || q.state < CORR_REQ_DONE) return;
  s->lat.push_back(q.t_done.load() - q.t_submit);
  q.latency_recorded = true;
  ++s->st.completed;
}

// Grow a pair of pinned/device arrays to hold n elements.
template <typename T>
bool ensure(T*& d, T*& h, size_t& cap, size_t n) {
  if (n <= cap) return true;
  cudaFree(d);
  cudaFreeHost(h);
  d = nullptr;
  h = nullptr;
  cap = 0;
  const size_t c = std::max<size_t>(n, 1024);
  if (cudaMalloc(&d, c * sizeof(T)) != cudaSuccess) return false;
  if (cudaMallocHost(&h, c * sizeof(T)) != cudaSuccess) return false;
  cap = c;
  return true;
}

}  // namespace

extern "C" {

int corr_svc_create(size_t hbm_budget, unsigned flags, void* stream, corr_svc** out) {
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (hbm_budget == 0 || (flags & ~CORR_SVC_DRY_RUN)) return CORR_EINVAL;
  corr_svc* s = new (std::nothrow) corr_svc;
  if (!s) return CORR_ENOMEM;
  s->dry = (flags & CORR_SVC_DRY_RUN) != 0;
  s->arena.init(hbm_budget);
  s->st.budget = hbm_budget;
  for (int i = kMaxSlots - 1; i >= 0; --i) s->free_slots.push_back(i);
  if (!s->dry) {
    int st = CORR_OK;
    do {
      if (stream && (cudaStream_t)stream != cudaStreamLegacy &&
          (cudaStream_t)stream != cudaStreamPerThread) {
        s->stream = (cudaStream_t)stream;
      } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
        s->own_stream = true;
      }
      if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
      if (cudaMalloc(&s->base, hbm_budget) != cudaSuccess) { st = CORR_ENOMEM; break; }
      if (cudaMalloc(&s->d_status, sizeof(int)) != cudaSuccess ||
          cudaMallocHost(&s->h_status, sizeof(int)) != cudaSuccess) { st = CORR_ENOMEM; break; }
      if (cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) { st = CORR_ECUDA; break; }
      if (herk_scratch_alloc(&s->scratch, &s->scratch_ctas) != cudaSuccess) { st = CORR_ENOMEM; break; }
      for (int p = 0; p < 2 && st == CORR_OK; ++p) {
        if (cudaMalloc(&s->d_insts[p], sizeof(HerkInst) * 2 * kMaxSlots) != cudaSuccess ||
            cudaMalloc(&s->d_tmaps[p], sizeof(CUtensorMap) * 2 * kMaxSlots) != cudaSuccess ||
            cudaMallocHost(&s->h_insts[p], sizeof(HerkInst) * 2 * kMaxSlots) != cudaSuccess ||
            cudaMallocHost(&s->h_tmaps[p], sizeof(CUtensorMap) * 2 * kMaxSlots) != cudaSuccess)
          st = CORR_ENOMEM;
        else if (cudaEventCreateWithFlags(&s->ev_tick[p], cudaEventDisableTiming) != cudaSuccess)
          st = CORR_ECUDA;
      }
    } while (0);
    if (st != CORR_OK) {
      cudaGetLastError();
      corr_svc_destroy(s);
      return st;
    }
  }
  *out = s;
  return CORR_OK;
}

int corr_svc_submit(corr_svc* s, const corr_req* r, int64_t* id) {
  if (!s || !r || !id || !valid_req(*r)) return CORR_EINVAL;
  std::unique_ptr<Req> q(new (std::nothrow) Req);
  if (!q) return CORR_ENOMEM;
  q->r = *r;
  q->R = r->n_inputs * (r->bits / 4);
  q->block_bytes = (size_t)q->R * r->n_chans * r->block_spectra;
  q->acc_bytes = (size_t)r->n_inputs * (r->n_inputs + 1) / 2 * r->n_chans * 16;
  q->tci = tci_direct(r->layout, r->bits, r->n_inputs);
  q->has_turn = needs_turn(r->layout, r->bits) && !q->tci;
  q->stride = q->has_turn ? ((long long)r->block_spectra + 31) / 32 * 32 : r->block_spectra;
  q->turn_bytes = q->has_turn ? (size_t)q->stride * q->R * r->n_chans : 0;
  if (req_bytes(*q) > s->arena.cap) return CORR_EBUSY;
  q->id = s->next_id++;
  q->t_submit = now_ms();
  *id = q->id;
  s->queue.push_back(q->id);
  s->reqs[q->id] = std::move(q);
  ++s->st.submitted;
  admit(s);
  return CORR_OK;
}

int corr_svc_state(corr_svc* s, int64_t id, int* state) {
  if (!s || !state) return CORR_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return CORR_EINVAL;
  *state = refresh(*it->second);
  record_latency(s, *it->second);
  return CORR_OK;
}

int corr_svc_push(corr_svc* s, int64_t id, const void* block, size_t nbytes) {
  TraceRange trace_("corr_svc_push");
  if (!s || !block) return CORR_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return CORR_EINVAL;
  Req& q = *it->second;
  if (nbytes != q.block_bytes) return CORR_EINVAL;
  if (q.state != CORR_REQ_ACTIVE || q.pushed >= q.r.n_blocks) return CORR_ESTATE;
  if (q.pushed - q.ticked >= 2) return CORR_EBUSY;
  const int b = (int)(q.pushed & 1);
  if (!s->dry) {
    // the buffer is free once the tick that last read it has finished
    if (cudaStreamWaitEvent(s->copy_stream, q.ev_used[b], 0) != cudaSuccess ||
        cudaMemcpyAsync(s->base + q.off_in[b], block, nbytes, cudaMemcpyDefault, s->copy_stream) !=
            cudaSuccess ||
        cudaEventRecord(q.ev_copy[b], s->copy_stream) != cudaSuccess)
      return CORR_ECUDA;
  }
  ++q.pushed;
  return CORR_OK;
}

int corr_svc_tick(corr_svc* s, int* n_requests) {
  TraceRange trace_("corr_svc_tick");
  if (!s) return CORR_EINVAL;
  std::vector<Req*> parts;
  for (auto& kv : s->reqs) {
    Req& q = *kv.second;
    if (q.state == CORR_REQ_ACTIVE && q.pushed > q.ticked) parts.push_back(&q);
  }
  if (n_requests) *n_requests = (int)parts.size();
  if (parts.empty()) return CORR_OK;
  const int p = s->parity;
  s->parity ^= 1;
  int launches = 0;
  if (!s->dry) {
    // the descriptor set of this parity is reused: its last tick must be done
    if (s->tick_used[p] && cudaEventSynchronize(s->ev_tick[p]) != cudaSuccess) return CORR_ECUDA;
    for (Req* q : parts) {
      const int b = (int)(q->ticked & 1);
      const uint8_t* in = s->base + q->off_in[b];
      if (cudaStreamWaitEvent(s->stream, q->ev_copy[b], 0) != cudaSuccess) return CORR_ECUDA;
      if (q->has_turn) {
        if (turn_rows(in, s->base + q->off_turn, q->r.layout, q->r.bits, q->r.n_inputs,
                      q->r.n_chans, q->r.block_spectra, q->stride, s->stream) != cudaSuccess)
          return CORR_ECUDA;
        ++launches;
      }
      const int inst = q->slot * 2 + b;
      HerkInst& I = s->h_insts[p][inst];
      memset(&I, 0, sizeof(I));
      I.x = q->has_turn ? s->base + q->off_turn : in;
      I.acc = reinterpret_cast<int64_t*>(s->base + q->off_acc);
      I.chan_stride = (long long)q->R * q->stride;
      I.row_stride = q->stride;
      I.n_inputs = q->r.n_inputs;
      I.n_chans = q->r.n_chans;
      I.t0 = 0;
      I.tn = q->r.block_spectra;
      I.rows_per_chan = q->rpc;
      I.accumulate = q->ticked > 0 ? 1 : 0;
      I.vec_ok = 1;
      s->h_tmaps[p][inst] = q->tmap[b];
    }
    // one launch per (sample width, nibble order, payload order read directly);
    // tasks longest first
    struct Cls { int bits, lo; bool tci; std::vector<Req*> qs; };
    std::vector<Cls> cls;
    for (Req* q : parts) {
      const int lo = (q->r.flags & CORR_F_LO_IS_REAL) ? 1 : 0;
      auto c = std::find_if(cls.begin(), cls.end(), [&](const Cls& x) {
        return x.bits == q->r.bits && x.lo == lo && x.tci == q->tci;
      });
      if (c == cls.end()) cls.push_back({q->r.bits, lo, q->tci, {q}});
      else c->qs.push_back(q);
    }
    size_t ntask = 0;
    for (auto& c : cls)
      for (Req* q : c.qs) ntask += q->tasks.size();
    const int nsm = sm_count();
    if (!ensure(s->d_tasks[p], s->h_tasks[p], s->task_cap[p], ntask) ||
        !ensure(s->d_first[p], s->h_first[p], s->first_cap[p], cls.size() * (nsm + 1)))
      return CORR_ENOMEM;
    struct Launch { size_t t0, f0; int nt, nc, bits, lo; bool tci; };
    std::vector<Launch> ls;
    size_t tpos = 0, fpos = 0;
    for (auto& c : cls) {
      std::vector<HerkTask> all;
      std::vector<double> cost;
      for (Req* q : c.qs) {
        const int inst = q->slot * 2 + (int)(q->ticked & 1);
        for (HerkTask t : q->tasks) {
          t.inst = inst;
          const int nb = t.cb[1] >= 0 ? 2 : 1;
          const bool a_in = t.rb == t.cb[0] || (nb == 2 && t.rb == t.cb[1]);
          const int st = herk_ring_stage(q->r.bits);
          cost.push_back((double)((q->r.block_spectra + st - 1) / st) * (a_in ? nb : nb + 1));
          all.push_back(t);
        }
      }
      const int nt = (int)all.size(), nc = std::min(nt, nsm);
      std::vector<int> order(nt);
      corr_plan_schedule(cost.data(), nt, nc, order.data(), s->h_first[p] + fpos);
      for (int j = 0; j < nt; ++j) s->h_tasks[p][tpos + j] = all[order[j]];
      ls.push_back({tpos, fpos, nt, nc, c.bits, c.lo, c.tci});
      tpos += nt;
      fpos += nc + 1;
    }
    if (cudaMemcpyAsync(s->d_insts[p], s->h_insts[p], sizeof(HerkInst) * 2 * kMaxSlots,
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->d_tmaps[p], s->h_tmaps[p], sizeof(CUtensorMap) * 2 * kMaxSlots,
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->d_tasks[p], s->h_tasks[p], sizeof(HerkTask) * tpos,
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->d_first[p], s->h_first[p], sizeof(int) * fpos, cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess)
      return CORR_ECUDA;
    for (const Launch& l : ls) {
      HerkArgs a;
      memset(&a, 0, sizeof(a));
      a.insts = s->d_insts[p];
      a.tmaps = s->d_tmaps[p];
      a.tasks = s->d_tasks[p] + l.t0;
      a.cta_first = s->d_first[p] + l.f0;
      a.status = s->d_status;
      a.lo_is_real = l.lo;
      a.bits = l.bits;
      a.n_tasks = l.nt;
      a.grid = l.nc;
      a.scratch = s->scratch;
      a.scratch_ctas = s->scratch_ctas;
      if (herk4_launch(a, nullptr, l.nt, s->stream, l.tci) != cudaSuccess) return CORR_ECUDA;
      ++launches;
    }
    if (cudaEventRecord(s->ev_tick[p], s->stream) != cudaSuccess) return CORR_ECUDA;
    s->tick_used[p] = true;
  }
  for (Req* q : parts) {
    const int b = (int)(q->ticked & 1);
    if (!s->dry && cudaEventRecord(q->ev_used[b], s->stream) != cudaSuccess) return CORR_ECUDA;
    ++q->ticked;
    ++s->st.blocks;
    s->st.chan_spectra += (double)q->r.n_chans * q->r.block_spectra;
    s->st.ops += 8.0 * q->r.n_inputs * (q->r.n_inputs + 1) / 2 * q->r.n_chans * q->r.block_spectra;
    if (q->ticked == q->r.n_blocks) {
      if (s->dry) {
        mark_done(q);
      } else if (cudaLaunchHostFunc(s->stream, mark_done, q) != cudaSuccess) {
        return CORR_ECUDA;
      }
    }
  }
  ++s->st.ticks;
  s->st.launches += launches;
  return CORR_OK;
}

int corr_svc_fetch(corr_svc* s, int64_t id, int64_t* vis) {
  TraceRange trace_("corr_svc_fetch");
  if (!s) return CORR_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return CORR_EINVAL;
  Req& q = *it->second;
  if (refresh(q) != CORR_REQ_DONE) return CORR_ESTATE;
  record_latency(s, q);
  if (vis && !s->dry) {
    if (cudaMemcpyAsync(vis, s->base + q.off_acc, q.acc_bytes, cudaMemcpyDefault, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      return CORR_ECUDA;
  }
  // every copy into the request's buffers was consumed by one of its ticks,
  // and the last tick has finished (the completion callback ran): the
  // memory and the events are free
  release(s, q);
  q.state = CORR_REQ_FETCHED;
  ++s->st.fetched;
  for (int b = 0; b < 2; ++b) {
    if (q.ev_copy[b]) cudaEventDestroy(q.ev_copy[b]);
    if (q.ev_used[b]) cudaEventDestroy(q.ev_used[b]);
    q.ev_copy[b] = q.ev_used[b] = nullptr;
  }
  admit(s);
  return CORR_OK;
}

int corr_svc_wait(corr_svc* s) {
  if (!s) return CORR_EINVAL;
  if (s->dry) return CORR_OK;
  if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return CORR_ECUDA;
  if (cudaMemcpy(s->h_status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CORR_ECUDA;
  const int st = *s->h_status;
  if (st == 0) return CORR_OK;
  if (cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) return CORR_ECUDA;
  if (st & kStTimeout) return CORR_ETIMEDOUT;
  if (st & kStRange) return CORR_ERANGE;
  return CORR_ECUDA;
}

int corr_svc_stats_get(corr_svc* s, corr_svc_stats* out) {
  if (!s || !out) return CORR_EINVAL;
  for (auto& kv : s->reqs) {
    refresh(*kv.second);
    record_latency(s, *kv.second);
  }
  corr_svc_stats r = s->st;
  r.in_use = s->arena.used;
  r.peak_in_use = s->arena.peak;
  r.active = 0;
  for (auto& kv : s->reqs) r.active += kv.second->state == CORR_REQ_ACTIVE ? 1 : 0;
  r.queued = (int)s->queue.size();
  std::vector<double> l = s->lat;
  std::sort(l.begin(), l.end());
  auto pct = [&](double f) {
    if (l.empty()) return 0.0;
    const size_t i = std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5));
    return l[i];
  };
  r.p50_ms = pct(0.5);
  r.p99_ms = pct(0.99);
  r.max_ms = l.empty() ? 0.0 : l.back();
  *out = r;
  return CORR_OK;
}

void corr_svc_destroy(corr_svc* s) {
  if (!s) return;
  if (s->dry) {  // no device state
    delete s;
    return;
  }
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs)
    for (int b = 0; b < 2; ++b) {
      if (kv.second->ev_copy[b]) cudaEventDestroy(kv.second->ev_copy[b]);
      if (kv.second->ev_used[b]) cudaEventDestroy(kv.second->ev_used[b]);
    }
  for (int p = 0; p < 2; ++p) {
    cudaFree(s->d_insts[p]);
    cudaFree(s->d_tmaps[p]);
    cudaFree(s->d_tasks[p]);
    cudaFree(s->d_first[p]);
    if (s->h_insts[p]) cudaFreeHost(s->h_insts[p]);
    if (s->h_tmaps[p]) cudaFreeHost(s->h_tmaps[p]);
    if (s->h_tasks[p]) cudaFreeHost(s->h_tasks[p]);
    if (s->h_first[p]) cudaFreeHost(s->h_first[p]);
    if (s->ev_tick[p]) cudaEventDestroy(s->ev_tick[p]);
  }
  cudaFree(s->base);
  cudaFree(s->d_status);
  cudaFree(s->scratch);
  if (s->h_status) cudaFreeHost(s->h_status);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
