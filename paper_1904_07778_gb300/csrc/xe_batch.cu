// Batches: several arrays correlated in one persistent launch (declared in
// include/xengine.h).  The paper's node (Sec. 2) serves F/N channels of one
// array; a batch serves arrays of different input counts, channel counts and
// block lengths at once.  Every array keeps its own input, corner-turn and
// visibility buffers; one run turns each array's block and then runs ONE
// persistent cross-multiply over the union of all arrays' tasks (each task
// names its array), replayed from a CUDA graph.  The schedule -- how tiles
// are grouped into tasks and which SM runs which task -- is chosen by the
// host, optionally by timing every candidate on the device (autotune).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "xe_internal.h"
#include "xengine.h"

using namespace xe;

struct corr_batch {
  int n = 0, bits = 4;
  unsigned flags = 0;
  // every array is read in payload order (no corner turns; the kernel
  // transposes as it unpacks)
  bool tci = false;
  std::vector<corr_shape> shapes;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<uint8_t*> input, turned;
  std::vector<int64_t*> acc;
  std::vector<HerkInst> insts;       // per array, host copy
  std::vector<CUtensorMap> tmaps;    // per array, host copy
  HerkInst* d_insts = nullptr;
  CUtensorMap* d_tmaps = nullptr;
  // batched launch: all tasks, grouped per CTA
  HerkTask* d_tasks = nullptr;
  int* d_cta_first = nullptr;
  int n_tasks = 0, n_ctas = 0;
  // plain form: each array's own task list
  std::vector<HerkTask*> d_tasks_one;
  std::vector<int> n_tasks_one;
  int schedule = CORR_SCHED_PAIRS_LPT;
  double tuned_ms[3] = {0, 0, 0};
  int tune_source = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* d_status = nullptr;
  int* h_status = nullptr;
  int2* scratch = nullptr;  // 8-bit: per-CTA partial sums of the cross-multiply
  int scratch_ctas = 0;
  // pipelined runs (corr_batch_set_pipeline): array pipe_inst is turned in
  // channel ranges pipe_c[j] .. pipe_c[j+1] on pipe_sms SMs of turn_stream;
  // task list 0 holds the other arrays' tasks, list 1 + j range j's
  int pipe_sms = 0, pipe_inst = -1;
  std::vector<int> pipe_c;
  std::vector<HerkTask*> d_pipe_tasks;
  std::vector<int> n_pipe_tasks;
  cudaStream_t turn_stream = nullptr;
  std::vector<cudaEvent_t> pipe_ev;  // [0] fork, [1 + j] range j turned
};

namespace {

int sm_count() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm > 0 ? nsm : 1;
}

void free_batch(corr_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto p : b->input) cudaFree(p);
  for (auto p : b->turned) cudaFree(p);
  for (auto p : b->acc) cudaFree(p);
  for (auto p : b->d_tasks_one) cudaFree(p);
  for (auto p : b->d_pipe_tasks) cudaFree(p);
  for (auto e : b->pipe_ev) cudaEventDestroy(e);
  if (b->turn_stream) cudaStreamDestroy(b->turn_stream);
  cudaFree(b->d_insts);
  cudaFree(b->d_tmaps);
  cudaFree(b->d_tasks);
  cudaFree(b->d_cta_first);
  cudaFree(b->d_status);
  cudaFree(b->scratch);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Cost of a task for the schedule: its stages times the 128-row blocks it
// streams through shared memory (the unpack, not the MMA, bounds a stage).
double task_cost(const HerkTask& t, const HerkInst& in, int bits) {
  const int nb = t.cb[1] >= 0 ? 2 : 1;
  const bool a_in = t.rb == t.cb[0] || (nb == 2 && t.rb == t.cb[1]);
  const int st = herk_ring_stage(bits);
  return (double)((in.tn + st - 1) / st) * (a_in ? nb : nb + 1);
}

// Build and upload the batched task list of one schedule.
int build_schedule(corr_batch* b, int sched) {
  std::vector<HerkTask> all;
  std::vector<double> cost;
  for (int k = 0; k < b->n; ++k) {
    int rpc = 0;
    const corr_shape& sh = b->shapes[k];
    std::vector<HerkTask> t =
        plan_tasks(sh.n_inputs, sh.n_chans, &rpc, sched == CORR_SCHED_SINGLES_LPT);
    for (HerkTask& x : t) {
      x.inst = k;
      cost.push_back(task_cost(x, b->insts[k], b->bits));
      all.push_back(x);
    }
  }
  const int nt = (int)all.size();
  const int nc = std::min(nt, sm_count());
  std::vector<int> order(nt), first(nc + 1);
  if (sched == CORR_SCHED_PAIRS_RR) {
    // round robin over the arrays' lists in order: CTA c takes c, c + nc, ...
    int pos = 0;
    for (int c = 0; c < nc; ++c) {
      first[c] = pos;
      for (int j = c; j < nt; j += nc) order[pos++] = j;
    }
    first[nc] = pos;
  } else if (corr_plan_schedule(cost.data(), nt, nc, order.data(), first.data()) != CORR_OK) {
    return CORR_EINVAL;
  }
  std::vector<HerkTask> sorted(nt);
  for (int j = 0; j < nt; ++j) sorted[j] = all[order[j]];
  cudaFree(b->d_tasks);
  cudaFree(b->d_cta_first);
  b->d_tasks = nullptr;
  b->d_cta_first = nullptr;
  if (cudaMalloc(&b->d_tasks, sizeof(HerkTask) * nt) != cudaSuccess ||
      cudaMalloc(&b->d_cta_first, sizeof(int) * (nc + 1)) != cudaSuccess)
    return CORR_ENOMEM;
  if (cudaMemcpy(b->d_tasks, sorted.data(), sizeof(HerkTask) * nt, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_cta_first, first.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return CORR_ECUDA;
  b->n_tasks = nt;
  b->n_ctas = nc;
  b->schedule = sched;
  return CORR_OK;
}

HerkArgs batched_args(const corr_batch* b) {
  HerkArgs a;
  memset(&a, 0, sizeof(a));
  a.insts = b->d_insts;
  a.tmaps = b->d_tmaps;
  a.tasks = b->d_tasks;
  a.cta_first = b->d_cta_first;
  a.status = b->d_status;
  a.lo_is_real = (b->flags & CORR_F_LO_IS_REAL) ? 1 : 0;
  a.bits = b->bits;
  a.n_tasks = b->n_tasks;
  a.grid = b->n_ctas;
  a.scratch = b->scratch;
  a.scratch_ctas = b->scratch_ctas;
  return a;
}

// Whether array k is corner-turned before the cross-multiply.
bool turns(const corr_batch* b, int k) {
  return !b->tci && needs_turn(b->shapes[k].layout, b->shapes[k].bits);
}

// Enqueue one run: every array's corner turn, then the batched launch.
cudaError_t enqueue_batched(corr_batch* b) {
  for (int k = 0; k < b->n; ++k) {
    const corr_shape& sh = b->shapes[k];
    if (!turns(b, k)) continue;
    cudaError_t e = turn_rows(b->input[k], b->turned[k], sh.layout, sh.bits, sh.n_inputs,
                              sh.n_chans, sh.n_time, b->insts[k].row_stride, b->stream);
    if (e != cudaSuccess) return e;
  }
  return herk4_launch(batched_args(b), nullptr, b->n_tasks, b->stream, b->tci);
}

// Enqueue one pipelined run: the split array's ranges are turned one after
// another on pipe_sms persistent CTAs of the turn stream; the batch's stream
// turns the other arrays, cross-multiplies them, and then each range once its
// turn is done, every launch capped at the SMs the turn leaves free (so that
// no kernel ever waits for another to start).
cudaError_t enqueue_pipelined(corr_batch* b) {
  const int k = b->pipe_inst, nch = (int)b->pipe_c.size() - 1;
  const corr_shape& sh = b->shapes[k];
  cudaError_t e;
  if ((e = cudaEventRecord(b->pipe_ev[0], b->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(b->turn_stream, b->pipe_ev[0], 0)) != cudaSuccess)
    return e;
  for (int j = 0; j < nch; ++j) {
    if ((e = turn_rows_chans(b->input[k], b->turned[k], sh.layout, sh.bits, sh.n_inputs,
                             sh.n_chans, sh.n_time, b->pipe_c[j], b->pipe_c[j + 1],
                             b->insts[k].row_stride, b->turn_stream, b->pipe_sms)) != cudaSuccess ||
        (e = cudaEventRecord(b->pipe_ev[1 + j], b->turn_stream)) != cudaSuccess)
      return e;
  }
  for (int q = 0; q < b->n; ++q) {
    const corr_shape& s = b->shapes[q];
    if (q == k || !turns(b, q)) continue;
    if ((e = turn_rows(b->input[q], b->turned[q], s.layout, s.bits, s.n_inputs, s.n_chans,
                       s.n_time, b->insts[q].row_stride, b->stream)) != cudaSuccess)
      return e;
  }
  HerkArgs a = batched_args(b);
  a.cta_first = nullptr;
  a.grid = sm_count() - b->pipe_sms;
  for (int j = 0; j <= nch; ++j) {
    // the last wait also joins the turn stream back into the batch's stream
    if (j > 0 && (e = cudaStreamWaitEvent(b->stream, b->pipe_ev[j], 0)) != cudaSuccess) return e;
    if (b->n_pipe_tasks[j] == 0) continue;
    a.tasks = b->d_pipe_tasks[j];
    a.n_tasks = b->n_pipe_tasks[j];
    if ((e = herk4_launch(a, nullptr, a.n_tasks, b->stream)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int capture_graph(corr_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return CORR_ECUDA;
  cudaError_t e = b->pipe_sms > 0 ? enqueue_pipelined(b) : enqueue_batched(b);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return CORR_ECUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return CORR_ECUDA;
  return CORR_OK;
}

int take_status(corr_batch* b) {
  if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return CORR_ECUDA;
  const int st = *b->h_status;
  if (st == 0) return CORR_OK;
  if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return CORR_ECUDA;
  if (st & kStTimeout) return CORR_ETIMEDOUT;
  if (st & kStRange) return CORR_ERANGE;
  return CORR_ECUDA;
}

// Median time of reps batched runs of the current schedule.
double time_schedule(corr_batch* b, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> ms;
  enqueue_batched(b);  // warm
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, b->stream);
    enqueue_batched(b);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms.push_back(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(ms.begin(), ms.end());
  return ms.empty() ? 0.0 : ms[ms.size() / 2];
}

// Autotuner cache: one JSON object per line, {"key": K, "schedule": S,
// "tuned_ms": [a, b, c]}, the key naming the GPU and every array's shape.
std::string tune_key(const corr_batch* b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  std::string k = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? p.name : "unknown";
  for (char& c : k)
    if (c == '"' || c == '\\') c = '_';
  k += "/" + std::to_string(sm_count());
  for (const corr_shape& s : b->shapes)
    k += "|" + std::to_string(s.n_inputs) + "," + std::to_string(s.n_chans) + "," +
         std::to_string(s.n_time) + "," + std::to_string(s.bits) + "," +
         std::to_string(s.layout) + "," + std::to_string(s.flags);
  return k;
}

bool cache_lookup(const char* path, const std::string& key, int* sched, double ms[3]) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  const std::string want = "{\"key\": \"" + key + "\", ";
  bool found = false;
  char line[8192];
  while (fgets(line, sizeof(line), f)) {
    if (strncmp(line, want.c_str(), want.size()) != 0) continue;
    int s = -1;
    double a = 0, b2 = 0, c = 0;
    if (sscanf(line + want.size(), "\"schedule\": %d, \"tuned_ms\": [%lf, %lf, %lf]", &s, &a, &b2,
               &c) == 4 &&
        s >= 0 && s <= 2) {  // the last matching line wins
      *sched = s;
      ms[0] = a;
      ms[1] = b2;
      ms[2] = c;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int sched, const double ms[3]) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"schedule\": %d, \"tuned_ms\": [%.6f, %.6f, %.6f]}\n", key.c_str(),
          sched, ms[0], ms[1], ms[2]);
  fclose(f);
}

}  // namespace

extern "C" {

int corr_plan_schedule(const double* cost, int n_tasks, int n_ctas, int* order, int* cta_first) {
  if (!cost || !order || !cta_first || n_tasks < 0 || n_ctas < 1) return CORR_EINVAL;
  for (int j = 0; j < n_tasks; ++j)
    if (!(cost[j] >= 0.0)) return CORR_EINVAL;
  std::vector<int> idx(n_tasks);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(n_ctas, 0.0);
  std::vector<std::vector<int>> lists(n_ctas);
  for (int j : idx) {
    int best = 0;
    for (int c = 1; c < n_ctas; ++c)
      if (load[c] < load[best]) best = c;
    load[best] += cost[j];
    lists[best].push_back(j);
  }
  int pos = 0;
  for (int c = 0; c < n_ctas; ++c) {
    cta_first[c] = pos;
    for (int j : lists[c]) order[pos++] = j;
  }
  cta_first[n_ctas] = pos;
  return CORR_OK;
}

int corr_batch_create(const corr_shape* shapes, int n, void* stream, int tune, corr_batch** out) {
  TraceRange trace_("corr_batch_create");
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (!shapes || n < 1) return CORR_EINVAL;
  for (int k = 0; k < n; ++k) {
    const corr_shape& s = shapes[k];
    const int chunk = s.bits == 8 ? kMaxChunk8 : kMaxChunk4;
    if (s.n_inputs < 1 || s.n_inputs > 1024 || s.n_chans < 1 || s.n_time < 1 ||
        (s.bits != 4 && s.bits != 8) || s.layout < CORR_L_TCI || s.layout > CORR_L_CIT ||
        (s.flags & ~CORR_F_LO_IS_REAL) || (s.bits == 8 && (s.flags & CORR_F_LO_IS_REAL)) ||
        s.n_time > chunk || s.bits != shapes[0].bits || s.flags != shapes[0].flags ||
        (!needs_turn(s.layout, s.bits) && s.n_time % 16 != 0))
      return CORR_EINVAL;
  }
  corr_batch* b = new (std::nothrow) corr_batch;
  if (!b) return CORR_ENOMEM;
  b->n = n;
  b->bits = shapes[0].bits;
  b->flags = shapes[0].flags;
  b->shapes.assign(shapes, shapes + n);
  b->tci = true;
  for (int k = 0; k < n; ++k) b->tci = b->tci && tci_direct(shapes[k].layout, shapes[k].bits, shapes[k].n_inputs);
  int st = CORR_OK;
  do {
    // graphs cannot be captured on the legacy or per-thread default streams:
    // those (and NULL) get a private stream
    if (stream && (cudaStream_t)stream != cudaStreamLegacy &&
        (cudaStream_t)stream != cudaStreamPerThread) {
      b->stream = (cudaStream_t)stream;
    } else {
      if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
      b->own_stream = true;
    }
    if (cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) { st = CORR_ECUDA; break; }
    if (cudaMallocHost(&b->h_status, sizeof(int)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (b->bits == 8 && herk_scratch_alloc(&b->scratch, &b->scratch_ctas) != cudaSuccess) { st = CORR_ENOMEM; break; }
    b->input.assign(n, nullptr);
    b->turned.assign(n, nullptr);
    b->acc.assign(n, nullptr);
    b->insts.resize(n);
    b->tmaps.resize(n);
    b->d_tasks_one.assign(n, nullptr);
    b->n_tasks_one.assign(n, 0);
    for (int k = 0; k < n && st == CORR_OK; ++k) {
      const corr_shape& s = shapes[k];
      const int R = s.n_inputs * (s.bits / 4);
      const size_t in_bytes = (size_t)R * s.n_chans * s.n_time;
      const size_t nbl = (size_t)s.n_inputs * (s.n_inputs + 1) / 2;
      if (cudaMalloc(&b->input[k], in_bytes) != cudaSuccess ||
          cudaMalloc(&b->acc[k], nbl * s.n_chans * 16) != cudaSuccess) { st = CORR_ENOMEM; break; }
      long long stride = s.n_time;
      const uint8_t* x = b->input[k];
      if (turns(b, k)) {
        stride = ((long long)s.n_time + 31) / 32 * 32;
        if (cudaMalloc(&b->turned[k], (size_t)stride * R * s.n_chans) != cudaSuccess) { st = CORR_ENOMEM; break; }
        x = b->turned[k];
      }
      int rpc = 0;
      std::vector<HerkTask> t = plan_tasks(s.n_inputs, s.n_chans, &rpc);
      HerkInst& in = b->insts[k];
      memset(&in, 0, sizeof(in));
      in.x = x;
      in.acc = b->acc[k];
      in.chan_stride = (long long)R * stride;
      in.row_stride = stride;
      in.n_inputs = s.n_inputs;
      in.n_chans = s.n_chans;
      in.t0 = 0;
      in.tn = s.n_time;
      in.rows_per_chan = rpc;
      in.accumulate = 0;
      in.vec_ok = 1;
      if (!make_herk_tmap(&b->tmaps[k], x, b->tci, s.bits, R, s.n_chans, s.n_time, stride, rpc)) { st = CORR_ECUDA; break; }
      b->n_tasks_one[k] = (int)t.size();
      if (cudaMalloc(&b->d_tasks_one[k], sizeof(HerkTask) * t.size()) != cudaSuccess) { st = CORR_ENOMEM; break; }
      if (cudaMemcpy(b->d_tasks_one[k], t.data(), sizeof(HerkTask) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) { st = CORR_ECUDA; break; }
    }
    if (st != CORR_OK) break;
    if (cudaMalloc(&b->d_insts, sizeof(HerkInst) * n) != cudaSuccess ||
        cudaMalloc(&b->d_tmaps, sizeof(CUtensorMap) * n) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMemcpy(b->d_insts, b->insts.data(), sizeof(HerkInst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tmaps, b->tmaps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice) != cudaSuccess) { st = CORR_ECUDA; break; }
    const char* cache = tune ? getenv("XE_TUNE_CACHE") : nullptr;
    int cached_s = -1;
    if (cache && *cache && cache_lookup(cache, tune_key(b), &cached_s, b->tuned_ms)) {
      b->tune_source = 2;
      st = build_schedule(b, cached_s);
    } else if (tune) {
      double best = 0.0;
      int best_s = CORR_SCHED_PAIRS_LPT;
      for (int sch = 0; sch < 3 && st == CORR_OK; ++sch) {
        st = build_schedule(b, sch);
        if (st != CORR_OK) break;
        const double ms = time_schedule(b, 5);
        b->tuned_ms[sch] = ms;
        if (sch == 0 || ms < best) {
          best = ms;
          best_s = sch;
        }
      }
      if (st != CORR_OK) break;
      // the tuning runs read whatever the inputs held: drop their status
      if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
          cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) { st = CORR_ECUDA; break; }
      st = build_schedule(b, best_s);
      b->tune_source = 1;
      if (cache && *cache) cache_store(cache, tune_key(b), best_s, b->tuned_ms);
    } else {
      st = build_schedule(b, CORR_SCHED_PAIRS_LPT);
    }
    if (st != CORR_OK) break;
    // set every launch attribute outside the capture, then capture one run
    if (enqueue_batched(b) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess ||
        cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) { st = CORR_ECUDA; break; }
    st = capture_graph(b);
  } while (0);
  if (st != CORR_OK) {
    cudaGetLastError();
    free_batch(b);
    return st;
  }
  *out = b;
  return CORR_OK;
}

void* corr_batch_input(corr_batch* b, int k) {
  return (b && k >= 0 && k < b->n) ? b->input[k] : nullptr;
}

int64_t* corr_batch_output(corr_batch* b, int k) {
  return (b && k >= 0 && k < b->n) ? b->acc[k] : nullptr;
}

int corr_batch_set_input(corr_batch* b, int k, const void* src, size_t nbytes) {
  if (!b || k < 0 || k >= b->n || !src) return CORR_EINVAL;
  const corr_shape& s = b->shapes[k];
  if (nbytes != (size_t)s.n_inputs * s.n_chans * s.n_time * (s.bits / 4)) return CORR_EINVAL;
  return cudaMemcpyAsync(b->input[k], src, nbytes, cudaMemcpyDefault, b->stream) == cudaSuccess
             ? CORR_OK
             : CORR_ECUDA;
}

int corr_batch_get_output(corr_batch* b, int k, int64_t* dst) {
  if (!b || k < 0 || k >= b->n || !dst) return CORR_EINVAL;
  const corr_shape& s = b->shapes[k];
  const size_t bytes = (size_t)s.n_inputs * (s.n_inputs + 1) / 2 * s.n_chans * 16;
  if (cudaMemcpyAsync(dst, b->acc[k], bytes, cudaMemcpyDefault, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return CORR_ECUDA;
  return CORR_OK;
}

int corr_batch_run(corr_batch* b) {
  TraceRange trace_("corr_batch_run");
  if (!b || !b->exec) return CORR_EINVAL;
  return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? CORR_OK : CORR_ECUDA;
}

int corr_batch_run_plain(corr_batch* b) {
  TraceRange trace_("corr_batch_run_plain");
  if (!b) return CORR_EINVAL;
  for (int k = 0; k < b->n; ++k) {
    const corr_shape& sh = b->shapes[k];
    if (turns(b, k) &&
        turn_rows(b->input[k], b->turned[k], sh.layout, sh.bits, sh.n_inputs, sh.n_chans,
                  sh.n_time, b->insts[k].row_stride, b->stream) != cudaSuccess)
      return CORR_ECUDA;
    HerkArgs a;
    memset(&a, 0, sizeof(a));
    a.in = b->insts[k];
    a.tasks = b->d_tasks_one[k];
    a.status = b->d_status;
    a.lo_is_real = (b->flags & CORR_F_LO_IS_REAL) ? 1 : 0;
    a.bits = b->bits;
    a.n_tasks = b->n_tasks_one[k];
    a.scratch = b->scratch;
    a.scratch_ctas = b->scratch_ctas;
    if (herk4_launch(a, &b->tmaps[k], a.n_tasks, b->stream, b->tci) != cudaSuccess) return CORR_ECUDA;
  }
  return CORR_OK;
}

int corr_batch_set_pipeline(corr_batch* b, int turn_sms, int n_chunks) {
  TraceRange trace_("corr_batch_set_pipeline");
  if (!b || turn_sms < 0 || turn_sms >= sm_count() || n_chunks < 1) return CORR_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CORR_ECUDA;
  if (turn_sms == 0) {
    b->pipe_sms = 0;
    return capture_graph(b);
  }
  // the array with the most bytes to turn that can be cut by channels
  int k = -1;
  double most = 0.0;
  for (int q = 0; q < b->n; ++q) {
    const corr_shape& s = b->shapes[q];
    const double bytes = (double)s.n_inputs * s.n_chans * s.n_time;
    if (s.bits == 4 && (s.layout == CORR_L_TCI || s.layout == CORR_L_TIC) && 2 * s.n_inputs > 64 &&
        bytes > most) {
      most = bytes;
      k = q;
    }
  }
  if (k < 0 || b->tci) return CORR_EINVAL;  // no corner turn to overlap
  const corr_shape& sh = b->shapes[k];
  // ranges start on whole 128-byte tiles of the input rows: channel c0 starts
  // at byte c0 of a [t][i][c] row and at byte c0 N of a [t][c][i] row
  const int unit = sh.layout == CORR_L_TIC ? 128 : 128 / std::gcd(sh.n_inputs, 128);
  const int nch = std::max(1, std::min(n_chunks, sh.n_chans / unit));
  std::vector<int> c(1, 0);
  for (int j = 1; j < nch; ++j) {
    const int cj = (int)((long long)j * sh.n_chans / nch) / unit * unit;
    if (cj > c.back()) c.push_back(cj);
  }
  c.push_back(sh.n_chans);
  // task lists: the other arrays, then each range of the split array
  std::vector<std::vector<HerkTask>> lists(c.size());
  for (int q = 0; q < b->n; ++q) {
    const corr_shape& s = b->shapes[q];
    int rpc = 0;
    for (HerkTask x : plan_tasks(s.n_inputs, s.n_chans, &rpc)) {
      x.inst = q;
      int li = 0;
      if (q == k) {
        li = 1;
        while (li + 1 < (int)c.size() && x.chan0 >= c[li]) ++li;
      }
      lists[li].push_back(x);
    }
  }
  // Build the new device task lists first.  The graph captured now may still
  // reference the old lists, so they are freed only after a new graph has
  // replaced it; on an early error the old graph and its lists stay as they
  // were.
  std::vector<HerkTask*> d_new(lists.size(), nullptr);
  std::vector<int> n_new(lists.size(), 0);
  auto drop_new = [&](int st) {
    for (auto p : d_new) cudaFree(p);
    cudaGetLastError();
    return st;
  };
  for (size_t j = 0; j < lists.size(); ++j) {
    n_new[j] = (int)lists[j].size();
    if (lists[j].empty()) continue;
    if (cudaMalloc(&d_new[j], sizeof(HerkTask) * lists[j].size()) != cudaSuccess) {
      d_new[j] = nullptr;
      return drop_new(CORR_ENOMEM);
    }
    if (cudaMemcpy(d_new[j], lists[j].data(), sizeof(HerkTask) * lists[j].size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return drop_new(CORR_ECUDA);
  }
  if (!b->turn_stream && cudaStreamCreateWithFlags(&b->turn_stream, cudaStreamNonBlocking) != cudaSuccess) {
    b->turn_stream = nullptr;
    return drop_new(CORR_ECUDA);
  }
  while (b->pipe_ev.size() < c.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return drop_new(CORR_ECUDA);
    b->pipe_ev.push_back(e);
  }
  std::vector<HerkTask*> d_old;
  d_old.swap(b->d_pipe_tasks);
  b->d_pipe_tasks = d_new;
  b->n_pipe_tasks = n_new;
  b->pipe_inst = k;
  b->pipe_c = c;
  b->pipe_sms = turn_sms;
  // set every launch attribute outside the capture, then capture one run
  int st = CORR_OK;
  if (enqueue_pipelined(b) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    st = CORR_ECUDA;
  } else {
    st = capture_graph(b);
  }
  if (st != CORR_OK) {  // back to the single-launch graph, which uses no range lists
    b->pipe_sms = 0;
    cudaGetLastError();
    capture_graph(b);
  }
  // no graph references the old lists any more (capture_graph destroyed it)
  for (auto p : d_old) cudaFree(p);
  return st;
}

int corr_batch_sync(corr_batch* b) {
  if (!b) return CORR_EINVAL;
  return take_status(b);
}

int corr_batch_info_get(corr_batch* b, corr_batch_info* out) {
  if (!b || !out) return CORR_EINVAL;
  out->schedule = b->schedule;
  out->n_tasks = b->n_tasks;
  out->n_ctas = b->n_ctas;
  int launches = 1;
  for (int q = 0; q < b->n; ++q) launches += turns(b, q) ? 1 : 0;
  if (b->pipe_sms > 0) {  // the split array: one turn and one cross-multiply per range
    const int nch = (int)b->pipe_c.size() - 1;
    launches = 2 * nch;
    for (int q = 0; q < b->n; ++q)
      if (q != b->pipe_inst && turns(b, q)) ++launches;
    if (b->n_pipe_tasks[0] > 0) ++launches;
  }
  out->launches_per_run = launches;
  for (int i = 0; i < 3; ++i) out->tuned_ms[i] = b->tuned_ms[i];
  out->tune_source = b->tune_source;
  return CORR_OK;
}

void corr_batch_destroy(corr_batch* b) { free_batch(b); }

}  // extern "C"
