// C ABI of the X-engine (declared in include/xengine.h): context lifetime,
// ingest staging, corner turn, the tensor-core cross-multiply, integration
// state and dumps.  Every step of the data path runs in this library's
// kernels on the context's stream.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "xe_internal.h"
#include "xengine.h"

using namespace xe;

namespace xe {

bool make_herk_tmap(CUtensorMap* m, const uint8_t* x, bool tci, int bits, int R, int n_chans,
                    int n_time, long long row_stride, int rpc) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // a box: one 128-row operand block of one stage (8 KB of packed bytes)
  const cuuint32_t box_t = (cuuint32_t)herk_ring_stage(bits);
  const cuuint32_t box_rows = (cuuint32_t)((rpc ? rpc : 128) * bits / 8);
  const cuuint32_t box_chans = (cuuint32_t)(rpc ? 128 / rpc : 1);
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3];
  if (tci) {
    dims[0] = (cuuint64_t)R, dims[1] = (cuuint64_t)n_chans, dims[2] = (cuuint64_t)n_time;
    strides[0] = (cuuint64_t)R, strides[1] = (cuuint64_t)R * n_chans;
    box[0] = box_rows, box[1] = box_chans, box[2] = box_t;
  } else {
    dims[0] = (cuuint64_t)n_time, dims[1] = (cuuint64_t)R, dims[2] = (cuuint64_t)n_chans;
    strides[0] = (cuuint64_t)row_stride, strides[1] = (cuuint64_t)row_stride * R;
    box[0] = box_t, box[1] = box_rows, box[2] = box_chans;
  }
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(x), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t herk_scratch_alloc(int2** p, int* ctas) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *ctas = nsm;
  return cudaMalloc(p, (size_t)nsm * kHerkScratchInt2 * sizeof(int2));
}

bool tci_direct(int layout, int bits, int n_inputs) {
  const int R = n_inputs * (bits / 4);  // byte rows per (spectrum, channel)
  // The channel stride (R bytes) must suit TMA.  Stacked arrays fill a box
  // exactly (R byte rows = one channel's rows of the 128-row block: 16 or 32
  // at 4 bits, 16, 32 or 64 at 8 bits); larger ones take whole boxes of 64
  // (4-bit) or 128 (8-bit) byte rows.  Reading the block directly beats
  // turning it first at every size measured (512 inputs, 1024 channels,
  // 4096 spectra, 4-bit: 3.15 against 3.46 ms a block; 8-bit, 2048 channels:
  // 17.3 against 18.9 ms), although many tasks then read each block's short
  // time-major boxes.
  if (layout != CORR_L_TCI || R % 16 != 0) return false;
  const int box = bits == 8 ? 128 : 64;  // byte rows of a 128-row block
  return R >= box || R == 16 || R == 32 || (bits == 8 && R == 64);
}

// Tasks of the real Gram matrix (n inputs: 2n rows of Y): every 128 x 128
// block (r, c), c <= r, of the lower triangle exactly once.  Row block r takes the column blocks
// r, r+1, ..., r + (nrb-1)/2 (mod nrb) -- for even nrb, r + nrb/2 goes to
// the smaller of the two -- so the work is spread evenly over the row
// blocks.  Columns r and r+1 form one 128 x 256 MMA task; further columns
// are 128 x 128 tasks.  Ordered by decreasing work.
std::vector<HerkTask> plan_tasks(int n, int c, int* rows_per_chan, bool singles) {
  std::vector<HerkTask> t;
  const int rows = 2 * n;
  if (rows <= 64) {
    int rpc = 2;
    while (rpc < rows) rpc <<= 1;
    *rows_per_chan = rpc;
    const int per = 128 / rpc;
    for (int c0 = 0; c0 < c; c0 += per) t.push_back({c0, 0, {0, -1}, 0});
    return t;
  }
  *rows_per_chan = 0;
  const int nrb = (rows + 127) / 128;
  for (int ch = 0; ch < c; ++ch)
    for (int r = 0; r < nrb; ++r) {
      std::vector<int> cols;
      for (int d = 0; 2 * d < nrb; ++d)
        if (2 * d != nrb || r < nrb / 2) cols.push_back((r + d) % nrb);
      if (nrb % 2 == 0 && r < nrb / 2 && 2 * (nrb / 2) == nrb) cols.push_back(r + nrb / 2);
      // the first two columns (r and r+1) share the A rows with a B block;
      // the others take one column each so at most two blocks are resident
      if (singles) {
        for (size_t k = 0; k < cols.size(); ++k) t.push_back({ch, r, {cols[k], -1}, 0});
      } else {
        t.push_back({ch, r, {cols[0], cols.size() > 1 ? cols[1] : -1}, 0});
        for (size_t k = 2; k < cols.size(); ++k) t.push_back({ch, r, {cols[k], -1}, 0});
      }
    }
  std::stable_sort(t.begin(), t.end(), [](const HerkTask& x, const HerkTask& y) {
    return (x.cb[1] >= 0) > (y.cb[1] >= 0);
  });
  return t;
}

}  // namespace xe

struct corr_ctx {
  int n_inputs = 0, n_chans = 0, n_time = 0, bits = 4, layout = 0;
  unsigned flags = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t copy_stream = nullptr;
  size_t block_bytes = 0;
  int64_t* acc = nullptr;  // int64 [C][B][2] long integration (acc_buf[cur] or bound)
  size_t acc_bytes = 0;
  bool acc_live = false;   // false: next push stores instead of adding
  int64_t* bound = nullptr;  // the caller's buffer of this integration (corr_bind)
  // Overlapped dumps (corr_dump_async): a reset switches to the other
  // accumulator while the copy of the finished one runs on dump_stream.
  int64_t* acc_buf[2] = {nullptr, nullptr};
  int cur = 0;
  cudaStream_t dump_stream = nullptr;
  cudaEvent_t acc_free[2] = {nullptr, nullptr};  // last copy out of acc_buf[k] done
  bool read_pending[2] = {false, false};
  struct AsyncDump {
    cudaEvent_t done;
    int slot;  // index into h_dump_status
  };
  std::vector<AsyncDump> dumps;  // outstanding, oldest first
  // dump events reused across dumps: the stream wait on `dump_ready` takes
  // its record at the call, so the next dump may record it again; a `done`
  // event returns to the pool once corr_dump_wait has seen it complete
  cudaEvent_t dump_ready = nullptr;
  std::vector<cudaEvent_t> done_pool;
  int* h_dump_status = nullptr;  // pinned, kMaxAsyncDumps status snapshots
  int* d_dump_status = nullptr;  // the same slots as the device writes them (mapped)
  uint8_t* stage[2] = {nullptr, nullptr};
  cudaEvent_t stage_free[2] = {nullptr, nullptr};
  cudaEvent_t stage_ready[2] = {nullptr, nullptr};
  int stage_next = 0;
  uint8_t* turned = nullptr;  // corner-turned copy of the block, [c][i][t] (= turned_buf[0])
  // Pipelined corner turn (corr_set_pipeline): the turn of block k+1 runs on
  // pipe_sms SMs of turn_stream while the cross-multiply of block k holds the
  // other SMs on herk_stream; the two turned buffers alternate.
  int pipe_sms = 0;
  unsigned pipe_k = 0;
  bool herk_pending = false;   // herk_stream has work the caller's stream has not joined
  uint8_t* turned_buf[2] = {nullptr, nullptr};
  cudaStream_t turn_stream = nullptr, herk_stream = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, turn_done[2] = {nullptr, nullptr};
  cudaEvent_t herk_done[2] = {nullptr, nullptr}, herk_last = nullptr;
  long long turned_stride = 0;  // bytes per (channel, input) row of `turned`
  HerkTask* tasks = nullptr;
  int n_tasks = 0;
  int2* scratch = nullptr;  // 8-bit: per-CTA partial sums of the cross-multiply
  int scratch_ctas = 0;
  // host-side caches of the push path: two block addresses known to be device
  // memory, and the tensor maps of the last two sources (the other parameters
  // of a map are fixed per context)
  const void* dev_seen[2] = {nullptr, nullptr};
  int dev_seen_next = 0;
  struct MapCache {
    const uint8_t* src = nullptr;
    bool tci = false;
    CUtensorMap map;
  } map_cache[2];
  int map_next = 0;
  // corr_push_many: the per-block instances and tensor maps of one launch
  // over several blocks (device tables, filled from pinned staging).  Two
  // tables alternate, so that a call can fill one while the cross-multiply
  // of the call before still reads the other; a table whose blocks and
  // accumulator match the call is reused without a copy.
  struct ManyTable {
    HerkInst* d_insts = nullptr;
    CUtensorMap* d_maps = nullptr;
    HerkInst* h_insts = nullptr;
    CUtensorMap* h_maps = nullptr;
    int cap = 0;
    std::vector<const void*> key;  // the blocks whose instances the table holds
    int64_t* key_acc = nullptr;    // ... and their accumulator
    cudaEvent_t done = nullptr;    // after the last launch that read the table
    bool used = false;
  } many[2];
  int many_next = 0;
  // the task list of a launch over k blocks: the base list repeated with
  // the instance index, task i = base[i % n_tasks] of block i / n_tasks; any
  // prefix is the list of fewer blocks, so one array serves every call
  HerkTask* many_tasks = nullptr;
  int many_tasks_inst = 0;  // instances the array covers
  std::vector<HerkTask> host_tasks;  // the base list
  int rows_per_chan = 0;
  int smem_bytes = 0;
  int* d_status = nullptr;
  int* h_status = nullptr;  // pinned
  double* rho_tmp = nullptr;
  uint8_t* flag_tmp = nullptr;
  bool seq_started = false;
  uint64_t next_seq = 0;
  // run-time counters and optional per-phase event timing
  corr_stats stats{};
  bool timing = false;
  // fault injection for the tests of the bounded device waits (HerkInst::fault; 0 = off)
  int fault = 0;
  struct Timed {
    int phase;
    cudaEvent_t begin, end;
  };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
};

namespace {

enum Phase { kTurn, kHerk, kCopyIn, kDump, kNorm };

cudaEvent_t take_event(corr_ctx* x) {
  if (!x->pool.empty()) {
    cudaEvent_t e = x->pool.back();
    x->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Start timing a phase on stream s (no-op while timing is off).
cudaEvent_t phase_begin(corr_ctx* x, cudaStream_t s) {
  if (!x->timing) return nullptr;
  cudaEvent_t e = take_event(x);
  if (e && cudaEventRecord(e, s) != cudaSuccess) {
    x->pool.push_back(e);
    return nullptr;
  }
  return e;
}

void phase_end(corr_ctx* x, int phase, cudaEvent_t begin, cudaStream_t s) {
  if (!begin) return;
  cudaEvent_t e = take_event(x);
  if (!e || cudaEventRecord(e, s) != cudaSuccess) {
    x->pool.push_back(begin);
    if (e) x->pool.push_back(e);
    return;
  }
  x->pending.push_back({phase, begin, e});
}

// Fold completed phase timings into the counters (streams must be idle).
void collect_timings(corr_ctx* x) {
  for (auto& t : x->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.begin, t.end) == cudaSuccess) {
      switch (t.phase) {
        case kTurn: x->stats.turn_ms += ms; ++x->stats.timed_turn; break;
        case kHerk: x->stats.herk_ms += ms; ++x->stats.timed_herk; break;
        case kCopyIn: x->stats.copy_in_ms += ms; break;
        case kDump: x->stats.dump_ms += ms; break;
        default: x->stats.norm_ms += ms; break;
      }
    } else {
      cudaGetLastError();
    }
    x->pool.push_back(t.begin);
    x->pool.push_back(t.end);
  }
  x->pending.clear();
}

int cuda_fail(cudaError_t e) {
  (void)e;
  return CORR_ECUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_ctx(corr_ctx* x) {
  if (!x) return;
  if (x->stream) cudaStreamSynchronize(x->stream);
  if (x->copy_stream) cudaStreamSynchronize(x->copy_stream);
  if (x->dump_stream) cudaStreamSynchronize(x->dump_stream);
  if (x->turn_stream) cudaStreamSynchronize(x->turn_stream);
  if (x->herk_stream) cudaStreamSynchronize(x->herk_stream);
  cudaFree(x->turned_buf[1]);
  for (int i = 0; i < 2; ++i)
    for (cudaEvent_t e : {x->ev_in[i], x->turn_done[i], x->herk_done[i]})
      if (e) cudaEventDestroy(e);
  if (x->herk_last) cudaEventDestroy(x->herk_last);
  if (x->turn_stream) cudaStreamDestroy(x->turn_stream);
  if (x->herk_stream) cudaStreamDestroy(x->herk_stream);
  cudaFree(x->acc_buf[0]);
  cudaFree(x->acc_buf[1]);
  for (int i = 0; i < 2; ++i)
    if (x->acc_free[i]) cudaEventDestroy(x->acc_free[i]);
  for (auto& d : x->dumps) cudaEventDestroy(d.done);
  for (cudaEvent_t e : x->done_pool) cudaEventDestroy(e);
  if (x->dump_ready) cudaEventDestroy(x->dump_ready);
  if (x->h_dump_status) cudaFreeHost(x->h_dump_status);
  if (x->dump_stream) cudaStreamDestroy(x->dump_stream);
  for (int i = 0; i < 2; ++i) {
    cudaFree(x->stage[i]);
    if (x->stage_free[i]) cudaEventDestroy(x->stage_free[i]);
    if (x->stage_ready[i]) cudaEventDestroy(x->stage_ready[i]);
  }
  cudaFree(x->many_tasks);
  for (auto& t : x->many) {
    cudaFree(t.d_insts);
    cudaFree(t.d_maps);
    if (t.h_insts) cudaFreeHost(t.h_insts);
    if (t.h_maps) cudaFreeHost(t.h_maps);
    if (t.done) cudaEventDestroy(t.done);
  }
  cudaFree(x->turned);
  cudaFree(x->tasks);
  cudaFree(x->scratch);
  cudaFree(x->d_status);
  cudaFree(x->rho_tmp);
  cudaFree(x->flag_tmp);
  for (auto& t : x->pending) {
    cudaEventDestroy(t.begin);
    cudaEventDestroy(t.end);
  }
  for (auto e : x->pool) cudaEventDestroy(e);
  if (x->h_status) cudaFreeHost(x->h_status);
  if (x->copy_stream) cudaStreamDestroy(x->copy_stream);
  if (x->own_stream && x->stream) cudaStreamDestroy(x->stream);
  delete x;
}

// Before the context's stream writes the current accumulator: wait for an
// overlapped dump that still reads it.
int guard_acc_write(corr_ctx* x, cudaStream_t writer) {
  if (!x->read_pending[x->cur]) return CORR_OK;
  if (cudaStreamWaitEvent(writer, x->acc_free[x->cur], 0) != cudaSuccess) return CORR_ECUDA;
  x->read_pending[x->cur] = false;
  return CORR_OK;
}

// End of an integration: the next one starts in the context's own accumulator.
void unbind(corr_ctx* x) {
  if (!x->bound) return;
  x->bound = nullptr;
  x->acc = x->acc_buf[x->cur];
}

// The stream on which the accumulators and the status word are written:
// the cross-multiply's own stream while the corner turn is pipelined.
cudaStream_t acc_stream(corr_ctx* x) {
  return x->pipe_sms > 0 && turn_can_persist(x->layout, x->bits) ? x->herk_stream : x->stream;
}

// Make the caller's stream wait for the pipelined cross-multiplies before it
// touches the accumulators or the status word.
int pipe_join(corr_ctx* x) {
  if (!x->herk_pending) return CORR_OK;
  if (cudaEventRecord(x->herk_last, x->herk_stream) != cudaSuccess ||
      cudaStreamWaitEvent(x->stream, x->herk_last, 0) != cudaSuccess)
    return CORR_ECUDA;
  x->herk_pending = false;
  return CORR_OK;
}

int status_code(int st) {
  if (st == 0) return CORR_OK;
  if (st & kStTimeout) return CORR_ETIMEDOUT;
  if (st & kStRange) return CORR_ERANGE;
  return CORR_ECUDA;
}

// Read and clear the device status word (waits for the stream).
int take_status(corr_ctx* x) {
  if (cudaMemcpyAsync(x->h_status, x->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                      x->stream) != cudaSuccess)
    return CORR_ECUDA;
  if (cudaStreamSynchronize(x->stream) != cudaSuccess) return CORR_ECUDA;
  const int st = *x->h_status;
  if (st == 0) return CORR_OK;
  if (cudaMemsetAsync(x->d_status, 0, sizeof(int), x->stream) != cudaSuccess) return CORR_ECUDA;
  if (cudaStreamSynchronize(x->stream) != cudaSuccess) return CORR_ECUDA;
  return status_code(st);
}

}  // namespace

extern "C" {

const char* corr_strerror(int status) {
  switch (status) {
    case CORR_OK: return "ok";
    case CORR_EINVAL: return "invalid argument";
    case CORR_ENOMEM: return "out of memory";
    case CORR_EBUSY: return "memory budget exhausted";
    case CORR_ERANGE: return "8-bit sample equal to -128";
    case CORR_ESEQ: return "block sequence gap or duplicate";
    case CORR_ETIMEDOUT: return "device-side wait timed out";
    case CORR_ECUDA: return "CUDA runtime error";
    case CORR_ESTATE: return "invalid state";
    case CORR_ECORRUPT: return "packet failed its CRC check";
    default: return "unknown status";
  }
}

int64_t corr_n_baselines(int n_inputs) {
  return n_inputs < 1 ? 0 : (int64_t)n_inputs * (n_inputs + 1) / 2;
}

int corr_create(int n_inputs, int n_chans, int n_time, int bits, int layout, unsigned flags,
                void* stream, corr_ctx** out) {
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_inputs < 1 || n_inputs > 1024 || n_chans < 1 || n_time < 1 || (bits != 4 && bits != 8) ||
      layout < CORR_L_TCI || layout > CORR_L_CIT || (flags & ~CORR_F_LO_IS_REAL) ||
      (bits == 8 && (flags & CORR_F_LO_IS_REAL)))
    return CORR_EINVAL;
  const size_t block_bytes = (size_t)n_inputs * n_chans * n_time * (size_t)(bits / 4);
  if (block_bytes / (size_t)n_inputs / (size_t)n_chans != (size_t)n_time * (bits / 4))
    return CORR_EINVAL;
  corr_ctx* x = new (std::nothrow) corr_ctx;
  if (!x) return CORR_ENOMEM;
  x->n_inputs = n_inputs;
  x->n_chans = n_chans;
  x->n_time = n_time;
  x->bits = bits;
  x->layout = layout;
  x->flags = flags;
  x->block_bytes = block_bytes;
  if (cudaGetDevice(&x->device) != cudaSuccess) {
    delete x;
    return CORR_ECUDA;
  }
  int st = CORR_OK;
  do {
    if (stream) {
      x->stream = (cudaStream_t)stream;
    } else {
      if (cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
      x->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&x->copy_stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
    x->acc_bytes = (size_t)corr_n_baselines(n_inputs) * n_chans * 2 * sizeof(int64_t);
    if (cudaMalloc(&x->acc_buf[0], x->acc_bytes) != cudaSuccess) { st = CORR_ENOMEM; break; }
    x->acc = x->acc_buf[0];
    x->turned_stride = ((long long)n_time + 31) / 32 * 32;  // 32-byte rows for the corner turn
    // byte rows per channel: one per input (4-bit), re and im bytes (8-bit)
    const int byte_rows = n_inputs * (bits / 4);
    if ((layout != CORR_L_CIT || bits == 8) &&
        cudaMalloc(&x->turned, (size_t)x->turned_stride * byte_rows * n_chans) != cudaSuccess) { st = CORR_ENOMEM; break; }
    x->turned_buf[0] = x->turned;
    if (cudaMalloc(&x->d_status, sizeof(int)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMemset(x->d_status, 0, sizeof(int)) != cudaSuccess) { st = CORR_ECUDA; break; }
    if (cudaMallocHost(&x->h_status, sizeof(int)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    for (int i = 0; i < 2; ++i) {
      if (cudaEventCreateWithFlags(&x->stage_free[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&x->stage_ready[i], cudaEventDisableTiming) != cudaSuccess) {
        st = CORR_ECUDA;
        break;
      }
    }
    if (st != CORR_OK) break;
    std::vector<HerkTask> tasks = plan_tasks(n_inputs, n_chans, &x->rows_per_chan);
    x->n_tasks = (int)tasks.size();
    x->host_tasks = tasks;
    if (bits == 8 && herk_scratch_alloc(&x->scratch, &x->scratch_ctas) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMalloc(&x->tasks, tasks.size() * sizeof(HerkTask)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMemcpy(x->tasks, tasks.data(), tasks.size() * sizeof(HerkTask), cudaMemcpyHostToDevice) != cudaSuccess) { st = CORR_ECUDA; break; }
    x->smem_bytes = herk4_max_smem();
    if (x->smem_bytes < 4 * 2 * (16384 + 8192) + 1024) { st = CORR_ECUDA; break; }
  } while (0);
  if (st != CORR_OK) {
    free_ctx(x);
    return st;
  }
  *out = x;
  return CORR_OK;
}

int corr_push(corr_ctx* x, const void* block, size_t nbytes, uint64_t seq) {
  TraceRange trace_("corr_push");
  if (!x || !block) return CORR_EINVAL;
  if (nbytes != x->block_bytes) return CORR_EINVAL;
  if (seq != CORR_SEQ_ANY) {
    if (x->seq_started && seq != x->next_seq) {
      ++x->stats.seq_rejects;
      return CORR_ESEQ;
    }
    x->seq_started = true;
    x->next_seq = seq + 1;
  }
  const uint8_t* src = static_cast<const uint8_t*>(block);
  // Pipelined: the turn runs on turn_stream after the caller's work so far
  // (the producer of this block) and after the cross-multiply that last read
  // its turned buffer; the cross-multiply runs on herk_stream.
  const bool pipe = x->pipe_sms > 0 && turn_can_persist(x->layout, x->bits);
  const int pk = x->pipe_k & 1;
  cudaStream_t ts = pipe ? x->turn_stream : x->stream;
  cudaStream_t hs = pipe ? x->herk_stream : x->stream;
  if (pipe && (cudaEventRecord(x->ev_in[pk], x->stream) != cudaSuccess ||
               cudaStreamWaitEvent(ts, x->ev_in[pk], 0) != cudaSuccess ||
               cudaStreamWaitEvent(ts, x->herk_done[pk], 0) != cudaSuccess))
    return CORR_ECUDA;
  int slot = -1;
  bool on_device = block == x->dev_seen[0] || block == x->dev_seen[1];
  if (!on_device && is_device_ptr(block)) {
    on_device = true;
    x->dev_seen[x->dev_seen_next] = block;
    x->dev_seen_next ^= 1;
  }
  if (!on_device) {
    slot = x->stage_next;
    x->stage_next ^= 1;
    if (!x->stage[slot] && cudaMalloc(&x->stage[slot], x->block_bytes) != cudaSuccess)
      return CORR_ENOMEM;
    if (cudaStreamWaitEvent(x->copy_stream, x->stage_free[slot], 0) != cudaSuccess)
      return CORR_ECUDA;
    cudaEvent_t tc = phase_begin(x, x->copy_stream);
    if (cudaMemcpyAsync(x->stage[slot], block, nbytes, cudaMemcpyHostToDevice, x->copy_stream) !=
        cudaSuccess)
      return CORR_ECUDA;
    phase_end(x, kCopyIn, tc, x->copy_stream);
    if (cudaEventRecord(x->stage_ready[slot], x->copy_stream) != cudaSuccess ||
        cudaStreamWaitEvent(ts, x->stage_ready[slot], 0) != cudaSuccess)
      return CORR_ECUDA;
    src = x->stage[slot];
  }
  const int N = x->n_inputs, C = x->n_chans, T = x->n_time;
  const bool eight = x->bits == 8;
  const int R = eight ? 2 * N : N;  // byte rows per channel
  long long row_stride = T;
  // payload order read directly (the kernel transposes as it unpacks) unless
  // the corner turn is pipelined or the block is not 16-byte aligned
  const bool tci = !pipe && tci_direct(x->layout, x->bits, N) &&
                   reinterpret_cast<uintptr_t>(src) % 16 == 0;
  if (needs_turn(x->layout, x->bits) && !tci) {
    uint8_t* turned = pipe ? x->turned_buf[pk] : x->turned;
    cudaEvent_t tt = phase_begin(x, ts);
    cudaError_t e = turn_rows(src, turned, x->layout, x->bits, N, C, T, x->turned_stride, ts,
                              pipe ? x->pipe_sms : 0);
    if (e != cudaSuccess) return cuda_fail(e);
    phase_end(x, kTurn, tt, ts);
    ++x->stats.turn_launches;
    src = turned;
    row_stride = x->turned_stride;
  }
  if (pipe) {
    // the caller's stream only waits for the turn, the block's one reader
    if (cudaEventRecord(x->turn_done[pk], ts) != cudaSuccess ||
        cudaStreamWaitEvent(x->stream, x->turn_done[pk], 0) != cudaSuccess ||
        cudaStreamWaitEvent(hs, x->turn_done[pk], 0) != cudaSuccess ||
        (slot >= 0 && cudaEventRecord(x->stage_free[slot], ts) != cudaSuccess))
      return CORR_ECUDA;
  }
  HerkArgs a;
  memset(&a, 0, sizeof(a));
  a.in.x = src;
  a.in.fault = x->fault;
  a.in.acc = x->acc;
  a.tasks = x->tasks;
  a.status = x->d_status;
  a.in.chan_stride = (long long)R * row_stride;
  a.in.row_stride = row_stride;
  a.in.n_inputs = N;
  a.in.n_chans = C;
  a.in.rows_per_chan = x->rows_per_chan;
  a.lo_is_real = (x->flags & CORR_F_LO_IS_REAL) ? 1 : 0;
  a.smem_bytes = x->smem_bytes;
  a.n_tasks = x->n_tasks;
  a.bits = x->bits;
  a.scratch = x->scratch;
  a.scratch_ctas = x->scratch_ctas;
  // The TMA kernel needs 16-byte aligned rows; otherwise plain loads.
  const bool aligned = row_stride % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0;
  const CUtensorMap* tmap = nullptr;
  if (tci || aligned) {
    for (const corr_ctx::MapCache& c : x->map_cache)
      if (c.src == src && c.tci == tci) tmap = &c.map;
    if (!tmap) {
      corr_ctx::MapCache& c = x->map_cache[x->map_next];
      c.src = nullptr;
      if (make_herk_tmap(&c.map, src, tci, x->bits, R, C, T, row_stride, x->rows_per_chan)) {
        c.src = src;
        c.tci = tci;
        tmap = &c.map;
        x->map_next ^= 1;
      }
    }
  }
  const bool use_tma = tmap != nullptr;
  if ((eight || tci) && !use_tma) return CORR_ECUDA;  // these are always TMA-aligned
  const int chunk = eight ? kMaxChunk8 : kMaxChunk4;
  if (int g = guard_acc_write(x, hs)) return g;
  if (pipe) a.grid = device_sm_count() - x->pipe_sms;  // the SMs the next block's turn leaves free
  for (int t0 = 0; t0 < T; t0 += chunk) {
    a.in.t0 = t0;
    a.in.tn = std::min(chunk, T - t0);
    a.in.accumulate = x->acc_live ? 1 : 0;
    a.in.vec_ok = aligned ? 1 : 0;
    cudaEvent_t th = phase_begin(x, hs);
    cudaError_t e = herk4_launch(a, tmap, x->n_tasks, hs, tci);
    if (e != cudaSuccess) return cuda_fail(e);
    phase_end(x, kHerk, th, hs);
    ++x->stats.herk_launches;
    x->acc_live = true;
  }
  ++x->stats.blocks;
  if (pipe) {
    if (cudaEventRecord(x->herk_done[pk], hs) != cudaSuccess) return CORR_ECUDA;
    ++x->pipe_k;
    x->herk_pending = true;
  } else if (slot >= 0 && cudaEventRecord(x->stage_free[slot], x->stream) != cudaSuccess) {
    return CORR_ECUDA;
  }
  return CORR_OK;
}

int corr_push_many(corr_ctx* x, const void* const* blocks, int n_blocks, size_t nbytes,
                   uint64_t seq) {
  TraceRange trace_("corr_push_many");
  if (!x || !blocks || n_blocks < 1 || n_blocks > CORR_MAX_PUSH_MANY) return CORR_EINVAL;
  if (nbytes != x->block_bytes) return CORR_EINVAL;
  for (int i = 0; i < n_blocks; ++i)
    if (!blocks[i]) return CORR_EINVAL;
  const int N = x->n_inputs, C = x->n_chans, T = x->n_time;
  const bool eight = x->bits == 8;
  const int chunk = eight ? kMaxChunk8 : kMaxChunk4;
  const int n_chunks = (T + chunk - 1) / chunk;
  const int n_inst = n_blocks * n_chunks;
  const bool tci = tci_direct(x->layout, x->bits, N);
  // One launch needs blocks the cross-multiply reads in place through TMA:
  // no corner turn, device memory, 16-byte aligned rows.
  // (the task list of the launch stays below 256 MB)
  bool one = n_blocks > 1 && x->pipe_sms == 0 && (tci || !needs_turn(x->layout, x->bits)) &&
             (tci || T % 16 == 0) && n_inst <= CORR_MAX_PUSH_MANY &&
             (long long)x->n_tasks * n_inst * (long long)sizeof(HerkTask) <= (256LL << 20);
  int reuse = -1;
  for (int k = 0; k < 2 && one; ++k) {
    const corr_ctx::ManyTable& t = x->many[k];
    if (t.key_acc == x->acc && (int)t.key.size() == n_blocks &&
        std::equal(t.key.begin(), t.key.end(), blocks))
      reuse = k;  // its blocks were checked when it was filled
  }
  for (int i = 0; i < n_blocks && one && reuse < 0; ++i)
    one = reinterpret_cast<uintptr_t>(blocks[i]) % 16 == 0 && is_device_ptr(blocks[i]);
  if (!one) {  // one push per block: same result, one launch (or more) each
    for (int i = 0; i < n_blocks; ++i) {
      const int st = corr_push(x, blocks[i], nbytes, seq == CORR_SEQ_ANY ? seq : seq + i);
      if (st != CORR_OK) return st;
    }
    return CORR_OK;
  }
  if (seq != CORR_SEQ_ANY && x->seq_started && seq != x->next_seq) {
    ++x->stats.seq_rejects;
    return CORR_ESEQ;
  }
  cudaStream_t hs = x->stream;
  if (int g = guard_acc_write(x, hs)) return g;
  if (x->many_tasks_inst < n_inst) {  // grow the task list (rare: a larger call)
    if (x->many_tasks && (cudaStreamSynchronize(hs) != cudaSuccess || cudaFree(x->many_tasks) != cudaSuccess))
      return CORR_ECUDA;
    x->many_tasks = nullptr;
    x->many_tasks_inst = 0;
    std::vector<HerkTask> all((size_t)n_inst * x->n_tasks);
    for (size_t i = 0; i < all.size(); ++i) {
      all[i] = x->host_tasks[i % x->n_tasks];
      all[i].inst = (int)(i / x->n_tasks);
    }
    if (cudaMalloc(&x->many_tasks, all.size() * sizeof(HerkTask)) != cudaSuccess) return CORR_ENOMEM;
    if (cudaMemcpy(x->many_tasks, all.data(), all.size() * sizeof(HerkTask), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return CORR_ECUDA;
    x->many_tasks_inst = n_inst;
  }
  const int R = eight ? 2 * N : N;
  const long long row_stride = T;
  corr_ctx::ManyTable* tb = reuse >= 0 ? &x->many[reuse] : &x->many[x->many_next];
  if (reuse < 0) {
    x->many_next ^= 1;
    // the launch that last read this table must be done before it changes
    if (tb->used && cudaEventSynchronize(tb->done) != cudaSuccess) return CORR_ECUDA;
    tb->key.clear();
    tb->key_acc = nullptr;
    if (tb->cap < n_inst) {
      cudaFree(tb->d_insts);
      cudaFree(tb->d_maps);
      if (tb->h_insts) cudaFreeHost(tb->h_insts);
      if (tb->h_maps) cudaFreeHost(tb->h_maps);
      tb->d_insts = nullptr, tb->d_maps = nullptr, tb->h_insts = nullptr, tb->h_maps = nullptr;
      tb->cap = 0;
      if (cudaMalloc(&tb->d_insts, (size_t)n_inst * sizeof(HerkInst)) != cudaSuccess ||
          cudaMalloc(&tb->d_maps, (size_t)n_inst * sizeof(CUtensorMap)) != cudaSuccess ||
          cudaMallocHost(&tb->h_insts, (size_t)n_inst * sizeof(HerkInst)) != cudaSuccess ||
          cudaMallocHost(&tb->h_maps, (size_t)n_inst * sizeof(CUtensorMap)) != cudaSuccess)
        return CORR_ENOMEM;
      tb->cap = n_inst;
    }
    if (!tb->done && cudaEventCreateWithFlags(&tb->done, cudaEventDisableTiming) != cudaSuccess) {
      tb->done = nullptr;
      return CORR_ECUDA;
    }
    for (int b = 0; b < n_blocks; ++b) {
      const uint8_t* src = static_cast<const uint8_t*>(blocks[b]);
      CUtensorMap map;
      if (!make_herk_tmap(&map, src, tci, x->bits, R, C, T, row_stride, x->rows_per_chan))
        return CORR_ECUDA;
      for (int c = 0; c < n_chunks; ++c) {
        HerkInst& in = tb->h_insts[b * n_chunks + c];
        memset(&in, 0, sizeof(in));
        in.x = src;
        in.acc = x->acc;
        in.chan_stride = (long long)R * row_stride;
        in.row_stride = row_stride;
        in.n_inputs = N;
        in.n_chans = C;
        in.t0 = c * chunk;
        in.tn = std::min(chunk, T - c * chunk);
        in.rows_per_chan = x->rows_per_chan;
        in.accumulate = 1;  // every block adds (reductions at L2): blocks run concurrently
        in.vec_ok = 1;
        tb->h_maps[b * n_chunks + c] = map;
      }
    }
    if (cudaMemcpyAsync(tb->d_insts, tb->h_insts, (size_t)n_inst * sizeof(HerkInst),
                        cudaMemcpyHostToDevice, hs) != cudaSuccess ||
        cudaMemcpyAsync(tb->d_maps, tb->h_maps, (size_t)n_inst * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice, hs) != cudaSuccess)
      return CORR_ECUDA;
    tb->key.assign(blocks, blocks + n_blocks);
    tb->key_acc = x->acc;
  }
  // a new integration starts from zero, since no block stores
  if (!x->acc_live && cudaMemsetAsync(x->acc, 0, x->acc_bytes, hs) != cudaSuccess)
    return CORR_ECUDA;
  HerkArgs a;
  memset(&a, 0, sizeof(a));
  a.in = tb->h_insts[0];
  a.insts = tb->d_insts;
  a.tmaps = tb->d_maps;
  a.tasks = x->many_tasks;
  a.n_tasks = x->n_tasks * n_inst;
  a.status = x->d_status;
  a.lo_is_real = (x->flags & CORR_F_LO_IS_REAL) ? 1 : 0;
  a.smem_bytes = x->smem_bytes;
  a.bits = x->bits;
  a.scratch = x->scratch;
  a.scratch_ctas = x->scratch_ctas;
  cudaEvent_t th = phase_begin(x, hs);
  cudaError_t e = herk4_launch(a, nullptr, a.n_tasks, hs, tci);
  if (e != cudaSuccess) return cuda_fail(e);
  phase_end(x, kHerk, th, hs);
  if (cudaEventRecord(tb->done, hs) != cudaSuccess) return CORR_ECUDA;
  tb->used = true;
  ++x->stats.herk_launches;
  x->stats.blocks += (uint64_t)n_blocks;
  x->acc_live = true;
  if (seq != CORR_SEQ_ANY) {
    x->seq_started = true;
    x->next_seq = seq + (uint64_t)n_blocks;
  }
  return CORR_OK;
}

int corr_set_pipeline(corr_ctx* x, int turn_sms) {
  if (!x || turn_sms < 0) return CORR_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CORR_ECUDA;
  if (turn_sms >= nsm) return CORR_EINVAL;
  if (turn_sms > 0 && !turn_can_persist(x->layout, x->bits)) return CORR_EINVAL;
  // switch between modes only with nothing in flight
  if (pipe_join(x) != CORR_OK || cudaStreamSynchronize(x->stream) != cudaSuccess ||
      cudaStreamSynchronize(x->copy_stream) != cudaSuccess)
    return CORR_ECUDA;
  if (turn_sms > 0) {  // create what is missing (a failed earlier call may have left some)
    for (cudaStream_t* st : {&x->turn_stream, &x->herk_stream})
      if (!*st && cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) != cudaSuccess) {
        *st = nullptr;
        return CORR_ECUDA;
      }
    for (cudaEvent_t* e : {&x->ev_in[0], &x->ev_in[1], &x->turn_done[0], &x->turn_done[1],
                           &x->herk_done[0], &x->herk_done[1], &x->herk_last})
      if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
        *e = nullptr;
        return CORR_ECUDA;
      }
  }
  if (turn_sms > 0 && !x->turned_buf[1]) {  // (also retried after an earlier failure)
    const int byte_rows = x->n_inputs * (x->bits / 4);
    if (cudaMalloc(&x->turned_buf[1], (size_t)x->turned_stride * byte_rows * x->n_chans) !=
        cudaSuccess) {
      x->turned_buf[1] = nullptr;
      return CORR_ENOMEM;
    }
  }
  x->pipe_sms = turn_sms;
  x->pipe_k = 0;
  return CORR_OK;
}

int corr_sync(corr_ctx* x) {
  if (!x) return CORR_EINVAL;
  if (pipe_join(x) != CORR_OK) return CORR_ECUDA;
  if (cudaStreamSynchronize(x->copy_stream) != cudaSuccess) return CORR_ECUDA;
  if (x->dump_stream && cudaStreamSynchronize(x->dump_stream) != cudaSuccess) return CORR_ECUDA;
  return take_status(x);
}

int corr_dump_async(corr_ctx* x, int64_t* vis, int reset) {
  TraceRange trace_("corr_dump_async");
  if (!x || !vis) return CORR_EINVAL;
  if ((int)x->dumps.size() >= CORR_MAX_ASYNC_DUMPS) return CORR_EBUSY;
  // everything below is ordered after the last cross-multiply on its own
  // stream, so that the caller's stream (and the next block's corner turn)
  // does not wait for it
  cudaStream_t as = acc_stream(x);
  // first use: create what is missing (a failed earlier call may have left some)
  if (!x->dump_stream && cudaStreamCreateWithFlags(&x->dump_stream, cudaStreamNonBlocking) != cudaSuccess) {
    x->dump_stream = nullptr;
    return CORR_ECUDA;
  }
  for (int i = 0; i < 2; ++i)
    if (!x->acc_free[i] && cudaEventCreateWithFlags(&x->acc_free[i], cudaEventDisableTiming) != cudaSuccess) {
      x->acc_free[i] = nullptr;
      return CORR_ECUDA;
    }
  if (!x->h_dump_status) {
    if (cudaHostAlloc(&x->h_dump_status, CORR_MAX_ASYNC_DUMPS * sizeof(int), cudaHostAllocMapped) !=
        cudaSuccess) {
      x->h_dump_status = nullptr;
      return CORR_ENOMEM;
    }
    if (cudaHostGetDevicePointer(&x->d_dump_status, x->h_dump_status, 0) != cudaSuccess) {
      cudaFreeHost(x->h_dump_status);
      x->h_dump_status = nullptr;
      return CORR_ECUDA;
    }
  }
  if (reset && !x->acc_buf[1] && cudaMalloc(&x->acc_buf[1], x->acc_bytes) != cudaSuccess)
    return CORR_ENOMEM;
  if (!x->acc_live) {  // nothing pushed since the last reset: an all-zero integration
    if (int g = guard_acc_write(x, as)) return g;
    if (cudaMemsetAsync(x->acc, 0, x->acc_bytes, as) != cudaSuccess) return CORR_ECUDA;
    x->acc_live = true;
  }
  // a status slot no outstanding dump uses
  int slot = 0;
  while (std::any_of(x->dumps.begin(), x->dumps.end(),
                     [slot](const corr_ctx::AsyncDump& d) { return d.slot == slot; }))
    ++slot;
  // snapshot and clear the status of the blocks in this integration, in
  // stream order, then hand the accumulator to the dump stream
  if (!x->dump_ready && cudaEventCreateWithFlags(&x->dump_ready, cudaEventDisableTiming) != cudaSuccess) {
    x->dump_ready = nullptr;
    return CORR_ECUDA;
  }
  cudaEvent_t ready = x->dump_ready, done = nullptr;
  if (!x->done_pool.empty()) {
    done = x->done_pool.back();
    x->done_pool.pop_back();
  } else if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
    return CORR_ECUDA;
  }
  int st = CORR_OK;
  if (take_status_launch(x->d_status, x->d_dump_status + slot, as) != cudaSuccess ||
      cudaEventRecord(ready, as) != cudaSuccess ||
      cudaStreamWaitEvent(x->dump_stream, ready, 0) != cudaSuccess)
    st = CORR_ECUDA;
  // a buffer bound with corr_bind already holds the sums: nothing to copy
  const bool copy = vis != x->acc;
  if (st == CORR_OK && copy) {
    cudaEvent_t td = phase_begin(x, x->dump_stream);
    if (cudaMemcpyAsync(vis, x->acc, x->acc_bytes, cudaMemcpyDefault, x->dump_stream) != cudaSuccess ||
        cudaEventRecord(x->acc_free[x->cur], x->dump_stream) != cudaSuccess)
      st = CORR_ECUDA;
    else
      phase_end(x, kDump, td, x->dump_stream);
  }
  if (st == CORR_OK && cudaEventRecord(done, x->dump_stream) != cudaSuccess) st = CORR_ECUDA;
  if (st != CORR_OK) {
    cudaEventDestroy(done);  // its last record may still be pending: not reused
    return st;
  }
  if (copy) x->read_pending[x->cur] = true;
  x->dumps.push_back({done, slot});
  ++x->stats.dumps;
  if (reset) {
    if (x->bound) {  // the context's own accumulator was not used
      unbind(x);
    } else {
      x->cur ^= 1;
      x->acc = x->acc_buf[x->cur];
    }
    x->acc_live = false;
    x->seq_started = false;
  }
  return CORR_OK;
}

int corr_dump_wait(corr_ctx* x) {
  TraceRange trace_("corr_dump_wait");
  if (!x) return CORR_EINVAL;
  if (x->dumps.empty()) return CORR_ESTATE;
  const corr_ctx::AsyncDump d = x->dumps.front();
  x->dumps.erase(x->dumps.begin());
  const cudaError_t e = cudaEventSynchronize(d.done);
  if (e != cudaSuccess) {
    cudaEventDestroy(d.done);
    return CORR_ECUDA;
  }
  x->done_pool.push_back(d.done);
  return status_code(x->h_dump_status[d.slot]);
}

int corr_dump(corr_ctx* x, int64_t* vis, int reset) {
  TraceRange trace_("corr_dump");
  if (!x) return CORR_EINVAL;
  if (pipe_join(x) != CORR_OK) return CORR_ECUDA;
  if (vis) {
    const bool dev = is_device_ptr(vis);
    if (x->acc_live) {
      if (vis != x->acc) {  // a bound buffer already holds the sums
        cudaEvent_t td = phase_begin(x, x->stream);
        if (cudaMemcpyAsync(vis, x->acc, x->acc_bytes, cudaMemcpyDefault, x->stream) != cudaSuccess)
          return CORR_ECUDA;
        phase_end(x, kDump, td, x->stream);
      }
    } else if (dev) {
      if (cudaMemsetAsync(vis, 0, x->acc_bytes, x->stream) != cudaSuccess) return CORR_ECUDA;
    } else {
      if (cudaStreamSynchronize(x->stream) != cudaSuccess) return CORR_ECUDA;
      memset(vis, 0, x->acc_bytes);
    }
  }
  ++x->stats.dumps;
  const int st = take_status(x);
  if (reset) {
    x->acc_live = false;
    x->seq_started = false;
    unbind(x);
  }
  return st;
}

int corr_bind(corr_ctx* x, int64_t* vis) {
  TraceRange trace_("corr_bind");
  if (!x || !vis || !is_device_ptr(vis)) return CORR_EINVAL;
  if (x->acc_live) return CORR_ESTATE;  // blocks already went into this integration
  x->bound = vis;
  x->acc = vis;
  return CORR_OK;
}

int corr_restore(corr_ctx* x, const int64_t* vis) {
  TraceRange trace_("corr_restore");
  if (!x || !vis) return CORR_EINVAL;
  if (pipe_join(x) != CORR_OK) return CORR_ECUDA;
  if (int g = guard_acc_write(x, x->stream)) return g;
  if (cudaMemcpyAsync(x->acc, vis, x->acc_bytes, cudaMemcpyDefault, x->stream) != cudaSuccess ||
      cudaStreamSynchronize(x->stream) != cudaSuccess)
    return CORR_ECUDA;
  x->acc_live = true;
  x->seq_started = false;
  return CORR_OK;
}

int corr_normalise(corr_ctx* x, double* rho) { return corr_normalise_flags(x, rho, nullptr); }

int corr_normalise_flags(corr_ctx* x, double* rho, uint8_t* zero_flag) {
  TraceRange trace_("corr_normalise");
  if (!x || !rho) return CORR_EINVAL;
  if (pipe_join(x) != CORR_OK) return CORR_ECUDA;
  const size_t bytes = x->acc_bytes;  // same element count, 8-byte elements
  const size_t flag_bytes = bytes / 16;  // one byte per baseline and channel
  if (!x->acc_live) {
    if (int g = guard_acc_write(x, x->stream)) return g;
    if (cudaMemsetAsync(x->acc, 0, x->acc_bytes, x->stream) != cudaSuccess) return CORR_ECUDA;
    x->acc_live = true;
  }
  const bool dev = is_device_ptr(rho);
  double* d = rho;
  if (!dev) {
    if (!x->rho_tmp && cudaMalloc(&x->rho_tmp, bytes) != cudaSuccess) return CORR_ENOMEM;
    d = x->rho_tmp;
  }
  const bool fdev = zero_flag && is_device_ptr(zero_flag);
  uint8_t* f = zero_flag;
  if (zero_flag && !fdev) {
    if (!x->flag_tmp && cudaMalloc(&x->flag_tmp, flag_bytes) != cudaSuccess) return CORR_ENOMEM;
    f = x->flag_tmp;
  }
  cudaEvent_t tn = phase_begin(x, x->stream);
  cudaError_t e = normalise_launch(x->acc, d, f, x->n_inputs, x->n_chans, x->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  phase_end(x, kNorm, tn, x->stream);
  ++x->stats.norm_launches;
  if (!dev && cudaMemcpyAsync(rho, d, bytes, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess)
    return CORR_ECUDA;
  if (zero_flag && !fdev &&
      cudaMemcpyAsync(zero_flag, f, flag_bytes, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess)
    return CORR_ECUDA;
  return take_status(x);
}

int corr_set_fault_injection(corr_ctx* x, int stage, int wait_log2) {
  if (!x || stage < -1 || stage >= (1 << 24) - 1 || wait_log2 < 0 || wait_log2 > 40)
    return CORR_EINVAL;
  if (pipe_join(x) != CORR_OK) return CORR_ECUDA;
  x->fault = (stage + 1) | (wait_log2 << 24);
  return CORR_OK;
}

int corr_set_timing(corr_ctx* x, int on) {
  if (!x) return CORR_EINVAL;
  x->timing = on != 0;
  return CORR_OK;
}

int corr_get_stats(corr_ctx* x, corr_stats* out) {
  if (!x || !out) return CORR_EINVAL;
  if (cudaStreamSynchronize(x->copy_stream) != cudaSuccess ||
      cudaStreamSynchronize(x->stream) != cudaSuccess)
    return CORR_ECUDA;
  collect_timings(x);
  *out = x->stats;
  return CORR_OK;
}

int corr_destroy(corr_ctx* x) {
  if (!x) return CORR_OK;
  free_ctx(x);
  return CORR_OK;
}

}  // extern "C"
