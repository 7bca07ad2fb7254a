// C ABI of the X-engine (declared in include/xengine.h): context lifetime,
// ingest staging, corner turn, the tensor-core cross-multiply, integration
// state and dumps.  Every step of the data path runs in this library's
// kernels on the context's stream.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "xe_internal.h"
#include "xengine.h"

using namespace xe;

struct corr_ctx {
  int n_inputs = 0, n_chans = 0, n_time = 0, bits = 4, layout = 0;
  unsigned flags = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t copy_stream = nullptr;
  size_t block_bytes = 0;
  int64_t* acc = nullptr;  // int64 [C][B][2] long integration
  size_t acc_bytes = 0;
  bool acc_live = false;   // false: next push stores instead of adding
  uint8_t* stage[2] = {nullptr, nullptr};
  cudaEvent_t stage_free[2] = {nullptr, nullptr};
  cudaEvent_t stage_ready[2] = {nullptr, nullptr};
  int stage_next = 0;
  uint8_t* turned = nullptr;  // corner-turned copy of the block, [c][i][t]
  HerkTask* tasks = nullptr;
  int n_tasks = 0;
  int rows_per_chan = 0;
  int smem_bytes = 0;
  int* d_status = nullptr;
  int* h_status = nullptr;  // pinned
  double* rho_tmp = nullptr;
  bool seq_started = false;
  uint64_t next_seq = 0;
};

namespace {

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

// Tasks of the lower-triangle tiling of the real Gram matrix (see
// HerkTask), ordered by decreasing work so that large tasks start first.
std::vector<HerkTask> plan_tasks(int n, int c, int* rows_per_chan) {
  std::vector<HerkTask> t;
  const int rows = 2 * n;
  if (rows <= 64) {
    int rpc = 2;
    while (rpc < rows) rpc <<= 1;
    *rows_per_chan = rpc;
    const int per = 128 / rpc;
    for (int c0 = 0; c0 < c; c0 += per) t.push_back({c0, 0, 0, 1});
    return t;
  }
  *rows_per_chan = 0;
  const int nrb = (rows + 127) / 128;
  for (int ch = 0; ch < c; ++ch)
    for (int rb = 0; rb < nrb; ++rb) {
      int cb = 0;
      while (cb <= rb) {
        if (rb - cb + 1 <= 4) {
          t.push_back({ch, rb, cb, rb + 1});
          cb = rb + 1;
        } else {
          t.push_back({ch, rb, cb, cb + 3});
          cb += 3;
        }
      }
    }
  std::stable_sort(t.begin(), t.end(), [](const HerkTask& x, const HerkTask& y) {
    const int wx = x.cb1 - x.cb0, wy = y.cb1 - y.cb0;
    return wx > wy;
  });
  return t;
}

void free_ctx(corr_ctx* x) {
  if (!x) return;
  if (x->stream) cudaStreamSynchronize(x->stream);
  if (x->copy_stream) cudaStreamSynchronize(x->copy_stream);
  cudaFree(x->acc);
  for (int i = 0; i < 2; ++i) {
    cudaFree(x->stage[i]);
    if (x->stage_free[i]) cudaEventDestroy(x->stage_free[i]);
    if (x->stage_ready[i]) cudaEventDestroy(x->stage_ready[i]);
  }
  cudaFree(x->turned);
  cudaFree(x->tasks);
  cudaFree(x->d_status);
  cudaFree(x->rho_tmp);
  if (x->h_status) cudaFreeHost(x->h_status);
  if (x->copy_stream) cudaStreamDestroy(x->copy_stream);
  if (x->own_stream && x->stream) cudaStreamDestroy(x->stream);
  delete x;
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
  if (st & kStTimeout) return CORR_ETIMEDOUT;
  if (st & kStRange) return CORR_ERANGE;
  return CORR_ECUDA;
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
  if (n_inputs < 1 || n_inputs > 1024 || n_chans < 1 || n_time < 1 || bits != 4 ||
      layout < CORR_L_TCI || layout > CORR_L_CIT || (flags & ~CORR_F_LO_IS_REAL))
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
    if (cudaMalloc(&x->acc, x->acc_bytes) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (layout != CORR_L_CIT && cudaMalloc(&x->turned, block_bytes) != cudaSuccess) { st = CORR_ENOMEM; break; }
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
    if (cudaMalloc(&x->tasks, tasks.size() * sizeof(HerkTask)) != cudaSuccess) { st = CORR_ENOMEM; break; }
    if (cudaMemcpy(x->tasks, tasks.data(), tasks.size() * sizeof(HerkTask), cudaMemcpyHostToDevice) != cudaSuccess) { st = CORR_ECUDA; break; }
    x->smem_bytes = herk4_max_smem();
    if (x->smem_bytes < 2 * 4 * 128 * 128 + 1024) { st = CORR_ECUDA; break; }
  } while (0);
  if (st != CORR_OK) {
    free_ctx(x);
    return st;
  }
  *out = x;
  return CORR_OK;
}

int corr_push(corr_ctx* x, const void* block, size_t nbytes, uint64_t seq) {
  if (!x || !block) return CORR_EINVAL;
  if (nbytes != x->block_bytes) return CORR_EINVAL;
  if (seq != CORR_SEQ_ANY) {
    if (x->seq_started && seq != x->next_seq) return CORR_ESEQ;
    x->seq_started = true;
    x->next_seq = seq + 1;
  }
  const uint8_t* src = static_cast<const uint8_t*>(block);
  int slot = -1;
  if (!is_device_ptr(block)) {
    slot = x->stage_next;
    x->stage_next ^= 1;
    if (!x->stage[slot] && cudaMalloc(&x->stage[slot], x->block_bytes) != cudaSuccess)
      return CORR_ENOMEM;
    if (cudaStreamWaitEvent(x->copy_stream, x->stage_free[slot], 0) != cudaSuccess ||
        cudaMemcpyAsync(x->stage[slot], block, nbytes, cudaMemcpyHostToDevice, x->copy_stream) !=
            cudaSuccess ||
        cudaEventRecord(x->stage_ready[slot], x->copy_stream) != cudaSuccess ||
        cudaStreamWaitEvent(x->stream, x->stage_ready[slot], 0) != cudaSuccess)
      return CORR_ECUDA;
    src = x->stage[slot];
  }
  const int N = x->n_inputs, C = x->n_chans, T = x->n_time;
  if (x->layout == CORR_L_TCI) {
    // [t][c][i] -> [c][i][t]: one transpose of a T x (C N) byte matrix
    cudaError_t e = turn_launch(src, x->turned, T, 1, C * N, x->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    src = x->turned;
  } else if (x->layout == CORR_L_TIC) {
    // [t][i][c] -> [c][i][t]
    cudaError_t e = turn_launch(src, x->turned, T, N, C, x->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    src = x->turned;
  }
  HerkArgs a;
  memset(&a, 0, sizeof(a));
  a.x = src;
  a.acc = x->acc;
  a.tasks = x->tasks;
  a.status = x->d_status;
  a.chan_stride = (long long)N * T;
  a.row_stride = T;
  a.n_inputs = N;
  a.n_chans = C;
  a.rows_per_chan = x->rows_per_chan;
  a.lo_is_real = (x->flags & CORR_F_LO_IS_REAL) ? 1 : 0;
  a.smem_bytes = x->smem_bytes;
  for (int t0 = 0; t0 < T; t0 += kMaxChunk4) {
    a.t0 = t0;
    a.tn = std::min(kMaxChunk4, T - t0);
    a.accumulate = x->acc_live ? 1 : 0;
    a.vec_ok = (T % 16 == 0) && (t0 % 16 == 0) && (reinterpret_cast<uintptr_t>(src) % 16 == 0);
    cudaError_t e = herk4_launch(a, x->n_tasks, x->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    x->acc_live = true;
  }
  if (slot >= 0 && cudaEventRecord(x->stage_free[slot], x->stream) != cudaSuccess)
    return CORR_ECUDA;
  return CORR_OK;
}

int corr_sync(corr_ctx* x) {
  if (!x) return CORR_EINVAL;
  if (cudaStreamSynchronize(x->copy_stream) != cudaSuccess) return CORR_ECUDA;
  return take_status(x);
}

int corr_dump(corr_ctx* x, int64_t* vis, int reset) {
  if (!x) return CORR_EINVAL;
  if (vis) {
    const bool dev = is_device_ptr(vis);
    if (x->acc_live) {
      if (cudaMemcpyAsync(vis, x->acc, x->acc_bytes, cudaMemcpyDefault, x->stream) != cudaSuccess)
        return CORR_ECUDA;
    } else if (dev) {
      if (cudaMemsetAsync(vis, 0, x->acc_bytes, x->stream) != cudaSuccess) return CORR_ECUDA;
    } else {
      if (cudaStreamSynchronize(x->stream) != cudaSuccess) return CORR_ECUDA;
      memset(vis, 0, x->acc_bytes);
    }
  }
  const int st = take_status(x);
  if (reset) {
    x->acc_live = false;
    x->seq_started = false;
  }
  return st;
}

int corr_normalise(corr_ctx* x, double* rho) {
  if (!x || !rho) return CORR_EINVAL;
  const size_t bytes = x->acc_bytes;  // same element count, 8-byte elements
  if (!x->acc_live) {
    if (cudaMemsetAsync(x->acc, 0, x->acc_bytes, x->stream) != cudaSuccess) return CORR_ECUDA;
    x->acc_live = true;
  }
  const bool dev = is_device_ptr(rho);
  double* d = rho;
  if (!dev) {
    if (!x->rho_tmp && cudaMalloc(&x->rho_tmp, bytes) != cudaSuccess) return CORR_ENOMEM;
    d = x->rho_tmp;
  }
  cudaError_t e = normalise_launch(x->acc, d, x->n_inputs, x->n_chans, x->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!dev && cudaMemcpyAsync(rho, d, bytes, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess)
    return CORR_ECUDA;
  return take_status(x);
}

int corr_destroy(corr_ctx* x) {
  if (!x) return CORR_OK;
  free_ctx(x);
  return CORR_OK;
}

}  // extern "C"
