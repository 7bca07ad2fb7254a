// corr_correlate_noalloc: one block through the corner turn and the
// cross-multiply into caller-provided visibilities without allocating.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that another framework owns, processes whose allocations are
// frozen after start-up, or real-time loops where a cudaMalloc could stall
// the stream.  For them this entry point keeps every intermediate -- the task
// list, the status word and the corner-turned copy of the block -- in one
// fixed file-scope device array instead of buffers from cudaMalloc.  The
// array occupies kNoAllocScratchBytes on every device that loads the library
// until the process exits.
#include <algorithm>
#include <mutex>

#include "xe_internal.h"
#include "xengine.h"

namespace xe {
namespace {

constexpr size_t kNoAllocScratchBytes = CORR_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch.  Host code must not use this name as an address: on
// the host it is only a stand-in, so the device address is looked up with
// cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call for that device).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CORR_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CORR_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CORR_OK;
}

// Tasks per channel of the lower-triangle tiling (same tiling as the
// context path): row block r takes column blocks r .. r + ceil(nrb/2) - 1
// (mod nrb), plus r + nrb/2 for r < nrb/2 when nrb is even; the first two
// share a task, every further column is a task of its own.
__host__ __device__ inline int row_cols(int nrb, int r) {
  int n = (nrb + 1) / 2;
  if (nrb % 2 == 0 && r < nrb / 2) ++n;
  return n;
}
__host__ __device__ inline int row_col(int nrb, int r, int k) {
  const int base = (nrb + 1) / 2;
  return k < base ? (r + k) % nrb : r + nrb / 2;
}

// Task e of the list: the 128 x 256 tasks (first two columns of a row) of
// every channel come first, then the single-column tasks, the order the
// context path's planner uses.  pairs / singles: tasks of each kind per channel.
__global__ void plan_kernel(HerkTask* tasks, long long n_tasks, int rpc, int pairs, int singles,
                            int n_chans, int nrb) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_tasks;
       e += (long long)gridDim.x * blockDim.x) {
    HerkTask t;
    t.inst = 0;
    if (rpc > 0) {
      t.chan0 = (int)(e * (128 / rpc));
      t.rb = 0;
      t.cb[0] = 0;
      t.cb[1] = -1;
    } else if (e < (long long)n_chans * pairs) {
      t.chan0 = (int)(e / pairs);
      int local = (int)(e % pairs), r = 0;
      for (; r < nrb; ++r) {
        if (row_cols(nrb, r) < 2) continue;
        if (local == 0) break;
        --local;
      }
      t.rb = r;
      t.cb[0] = row_col(nrb, r, 0);
      t.cb[1] = row_col(nrb, r, 1);
    } else {
      const long long e2 = e - (long long)n_chans * pairs;
      t.chan0 = (int)(e2 / singles);
      int local = (int)(e2 % singles), r = 0, k = 0;
      for (; r < nrb; ++r) {
        const int ncol = row_cols(nrb, r);
        const int first = ncol > 1 ? 2 : 0;  // columns of this row in single-column tasks
        if (local < ncol - first) {
          k = first + local;
          break;
        }
        local -= ncol - first;
      }
      t.rb = r;
      t.cb[0] = row_col(nrb, r, k);
      t.cb[1] = -1;
    }
    tasks[e] = t;
  }
}

__global__ void copy_status_kernel(const int* from, int* to) { *to = *from; }

// Device (or managed) memory of the current device.  Memory of another GPU
// would be read and written by this device's kernels: rejected.
bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev;
  return at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace xe

using namespace xe;

extern "C" int corr_correlate_noalloc_bits(const void* block, int n_inputs, int n_chans,
                                           int n_time, int bits, int layout, unsigned flags,
                                           int64_t* vis, int* status, void* stream) {
  TraceRange trace_("corr_correlate_noalloc");
  if (!block || !vis || n_inputs < 1 || n_inputs > 1024 || n_chans < 1 || n_time < 1 ||
      (bits != 4 && bits != 8) || layout < CORR_L_TCI || layout > CORR_L_CIT ||
      (flags & ~CORR_F_LO_IS_REAL) || (bits == 8 && (flags & CORR_F_LO_IS_REAL)))
    return CORR_EINVAL;
  if (!is_device(block) || !is_device(vis) || (status && !is_device(status))) return CORR_EINVAL;
  const int N = n_inputs, C = n_chans, T = n_time;
  const bool eight = bits == 8;
  const int R = eight ? 2 * N : N;  // byte rows per channel
  // scratch layout: [status (256 B)] [tasks] [8-bit partial sums] [corner-turned block]
  int rpc = 0, pairs = 0, singles = 0, nrb = 0;
  long long n_tasks;
  if (2 * N <= 64) {
    rpc = 2;
    while (rpc < 2 * N) rpc <<= 1;
    n_tasks = ((long long)C + 128 / rpc - 1) / (128 / rpc);
  } else {
    nrb = (2 * N + 127) / 128;
    for (int r = 0; r < nrb; ++r) {
      const int ncol = row_cols(nrb, r);
      pairs += ncol > 1 ? 1 : 0;
      singles += ncol > 1 ? ncol - 2 : 1;
    }
    n_tasks = (long long)(pairs + singles) * C;
  }
  const long long task_bytes = (n_tasks * (long long)sizeof(HerkTask) + 255) / 256 * 256;
  // payload-order blocks whose rows suit TMA are read in place; other
  // layouts (and 8-bit [c][i][t], whose byte pairs split into rows) are turned
  const bool tci = tci_direct(layout, bits, N) && reinterpret_cast<uintptr_t>(block) % 16 == 0;
  const bool turn = !tci && needs_turn(layout, bits);
  // turned rows padded to 32 bytes: the corner turn's fast path, as in corr_create
  const long long row_stride = turn ? ((long long)T + 31) / 32 * 32 : T;
  const long long turned_bytes = turn ? row_stride * R * C : 0;
  const int n_sm = device_sm_count();
  const long long scr_bytes = eight ? (long long)n_sm * kHerkScratchInt2 * (long long)sizeof(int2) : 0;
  if (256 + task_bytes + scr_bytes + turned_bytes > (long long)kNoAllocScratchBytes) return CORR_EINVAL;
  // the cross-multiply needs four ring slots of its largest stage (as corr_create checks)
  const int smem = herk4_max_smem();
  if (smem < 4 * 2 * (16384 + 8192) + 1024) return CORR_ECUDA;
  void* base = nullptr;
  int st = scratch_address(&base);
  if (st != CORR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* b8 = static_cast<uint8_t*>(base);
  int* d_status = reinterpret_cast<int*>(b8);
  HerkTask* tasks = reinterpret_cast<HerkTask*>(b8 + 256);
  int2* scr = reinterpret_cast<int2*>(b8 + 256 + task_bytes);
  uint8_t* turned = b8 + 256 + task_bytes + scr_bytes;

  // the scratch keeps the previous call's contents: clear the status word
  if (cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess) return CORR_ECUDA;
  const int pblocks = (int)std::min<long long>((n_tasks + 255) / 256, 1024);
  plan_kernel<<<pblocks, 256, 0, s>>>(tasks, n_tasks, rpc, pairs, singles, C, nrb);
  if (cudaGetLastError() != cudaSuccess) return CORR_ECUDA;

  const uint8_t* src = static_cast<const uint8_t*>(block);
  if (turn) {
    if (turn_rows(src, turned, layout, bits, N, C, T, row_stride, s) != cudaSuccess) return CORR_ECUDA;
    src = turned;
  }
  HerkArgs a{};
  a.in.x = src;
  a.in.acc = vis;
  a.tasks = tasks;
  a.status = d_status;
  a.in.chan_stride = (long long)R * row_stride;
  a.in.row_stride = row_stride;
  a.in.n_inputs = N;
  a.in.n_chans = C;
  a.in.rows_per_chan = rpc;
  a.lo_is_real = (flags & CORR_F_LO_IS_REAL) ? 1 : 0;
  a.smem_bytes = smem;
  a.n_tasks = (int)n_tasks;
  a.bits = bits;
  a.scratch = eight ? scr : nullptr;
  a.scratch_ctas = eight ? n_sm : 0;
  CUtensorMap tmap;
  const bool aligned = row_stride % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0;
  const bool use_tma =
      (tci || aligned) && make_herk_tmap(&tmap, src, tci, bits, R, C, T, row_stride, rpc);
  if ((eight || tci) && !use_tma) return CORR_ECUDA;  // these read through TMA only
  const int chunk = eight ? kMaxChunk8 : kMaxChunk4;
  for (int t0 = 0; t0 < T; t0 += chunk) {
    a.in.t0 = t0;
    a.in.tn = std::min(chunk, T - t0);
    a.in.accumulate = t0 > 0 ? 1 : 0;
    a.in.vec_ok = aligned ? 1 : 0;
    if (herk4_launch(a, use_tma ? &tmap : nullptr, (int)n_tasks, s, tci) != cudaSuccess)
      return CORR_ECUDA;
  }
  if (status) {
    copy_status_kernel<<<1, 1, 0, s>>>(d_status, status);
    if (cudaGetLastError() != cudaSuccess) return CORR_ECUDA;
  }
  return CORR_OK;
}

extern "C" int corr_correlate_noalloc(const void* block, int n_inputs, int n_chans, int n_time,
                                      int layout, unsigned flags, int64_t* vis, int* status,
                                      void* stream) {
  return corr_correlate_noalloc_bits(block, n_inputs, n_chans, n_time, 4, layout, flags, vis,
                                     status, stream);
}
