// X-engine cross-multiply-and-accumulate (Sec. 2 "CMAC"; Sec. 2.2) for
// 4-bit complex samples on sm_103a tensor cores.
//
// Per channel, V_ij = sum_t x_i(t) conj(x_j(t)) for i >= j.  With Y the
// real (2N x T) matrix whose row 2i is Re x_i and row 2i+1 is Im x_i, and
// G = Y Y^T, the visibilities are
//     Re V_ij = G[2i][2j] + G[2i+1][2j+1],   Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// The kernel forms the lower-triangle 128 x 128 tiles of G with
// tcgen05.mma kind::f8f6f4 (E4M3 operands, FP32 accumulators in tensor
// memory).
//
// Operand encoding.  A 4-bit two's-complement nibble n (value v in -8..7)
// is fed to the tensor core as the offset code u = n ^ 8 = v + 8 in 0..15.
// The E4M3 byte with bit pattern u (exponent field 0 or 1) has the value
// u * 2^-9 exactly, so unpacking a byte of two nibbles into two E4M3 bytes is
// one mask and one XOR.  The tensor core then accumulates
//     Gu[p][q] = 2^-18 sum_t u_p u_q,
// exact in FP32 while the integer sum stays below 2^24 (at most 225 per
// spectrum, so up to 65536 spectra per accumulation).  The signed Gram
// follows from the row sums U_p = sum_t u_p:
//     G[p][q] = sum (u_p - 8)(u_q - 8) = 2^18 Gu[p][q] - 8 U_p - 8 U_q + 64 T.
// Padded spectra and padded rows use u = 0 and drop out of every term.
//
// Roles in one CTA (one task = one 128-row block of G of one channel, or of
// several stacked small channels, against up to four 128-column blocks):
//   warps 0-3  load packed bytes from HBM (16-byte streaming loads), unpack
//              them into the 128-byte-swizzled K-major operand layout in
//              shared memory, and keep the row sums; afterwards they drain
//              the tensor-memory accumulators, apply the correction, fold the
//              2 x 2 real blocks into complex visibilities and add them into
//              the int64 integration buffer.
//   warp 4     one thread issues the MMAs stage by stage.
#include <cstdio>

#include "xe_device.cuh"

namespace xe {
namespace {

constexpr int kThreads = 160;
constexpr int kProducers = 128;
constexpr int kMaxStages = 8;
constexpr int kMaxBlocks = 4;                 // 128-row operand blocks per stage
constexpr int kStageT = 128;                  // spectra per stage = one swizzle row
constexpr int kBlockBytes = 128 * kStageT;    // one 128-row block of one stage
constexpr int kMaxItems = kMaxBlocks * 4;     // 16-byte items per producer thread per stage

struct Shared {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
  int32_t usum[kMaxBlocks * 128];
};

__device__ __forceinline__ void raise_timeout(int* status, volatile int* abort) {
  *abort = 1;
  atomicOr(status, kStTimeout);
}

__device__ __forceinline__ uint32_t swz_offset(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

__global__ void __launch_bounds__(kThreads, 1) herk4_kernel(const HerkArgs a) {
  extern __shared__ uint8_t dyn_raw[];
  __shared__ Shared sm;
  uint8_t* ops = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_raw) + 1023) &
                                            ~static_cast<uintptr_t>(1023));
  const HerkTask task = a.tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool stacked = a.rows_per_chan > 0;
  const int nb = task.cb1 - task.cb0;
  const bool a_sep = task.rb >= task.cb1;
  const int nblk = nb + (a_sep ? 1 : 0);
  const int a_slot = a_sep ? nb : task.rb - task.cb0;
  const int stage_bytes = nblk * kBlockBytes;
  int nst = (a.smem_bytes - 1024) / stage_bytes;
  if (nst > kMaxStages) nst = kMaxStages;
  const int nk = (a.tn + kStageT - 1) / kStageT;
  const uint32_t ncols = nb <= 1 ? 128u : (nb == 2 ? 256u : 512u);
  volatile int* abort = &sm.abort;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&sm.full[s], kProducers);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.done, 1);
    sm.abort = 0;
  }
  if (warp == 0) tmem_alloc(&sm.tmem_base, ncols);
  fence_mbar_init();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 4) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id256 = umma_idesc(0, 128, 256), id128 = umma_idesc(0, 128, 128);
      const uint32_t ops_addr = smem_addr(ops);
      for (int k = 0; k < nk; ++k) {
        const int s = k % nst;
        if (!mbar_wait(&sm.full[s], (uint32_t)(k / nst) & 1u, abort)) {
          raise_timeout(a.status, abort);
          break;
        }
        tc_after_sync();
        const uint32_t st = ops_addr + (uint32_t)(s * stage_bytes);
        const uint64_t adesc = umma_desc_sw128(st + (uint32_t)(a_slot * kBlockBytes));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          for (int n0 = 0; n0 < nb; n0 += 2) {
            const bool wide = nb - n0 >= 2;
            const uint64_t bdesc = umma_desc_sw128(st + (uint32_t)(n0 * kBlockBytes));
            umma_f8(tmem + (uint32_t)(n0 * 128), adesc + 2 * kk, bdesc + 2 * kk,
                    wide ? id256 : id128, (k | kk) != 0);
          }
        }
        umma_commit(&sm.empty[s]);
      }
      umma_commit(&sm.done);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ producers
    const int chunk = tid & 7;
    const int nit = nblk * 4;
    const uint8_t* src[kMaxItems];
    int32_t sre[kMaxItems], sim[kMaxItems];
#pragma unroll
    for (int it = 0; it < kMaxItems; ++it) {
      src[it] = nullptr;
      sre[it] = 0;
      sim[it] = 0;
      if (it < nit) {
        const int pair = it * 16 + (tid >> 3);
        const int slot = pair >> 6, m = pair & 63;
        int ch, in;
        if (stacked) {
          const int half = a.rows_per_chan >> 1;
          ch = task.chan0 + m / half;
          in = m % half;
        } else {
          const int blk = slot < nb ? task.cb0 + slot : task.rb;
          ch = task.chan0;
          in = blk * 64 + m;
        }
        if (in < a.n_inputs && ch < a.n_chans)
          src[it] = a.x + (long long)ch * a.chan_stride + (long long)in * a.row_stride + a.t0 +
                    chunk * 16;
      }
    }
    for (int k = 0; k < nk; ++k) {
      const int s = k % nst;
      if (k >= nst && !mbar_wait(&sm.empty[s], (uint32_t)(k / nst - 1) & 1u, abort)) {
        raise_timeout(a.status, abort);
        break;
      }
      uint8_t* st = ops + s * stage_bytes;
      const int tk = k * kStageT + chunk * 16;  // first spectrum of this thread's chunk
#pragma unroll
      for (int it = 0; it < kMaxItems; ++it) {
        if (it < nit) {
          uint32_t w[4] = {0u, 0u, 0u, 0u};
          uint32_t keep[4] = {0u, 0u, 0u, 0u};
          if (src[it] != nullptr) {
            const uint8_t* p = src[it] + k * kStageT;
            if (a.vec_ok && tk + 16 <= a.tn) {
              const uint4 v = ld_stream16(p);
              w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
              keep[0] = keep[1] = keep[2] = keep[3] = 0xFFFFFFFFu;
            } else {
              for (int b = 0; b < 16; ++b) {
                if (tk + b < a.tn) {
                  w[b >> 2] |= (uint32_t)p[b] << ((b & 3) * 8);
                  keep[b >> 2] |= 0xFFu << ((b & 3) * 8);
                }
              }
            }
          }
          uint32_t re[4], im[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t lo = ((w[q] & 0x0F0F0F0Fu) ^ 0x08080808u) & keep[q];
            const uint32_t hi = (((w[q] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u) & keep[q];
            re[q] = a.lo_is_real ? lo : hi;
            im[q] = a.lo_is_real ? hi : lo;
            sre[it] = __dp4a(re[q], 0x01010101u, (uint32_t)sre[it]);
            sim[it] = __dp4a(im[q], 0x01010101u, (uint32_t)sim[it]);
          }
          const int pair = it * 16 + (tid >> 3);
          uint8_t* blk = st + (pair >> 6) * kBlockBytes;
          const int r0 = (pair & 63) * 2;
          *reinterpret_cast<uint4*>(blk + swz_offset(r0, chunk)) = make_uint4(re[0], re[1], re[2], re[3]);
          *reinterpret_cast<uint4*>(blk + swz_offset(r0 + 1, chunk)) = make_uint4(im[0], im[1], im[2], im[3]);
        }
      }
      fence_smem_to_async();
      mbar_arrive(&sm.full[s]);
    }
    // Row sums: the eight lanes of a pair hold its eight 16-spectrum chunks.
#pragma unroll
    for (int it = 0; it < kMaxItems; ++it) {
      if (it < nit) {
        int r = sre[it], m = sim[it];
        r += __shfl_xor_sync(0xFFFFFFFFu, r, 1);
        r += __shfl_xor_sync(0xFFFFFFFFu, r, 2);
        r += __shfl_xor_sync(0xFFFFFFFFu, r, 4);
        m += __shfl_xor_sync(0xFFFFFFFFu, m, 1);
        m += __shfl_xor_sync(0xFFFFFFFFu, m, 2);
        m += __shfl_xor_sync(0xFFFFFFFFu, m, 4);
        if (chunk == 0) {
          const int pair = it * 16 + (tid >> 3);
          sm.usum[(pair >> 6) * 128 + (pair & 63) * 2] = r;
          sm.usum[(pair >> 6) * 128 + (pair & 63) * 2 + 1] = m;
        }
      }
    }
    named_bar_sync(1, kProducers);

    // ------------------------------------------------------------ epilogue
    int never = 0;
    bool good = mbar_wait(&sm.done, 0, &never);
    good = __all_sync(0xFFFFFFFFu, good);
    if (!good && lane == 0) raise_timeout(a.status, abort);
    tc_after_sync();
    if (good && !*abort) {
      const int p = tid;  // row of the A block == tensor-memory lane
      const int n = a.n_inputs;
      int ch, i, plane;
      bool row_ok;
      if (stacked) {
        const int rpc = a.rows_per_chan;
        ch = task.chan0 + p / rpc;
        const int rr = p % rpc;
        i = rr >> 1;
        plane = rr & 1;
        row_ok = i < n && ch < a.n_chans;
      } else {
        ch = task.chan0;
        const int prow = task.rb * 128 + p;
        i = prow >> 1;
        plane = prow & 1;
        row_ok = i < n;
      }
      const int base_term = 64 * a.tn - 8 * sm.usum[a_slot * 128 + p];
      const long long nbl = (long long)n * (n + 1) / 2;
      int64_t* rowp = a.acc + ((long long)ch * nbl + (long long)i * (i + 1) / 2) * 2 + plane;
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
      for (int cc = 0; cc < nb * 4; ++cc) {
        uint32_t r[32];
        tmem_load32(trow + (uint32_t)(cc * 32), r);
        int g[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int q = cc * 32 + k;
          g[k] = __float2int_rn(__uint_as_float(r[k]) * 262144.0f) + base_term -
                 8 * sm.usum[q];  // column slots are 0..nb-1, contiguous
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int x = __shfl_xor_sync(0xFFFFFFFFu, g[2 * m + 1], 1);
          const int v = plane ? g[2 * m] - x : g[2 * m] + x;
          const int q = cc * 32 + 2 * m;
          int j;
          bool ok;
          if (stacked) {
            const int rpc = a.rows_per_chan;
            j = (q % rpc) >> 1;
            ok = row_ok && task.chan0 + q / rpc == ch && j <= i;
          } else {
            j = (128 * task.cb0 + q) >> 1;
            ok = row_ok && j <= i;
          }
          if (ok) {
            int64_t* d = rowp + 2 * j;
            if (a.accumulate)
              *d += v;
            else
              *d = v;
          }
        }
      }
    }
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, ncols);
}

}  // namespace

int herk4_max_smem() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, herk4_kernel) != cudaSuccess) return 0;
  return optin - (int)fa.sharedSizeBytes - 1024;
}

cudaError_t herk4_launch(const HerkArgs& a, int n_tasks, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(herk4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       a.smem_bytes);
  if (e != cudaSuccess) return e;
  herk4_kernel<<<n_tasks, kThreads, a.smem_bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace xe
