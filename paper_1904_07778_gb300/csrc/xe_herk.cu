// X-engine cross-multiply-and-accumulate (Sec. 2 "CMAC"; Sec. 2.2) for
// 4-bit complex samples on sm_103a tensor cores.
//
// Per channel, V_ij = sum_t x_i(t) conj(x_j(t)) for i >= j.  With Y the
// real (2N x T) matrix whose row 2i is Re x_i and row 2i+1 is Im x_i, and
// G = Y Y^T (symmetric), the visibilities are
//     Re V_ij = G[2i][2j] + G[2i+1][2j+1],   Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// The kernels form 128 x 128 blocks of G with tcgen05.mma kind::f8f6f4
// (E4M3 operands, FP32 accumulators in tensor memory), one or two column
// blocks per task (128 x 128 or 128 x 256 MMAs).
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
// Spectra outside the launch's time range use u = 0 and drop out of every
// term; padded rows are computed but never written.
//
// Kernels:
//   herk4_tma_kernel  (fast path) one warp streams packed bytes into a ring
//       of shared-memory stages with TMA; four groups of two warps unpack
//       stages k = g (mod 4) into the 128-byte-swizzled K-major operand ring,
//       so the latency of one stage overlaps three others; one warp issues
//       the MMAs; the eight unpack warps then drain tensor memory.
//   herk4_ldg_kernel  (any alignment) four warps load with 16-byte or byte
//       loads from global memory instead of TMA.
#include <algorithm>

#include "xe_device.cuh"

namespace xe {
namespace {

constexpr int kMaxStages = 8;
constexpr int kMaxBlocks = 2;                 // 128-row operand blocks per stage
constexpr int kStageT = 128;                  // spectra per stage = one swizzle row
constexpr int kOpBlockBytes = 128 * kStageT;  // unpacked: 128 rows x 128 spectra
constexpr int kPkBlockBytes = 64 * kStageT;   // packed: 64 inputs x 128 spectra

struct TaskGeom {
  int nb;       // column blocks (1 or 2) = B slots 0..nb-1
  int nblk;     // resident 128-row blocks per stage
  int a_slot;   // slot holding the A rows
  int rb;       // A row block
  int cb0, cb1; // column blocks of slots 0 and 1
  uint32_t ncols;
};

__device__ __forceinline__ TaskGeom task_geom(const HerkTask& t) {
  TaskGeom g;
  g.nb = t.cb[1] >= 0 ? 2 : 1;
  g.rb = t.rb;
  g.cb0 = t.cb[0];
  g.cb1 = t.cb[1];
  g.a_slot = t.rb == t.cb[0] ? 0 : (g.nb == 2 && t.rb == t.cb[1] ? 1 : g.nb);
  g.nblk = g.a_slot == g.nb ? g.nb + 1 : g.nb;
  g.ncols = g.nb == 1 ? 128u : 256u;
  return g;
}

// Row block held by operand slot s (B slots first, then a separate A slot).
__device__ __forceinline__ int slot_block(const TaskGeom& g, int s) {
  return s == 0 ? g.cb0 : (s < g.nb ? g.cb1 : g.rb);
}

__device__ __forceinline__ void raise_timeout(int* status, volatile int* abort) {
  *abort = 1;
  atomicOr(status, kStTimeout);
}

__device__ __forceinline__ uint32_t swz_offset(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Unpack 16 packed samples (4 words) into 16 real and 16 imaginary offset
// codes and add them to the row sums; with MASK, `keep` zeroes samples
// outside the time range.
template <bool LO_IS_REAL, bool MASK>
__device__ __forceinline__ void unpack16(const uint32_t (&w)[4], const uint32_t (&keep)[4],
                                         uint32_t (&re)[4], uint32_t (&im)[4], int32_t& sre,
                                         int32_t& sim) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t lo = (w[q] & 0x0F0F0F0Fu) ^ 0x08080808u;
    uint32_t hi = ((w[q] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
    if (MASK) {
      lo &= keep[q];
      hi &= keep[q];
    }
    re[q] = LO_IS_REAL ? lo : hi;
    im[q] = LO_IS_REAL ? hi : lo;
  }
  // bytes are <= 15, so four words add without carries between bytes
  sre = (int32_t)__dp4a(re[0] + re[1] + re[2] + re[3], 0x01010101u, (uint32_t)sre);
  sim = (int32_t)__dp4a(im[0] + im[1] + im[2] + im[3], 0x01010101u, (uint32_t)sim);
}

__device__ __forceinline__ void store_pair(uint8_t* stage, int pair, int chunk,
                                           const uint32_t (&re)[4], const uint32_t (&im)[4]) {
  uint8_t* blk = stage + (pair >> 6) * kOpBlockBytes;
  const int r0 = (pair & 63) * 2;
  *reinterpret_cast<uint4*>(blk + swz_offset(r0, chunk)) = make_uint4(re[0], re[1], re[2], re[3]);
  *reinterpret_cast<uint4*>(blk + swz_offset(r0 + 1, chunk)) = make_uint4(im[0], im[1], im[2], im[3]);
}

// Masks for a 16-spectrum chunk starting at spectrum tk of a launch of tn.
__device__ __forceinline__ void time_keep(int tk, int tn, uint32_t (&keep)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (tk + 4 * q + b < tn) m |= 0xFFu << (8 * b);
    keep[q] = m;
  }
}

// Row sums: the eight lanes of a pair hold its eight 16-spectrum chunks;
// item it of a thread covers pair it * (NT / 8) + tid / 8.  Partial sums of
// several unpack groups are added with shared-memory atomics.
template <int NT, int NI>
__device__ __forceinline__ void publish_row_sums(int32_t (&sre)[NI], int32_t (&sim)[NI], int nit,
                                                 int tid, int32_t* usum) {
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    if (it < nit) {
      int r = sre[it], m = sim[it];
      r += __shfl_xor_sync(0xFFFFFFFFu, r, 1);
      r += __shfl_xor_sync(0xFFFFFFFFu, r, 2);
      r += __shfl_xor_sync(0xFFFFFFFFu, r, 4);
      m += __shfl_xor_sync(0xFFFFFFFFu, m, 1);
      m += __shfl_xor_sync(0xFFFFFFFFu, m, 2);
      m += __shfl_xor_sync(0xFFFFFFFFu, m, 4);
      if ((tid & 7) == 0) {
        const int pair = it * (NT / 8) + (tid >> 3);
        atomicAdd(&usum[(pair >> 6) * 128 + (pair & 63) * 2], r);
        atomicAdd(&usum[(pair >> 6) * 128 + (pair & 63) * 2 + 1], m);
      }
    }
  }
}

// MMA issue loop (one thread): stage k of the operand ring holds the B rows
// in slots 0..nb-1 (contiguous) and the A rows in slot a_slot.
__device__ __forceinline__ void mma_loop(const TaskGeom& g, int nk, int nst, uint32_t ops_addr,
                                         uint32_t stage_bytes, uint32_t tmem, uint64_t* full,
                                         uint64_t* empty, uint64_t* done, int* status,
                                         volatile int* abort) {
  const uint32_t idesc = umma_idesc(0, 128, 128 * g.nb);
  int s = 0;
  uint32_t ph = 0;
  for (int k = 0; k < nk; ++k) {
    if (!mbar_wait(&full[s], ph, abort)) {
      raise_timeout(status, abort);
      break;
    }
    tc_after_sync();
    const uint32_t st = ops_addr + (uint32_t)s * stage_bytes;
    const uint64_t adesc = umma_desc_sw128(st + (uint32_t)(g.a_slot * kOpBlockBytes));
    const uint64_t bdesc = umma_desc_sw128(st);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      umma_f8(tmem, adesc + 2 * kk, bdesc + 2 * kk, idesc, (k | kk) != 0);
    umma_commit(&empty[s]);
    if (++s == nst) {
      s = 0;
      ph ^= 1u;
    }
  }
  umma_commit(done);
}

// Drain the accumulators, correct the offset codes, fold 2 x 2 real blocks
// into complex visibilities and store or add them into the int64
// integration buffer.  NW warps: warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31 (rows of the A block) and the (w / 4)-th share of the
// 32-column chunks.  Column block c < rb is a lower-triangle block, c == rb
// the diagonal block (entries j <= i only), c > rb the transpose of block
// (c, rb): there the thread's row is the second input of the baseline and
// the imaginary part changes sign.
template <int NW>
__device__ __forceinline__ void epilogue(const HerkArgs& a, const HerkTask& task, const TaskGeom& g,
                                         const int32_t* usum, uint32_t tmem, int tid) {
  const int warp = tid >> 5;
  const int quad = warp & 3, part = warp >> 2;
  const bool stacked = a.rows_per_chan > 0;
  const int p = quad * 32 + (tid & 31);
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
  const int base_term = 64 * a.tn - 8 * usum[g.a_slot * 128 + p];
  const long long nbl = (long long)n * (n + 1) / 2;
  int64_t* chp = a.acc + (long long)ch * nbl * 2;
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
  const int nch = g.nb * 4, per = nch / (NW / 4);
  for (int cc = part * per; cc < (part + 1) * per; ++cc) {
    uint32_t r[32];
    tmem_load32(trow + (uint32_t)(cc * 32), r);
    int gv[32];
#pragma unroll
    for (int k = 0; k < 32; ++k)
      gv[k] = __float2int_rn(__uint_as_float(r[k]) * 262144.0f) + base_term - 8 * usum[cc * 32 + k];
    const int cblk = slot_block(g, cc >> 2);
    const bool upper = !stacked && cblk > task.rb;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int x = __shfl_xor_sync(0xFFFFFFFFu, gv[2 * m + 1], 1);
      int v = plane ? gv[2 * m] - x : gv[2 * m] + x;
      const int q = (cc & 3) * 32 + 2 * m;  // column within its block
      long long b;
      bool ok;
      if (stacked) {
        const int rpc = a.rows_per_chan;
        const int j = (q % rpc) >> 1;
        ok = row_ok && task.chan0 + q / rpc == ch && j <= i;
        b = (long long)i * (i + 1) / 2 + j;
      } else {
        const int j = (128 * cblk + q) >> 1;
        if (upper) {
          // block (c, rb) transposed: baseline (j, i) with j > i
          ok = row_ok && j < n;
          b = (long long)j * (j + 1) / 2 + i;
          if (plane) v = -v;
        } else {
          ok = row_ok && j <= i;
          b = (long long)i * (i + 1) / 2 + j;
        }
      }
      if (ok) {
        int64_t* d = chp + 2 * b + plane;
        if (a.accumulate)
          *d += v;
        else
          *d = v;
      }
    }
  }
}

struct Ctrl {
  uint64_t full_p[kMaxStages];   // packed stage loaded (TMA transaction bytes)
  uint64_t empty_p[kMaxStages];  // packed stage consumed by the unpackers
  uint64_t full_o[kMaxStages];   // operand stage written
  uint64_t empty_o[kMaxStages];  // operand stage consumed by the MMAs
  uint64_t done;
  uint32_t tmem_base;
  int abort;
  int32_t usum[kMaxBlocks * 128];
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) &
                                    ~static_cast<uintptr_t>(1023));
}

__device__ __forceinline__ void ctrl_init_common(Ctrl& sm, int tid) {
  if (tid == 0) {
    mbar_init(&sm.done, 1);
    sm.abort = 0;
  }
  for (int i = tid; i < kMaxBlocks * 128; i += blockDim.x) sm.usum[i] = 0;
}

// -------------------------------------------------------------- TMA kernel
// Warps 0..15: four unpack groups of four warps (then the epilogue); warp
// 16 issues MMAs; warp 17 issues TMA loads.
constexpr int kGroups = 4;
constexpr int kGroupWarps = 4;
constexpr int kGroupThreads = kGroupWarps * 32;
constexpr int kUnpackWarps = kGroups * kGroupWarps;
constexpr int kTmaThreads = kUnpackWarps * 32 + 64;
constexpr int kTmaItems = kMaxBlocks * 512 / kGroupThreads;  // per thread per stage

template <bool LO_IS_REAL>
__global__ void __launch_bounds__(kTmaThreads, 1)
    herk4_tma_kernel(const __grid_constant__ CUtensorMap tmap, const HerkArgs a) {
  extern __shared__ uint8_t dyn_raw[];
  __shared__ Ctrl sm;
  uint8_t* ops = align1024(dyn_raw);
  const HerkTask task = a.tasks[blockIdx.x];
  const TaskGeom g = task_geom(task);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool stacked = a.rows_per_chan > 0;
  const int op_stage = g.nblk * kOpBlockBytes, pk_stage = g.nblk * kPkBlockBytes;
  // Ring depths are multiples of the number of unpack groups, so that stage
  // k always lands in a slot that only group k % kGroups fills: a group then
  // waits on a slot whose previous fill was its own, and an mbarrier can
  // never be more than one phase away from the phase awaited (a parity wait
  // on an older phase would pass falsely).
  const int avail = a.smem_bytes - 1024;
  int no = kGroups * ((avail - kGroups * pk_stage) / (kGroups * op_stage));
  if (no > kMaxStages) no = kMaxStages;
  int np = kGroups * ((avail - no * op_stage) / (kGroups * pk_stage));
  if (np > kMaxStages) np = kMaxStages;
  uint8_t* pk = ops + no * op_stage;
  const int nk = (a.tn + kStageT - 1) / kStageT;
  volatile int* abort = &sm.abort;

  ctrl_init_common(sm, tid);
  if (tid == 0) {
    for (int s = 0; s < np; ++s) {
      mbar_init(&sm.full_p[s], 1);
      mbar_init(&sm.empty_p[s], kGroupWarps);
    }
    for (int s = 0; s < no; ++s) {
      mbar_init(&sm.full_o[s], kGroupWarps);
      mbar_init(&sm.empty_o[s], 1);
    }
  }
  if (warp == 0) tmem_alloc(&sm.tmem_base, g.ncols);
  fence_mbar_init();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == kUnpackWarps + 1) {
    // ------------------------------------------------------------ TMA loader
    if (lane == 0) {
      tma_prefetch_desc(&tmap);
      const uint32_t pk_addr = smem_addr(pk);
      int s = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nk; ++k) {
        if (k >= np && !mbar_wait(&sm.empty_p[s], ph ^ 1u, abort)) {
          raise_timeout(a.status, abort);
          break;
        }
        mbar_expect_tx(&sm.full_p[s], (uint32_t)pk_stage);
        const int t = a.t0 + k * kStageT;
        for (int slot = 0; slot < g.nblk; ++slot) {
          const uint32_t dst = pk_addr + (uint32_t)(s * pk_stage + slot * kPkBlockBytes);
          if (stacked)
            tma_load_3d(dst, &tmap, t, 0, task.chan0, &sm.full_p[s]);
          else
            tma_load_3d(dst, &tmap, t, 64 * slot_block(g, slot), task.chan0, &sm.full_p[s]);
        }
        if (++s == np) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    __syncwarp();
  } else if (warp == kUnpackWarps) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0)
      mma_loop(g, nk, no, smem_addr(ops), (uint32_t)op_stage, tmem, sm.full_o, sm.empty_o,
               &sm.done, a.status, abort);
    __syncwarp();
  } else {
    // ------------------------------------------------------------ unpackers
    const int grp = warp / kGroupWarps;
    const int gt = tid - grp * kGroupThreads;  // thread within the group
    const int chunk = gt & 7;
    const int nit = g.nblk * 512 / kGroupThreads;
    int32_t sre[kTmaItems], sim[kTmaItems];
#pragma unroll
    for (int it = 0; it < kTmaItems; ++it) sre[it] = sim[it] = 0;
    const uint32_t ones[4] = {~0u, ~0u, ~0u, ~0u};
    // this group's stages are k = grp, grp + kGroups, ...
    int sp = grp % np, so = grp % no;
    uint32_t php = (uint32_t)((grp / np) & 1), pho = (uint32_t)((grp / no) & 1);
    for (int k = grp; k < nk; k += kGroups) {
      if (!mbar_wait(&sm.full_p[sp], php, abort) ||
          (k >= no && !mbar_wait(&sm.empty_o[so], pho ^ 1u, abort))) {
        raise_timeout(a.status, abort);
        break;
      }
      const uint8_t* src = pk + sp * pk_stage + chunk * 16;
      uint8_t* dst = ops + so * op_stage;
      const bool tail = (k + 1) * kStageT > a.tn;
      uint32_t keep[4] = {~0u, ~0u, ~0u, ~0u};
      if (tail) time_keep(k * kStageT + chunk * 16, a.tn, keep);
      // all shared-memory loads of the stage first, then hand the packed
      // stage back to the loader so that it refills while this group unpacks
      uint4 v[kTmaItems];
#pragma unroll
      for (int it = 0; it < kTmaItems; ++it)
        if (it < nit)
          v[it] = *reinterpret_cast<const uint4*>(
              src + (it * (kGroupThreads / 8) + (gt >> 3)) * kStageT);
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty_p[sp]);
#pragma unroll
      for (int it = 0; it < kTmaItems; ++it) {
        if (it < nit) {
          const int pair = it * (kGroupThreads / 8) + (gt >> 3);
          const uint32_t w[4] = {v[it].x, v[it].y, v[it].z, v[it].w};
          uint32_t re[4], im[4];
          if (tail)
            unpack16<LO_IS_REAL, true>(w, keep, re, im, sre[it], sim[it]);
          else
            unpack16<LO_IS_REAL, false>(w, ones, re, im, sre[it], sim[it]);
          store_pair(dst, pair, chunk, re, im);
        }
      }
      // one arrival per warp: every lane makes its stores visible to the
      // tensor core (async proxy), then the warp synchronises
      fence_smem_to_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.full_o[so]);
      sp += kGroups;
      while (sp >= np) {
        sp -= np;
        php ^= 1u;
      }
      so += kGroups;
      while (so >= no) {
        so -= no;
        pho ^= 1u;
      }
    }
    publish_row_sums<kGroupThreads>(sre, sim, nit, gt, sm.usum);
    named_bar_sync(1, kUnpackWarps * 32);
    int never = 0;
    bool good = mbar_wait(&sm.done, 0, &never);
    good = __all_sync(0xFFFFFFFFu, good);
    if (!good && lane == 0) raise_timeout(a.status, abort);
    tc_after_sync();
    if (good && !*abort) epilogue<kUnpackWarps>(a, task, g, sm.usum, tmem, tid);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, g.ncols);
}

// -------------------------------------------------------------- LDG kernel
// Warps 0..3 load, unpack and drain; warp 4 issues MMAs.
constexpr int kLdgThreads = 160;
constexpr int kLdgItems = kMaxBlocks * 4;

template <bool LO_IS_REAL>
__global__ void __launch_bounds__(kLdgThreads, 1) herk4_ldg_kernel(const HerkArgs a) {
  extern __shared__ uint8_t dyn_raw[];
  __shared__ Ctrl sm;
  uint8_t* ops = align1024(dyn_raw);
  const HerkTask task = a.tasks[blockIdx.x];
  const TaskGeom g = task_geom(task);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool stacked = a.rows_per_chan > 0;
  const int stage_bytes = g.nblk * kOpBlockBytes;
  int nst = (a.smem_bytes - 1024) / stage_bytes;
  if (nst > kMaxStages) nst = kMaxStages;
  const int nk = (a.tn + kStageT - 1) / kStageT;
  volatile int* abort = &sm.abort;

  ctrl_init_common(sm, tid);
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&sm.full_o[s], 128);
      mbar_init(&sm.empty_o[s], 1);
    }
  }
  if (warp == 0) tmem_alloc(&sm.tmem_base, g.ncols);
  fence_mbar_init();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 4) {
    if (lane == 0)
      mma_loop(g, nk, nst, smem_addr(ops), (uint32_t)stage_bytes, tmem, sm.full_o, sm.empty_o,
               &sm.done, a.status, abort);
    __syncwarp();
  } else {
    const int chunk = tid & 7;
    const int nit = g.nblk * 4;
    const uint8_t* src[kLdgItems];
    int32_t sre[kLdgItems], sim[kLdgItems];
#pragma unroll
    for (int it = 0; it < kLdgItems; ++it) {
      src[it] = nullptr;
      sre[it] = sim[it] = 0;
      if (it < nit) {
        const int pair = it * 16 + (tid >> 3);
        const int slot = pair >> 6, m = pair & 63;
        int ch, in;
        if (stacked) {
          const int half = a.rows_per_chan >> 1;
          ch = task.chan0 + m / half;
          in = m % half;
        } else {
          ch = task.chan0;
          in = slot_block(g, slot) * 64 + m;
        }
        if (in < a.n_inputs && ch < a.n_chans)
          src[it] = a.x + (long long)ch * a.chan_stride + (long long)in * a.row_stride + a.t0 +
                    chunk * 16;
      }
    }
    int s = 0;
    uint32_t ph = 0;
    for (int k = 0; k < nk; ++k) {
      if (k >= nst && !mbar_wait(&sm.empty_o[s], ph ^ 1u, abort)) {
        raise_timeout(a.status, abort);
        break;
      }
      uint8_t* st = ops + s * stage_bytes;
      const int tk = k * kStageT + chunk * 16;
      uint32_t w[kLdgItems][4], keep[kLdgItems][4];
      // issue every load of the stage before using any of them
#pragma unroll
      for (int it = 0; it < kLdgItems; ++it) {
        if (it < nit) {
#pragma unroll
          for (int q = 0; q < 4; ++q) w[it][q] = keep[it][q] = 0u;
          if (src[it] != nullptr) {
            const uint8_t* p = src[it] + k * kStageT;
            if (a.vec_ok && tk + 16 <= a.tn) {
              const uint4 v = ld_stream16(p);
              w[it][0] = v.x; w[it][1] = v.y; w[it][2] = v.z; w[it][3] = v.w;
              keep[it][0] = keep[it][1] = keep[it][2] = keep[it][3] = 0xFFFFFFFFu;
            } else {
              for (int b = 0; b < 16; ++b) {
                if (tk + b < a.tn) {
                  w[it][b >> 2] |= (uint32_t)p[b] << ((b & 3) * 8);
                  keep[it][b >> 2] |= 0xFFu << ((b & 3) * 8);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int it = 0; it < kLdgItems; ++it) {
        if (it < nit) {
          uint32_t re[4], im[4];
          unpack16<LO_IS_REAL, true>(w[it], keep[it], re, im, sre[it], sim[it]);
          store_pair(st, it * 16 + (tid >> 3), chunk, re, im);
        }
      }
      fence_smem_to_async();
      mbar_arrive(&sm.full_o[s]);
      if (++s == nst) {
        s = 0;
        ph ^= 1u;
      }
    }
    publish_row_sums<128>(sre, sim, nit, tid, sm.usum);
    named_bar_sync(1, 128);
    int never = 0;
    bool good = mbar_wait(&sm.done, 0, &never);
    good = __all_sync(0xFFFFFFFFu, good);
    if (!good && lane == 0) raise_timeout(a.status, abort);
    tc_after_sync();
    if (good && !*abort) epilogue<4>(a, task, g, sm.usum, tmem, tid);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, g.ncols);
}

int max_dyn_smem(const void* fn) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
  return optin - (int)fa.sharedSizeBytes;
}

template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

int herk4_max_smem() {
  int m = max_dyn_smem((const void*)herk4_tma_kernel<false>);
  m = std::min(m, max_dyn_smem((const void*)herk4_tma_kernel<true>));
  m = std::min(m, max_dyn_smem((const void*)herk4_ldg_kernel<false>));
  m = std::min(m, max_dyn_smem((const void*)herk4_ldg_kernel<true>));
  return m;
}

cudaError_t herk4_launch(const HerkArgs& a, const CUtensorMap* tmap, int n_tasks,
                         cudaStream_t s) {
  cudaError_t e;
  if (tmap) {
    if (a.lo_is_real) {
      if ((e = set_smem(herk4_tma_kernel<true>, a.smem_bytes)) != cudaSuccess) return e;
      herk4_tma_kernel<true><<<n_tasks, kTmaThreads, a.smem_bytes, s>>>(*tmap, a);
    } else {
      if ((e = set_smem(herk4_tma_kernel<false>, a.smem_bytes)) != cudaSuccess) return e;
      herk4_tma_kernel<false><<<n_tasks, kTmaThreads, a.smem_bytes, s>>>(*tmap, a);
    }
  } else {
    if (a.lo_is_real) {
      if ((e = set_smem(herk4_ldg_kernel<true>, a.smem_bytes)) != cudaSuccess) return e;
      herk4_ldg_kernel<true><<<n_tasks, kLdgThreads, a.smem_bytes, s>>>(a);
    } else {
      if ((e = set_smem(herk4_ldg_kernel<false>, a.smem_bytes)) != cudaSuccess) return e;
      herk4_ldg_kernel<false><<<n_tasks, kLdgThreads, a.smem_bytes, s>>>(a);
    }
  }
  return cudaGetLastError();
}

}  // namespace xe
