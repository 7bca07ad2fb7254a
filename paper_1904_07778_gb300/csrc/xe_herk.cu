// X-engine cross-multiply-and-accumulate (Sec. 2 "CMAC"; Sec. 2.2) for
// 4-bit and 8-bit complex samples on sm_103a tensor cores.
//
// Per channel, V_ij = sum_t x_i(t) conj(x_j(t)) for i >= j.  With Y the
// real (2N x T) matrix whose row 2i is Re x_i and row 2i+1 is Im x_i, and
// G = Y Y^T (symmetric), the visibilities are
//     Re V_ij = G[2i][2j] + G[2i+1][2j+1],   Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// The kernels form 128 x 128 blocks of G with tcgen05.mma (FP32 accumulators
// in tensor memory), one or two column blocks per task (128 x 128 or
// 128 x 256 MMAs).
//
// 4-bit operands (kind::f8f6f4).  A 4-bit two's-complement nibble n (value
// v in -8..7) is fed to the tensor core as the offset code u = n ^ 8 = v + 8
// in 0..15.  The E4M3 byte with bit pattern u (exponent field 0 or 1) has
// the value u * 2^-9 exactly, so unpacking a byte of two nibbles into two
// E4M3 bytes is one mask and one XOR.  The tensor core then accumulates
//     Gu[p][q] = 2^-18 sum_t u_p u_q,
// exact in FP32 while the integer sum stays below 2^24 (at most 225 per
// spectrum, so up to 65536 spectra per accumulation).  The signed Gram
// follows from the row sums U_p = sum_t u_p:
//     G[p][q] = sum (u_p - 8)(u_q - 8) = 2^18 Gu[p][q] - 8 U_p - 8 U_q + 64 T.
// Spectra outside the launch's time range use u = 0 and drop out of every
// term; padded rows are computed but never written.
//
// 8-bit operands (kind::f16).  A byte in -127..127 is an FP16 value of the
// same integer, so Y holds the samples themselves and G needs no
// correction.  A product is at most 127^2 < 2^14, so an FP32 accumulation
// stays exact over 1024 spectra (127^2 * 1024 < 2^24); longer tasks are
// accumulated 1024 spectra at a time, and the drain adds the pieces as
// integers.
//
// Kernels:
//   herk4_ring_kernel (fast path) persistent, one CTA per SM: a TMA warp
//       streams packed bytes into a ring of shared-memory slots, four groups
//       of four warps unpack them in place into the 128-byte-swizzled K-major
//       operand layout, one warp issues the MMAs into two alternating
//       tensor-memory accumulators, and eight warps drain the previous
//       accumulation.
//   herk4_ldg_kernel  (4-bit, any alignment) four warps load with 16-byte or
//       byte loads from global memory instead of TMA.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "xe_device.cuh"

namespace xe {
namespace {

constexpr int kMaxStages = 12;
constexpr int kMaxBlocks = 2;                 // 128-row operand blocks per stage
constexpr int kStageT = 128;                  // spectra per stage = one swizzle row
constexpr int kOpBlockBytes = 128 * kStageT;  // unpacked: 128 rows x 128 spectra

struct TaskGeom {
  int nb;       // column blocks (1 or 2) = B slots 0..nb-1
  int nblk;     // distinct 128-row blocks of the task
  int a_slot;   // slot holding the A rows
  int rb;       // A row block
  int cb0, cb1; // column blocks of slots 0 and 1
  int dbl;      // ring kernel: one block (A = B), a stage holds two time ranges of it
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
  g.dbl = g.nblk == 1 ? 1 : 0;
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

// Unpack 16 packed 4-bit samples (4 words) into 16 real and 16 imaginary
// offset codes and add them to the row sums; with MASK, `keep` zeroes
// samples outside the time range.
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

// a - b for two FP16 lanes
__device__ __forceinline__ uint32_t f16x2_sub(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Sixteen 8-bit samples (4 little-endian words; `keep` zeroes samples outside
// the time range) to sixteen FP16 values of the same integers, eight f16x2
// words in sample order.  Byte b becomes the half with bit pattern
// 0x6400 | (b ^ 0x80), whose value is 1024 + (v + 128), and 1152 is
// subtracted in FP16: every operand and result is an integer below 2048 in
// magnitude, so both steps are exact.  `bad` gets a bit if a kept byte is
// 0x80 (-128, outside the symmetric range).
__device__ __forceinline__ void s8_to_f16(const uint32_t (&w)[4], const uint32_t (&keep)[4],
                                          uint32_t (&h)[8], uint32_t& bad) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t z = (w[q] ^ 0x80808080u) | ~keep[q];  // a zero byte: a kept 0x80
    bad |= (z - 0x01010101u) & ~z & 0x80808080u;
    const uint32_t u = (w[q] & keep[q]) ^ 0x80808080u;
    h[2 * q] = f16x2_sub(__byte_perm(u, 0x64646464u, 0x4140), 0x64806480u);
    h[2 * q + 1] = f16x2_sub(__byte_perm(u, 0x64646464u, 0x4342), 0x64806480u);
  }
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

// Row sums: the CH lanes of a pair hold its CH 16-spectrum chunks; item it
// of a thread covers pair it * (NT / CH) + tid / CH.  Partial sums of
// several unpack groups are added with shared-memory atomics.
template <int NT, int NI, int CH = 8>
__device__ __forceinline__ void publish_row_sums(int32_t (&sre)[NI], int32_t (&sim)[NI], int nit,
                                                 int tid, int32_t* usum) {
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    if (it < nit) {
      int r = sre[it], m = sim[it];
#pragma unroll
      for (int x = 1; x < CH; x <<= 1) {
        r += __shfl_xor_sync(0xFFFFFFFFu, r, x);
        m += __shfl_xor_sync(0xFFFFFFFFu, m, x);
      }
      if ((tid & (CH - 1)) == 0) {
        const int pair = it * (NT / CH) + tid / CH;
        atomicAdd(&usum[(pair >> 6) * 128 + (pair & 63) * 2], r);
        atomicAdd(&usum[(pair >> 6) * 128 + (pair & 63) * 2 + 1], m);
      }
    }
  }
}

// ---- payload-order ([t][c][i]) stages -------------------------------------
// A stage of a block read straight from the payload order is [t][64 bytes]:
// 128 spectra of 64 byte rows (the inputs of one block, or of the stacked
// channels).  The unpack gathers each row's bytes across time with 32-bit
// shared loads and 4 x 4 byte transposes.  Within a stage the operands'
// K order is a permutation of time -- the same for every row, so the Gram
// matrix and the row sums are unchanged: K position 16 c + j holds spectrum
// tci_t(c, j), which makes both the gathers and the operand stores free of
// bank conflicts (lanes 2q and 2q + 1 of a warp read opposite parities).
__device__ __forceinline__ int tci_t(int c, int j) { return 32 * (c >> 1) + 2 * j + (c & 1); }

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void transpose4x4b(uint32_t& a0, uint32_t& a1, uint32_t& a2,
                                              uint32_t& a3) {
  const uint32_t t0 = __byte_perm(a0, a1, 0x5140), t1 = __byte_perm(a0, a1, 0x7362);
  const uint32_t t2 = __byte_perm(a2, a3, 0x5140), t3 = __byte_perm(a2, a3, 0x7362);
  a0 = __byte_perm(t0, t2, 0x5410);
  a1 = __byte_perm(t0, t2, 0x7632);
  a2 = __byte_perm(t1, t3, 0x5410);
  a3 = __byte_perm(t1, t3, 0x7632);
}

// Masks of the 16 bytes (K positions 16 c .. 16 c + 15) of chunk c in a stage
// starting at spectrum tk of a launch of tn spectra.
__device__ __forceinline__ void tci_keep(int c, int tk, int tn, uint32_t (&keep)[4]) {
  const int lim = tn - tk - 32 * (c >> 1) - (c & 1);  // byte j is valid if 2 j < lim
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (2 * (4 * q + b) < lim) m |= 0xFFu << (8 * b);
    keep[q] = m;
  }
}

// 8-bit payload-order stages ([t][128 bytes], 64 spectra): a thread holds
// byte j of its 16 gathered spectra at spectrum 16 c + (j ^ sw8) of the
// stage; masks of those bytes for lim = valid spectra from the stage's start.
__device__ __forceinline__ void tci8_keep(int c, int sw8, int lim, uint32_t (&keep)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (16 * c + ((4 * q + b) ^ sw8) < lim) m |= 0xFFu << (8 * b);
    keep[q] = m;
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

// Drain the accumulators, correct the offset codes (4-bit), fold 2 x 2 real
// blocks into complex visibilities and store or add them into the int64
// integration buffer.  The calling warp reads tensor-memory lanes
// 32 quad .. + 31 (rows of the A block; quad must be the warp index mod 4)
// and the part-th of nparts shares of the 16-column chunks.  Column block
// c < rb is a lower-triangle block, c == rb the diagonal block (entries
// j <= i only), c > rb the transpose of block (c, rb): there the thread's
// row is the second input of the baseline and the imaginary part changes
// sign.  The two lanes of an input (rows 2i and 2i + 1) exchange halves so
// that each holds whole (Re, Im) pairs: the even-numbered columns j of the
// chunk go to the lane of row 2i, the odd ones to row 2i + 1, and each
// visibility is one 16-byte store (adjacent lanes fill 32 contiguous bytes
// in lower blocks, 16 lanes fill 256 contiguous bytes in upper blocks).
//
// F16 (8-bit samples): the accumulators hold G itself.  A task is drained
// once per accumulation of at most 1024 spectra; every accumulation but the
// last leaves its int32 visibilities in the CTA's scratch (int2 per
// position, entry (4 cc + u) 128 + p, written and read by the same thread),
// which the next one adds in, and the last goes to the integration buffer.
// The int32 sums stay below 2 * 127^2 * 32768 < 2^31 for the longest block.
template <bool F16>
__device__ __forceinline__ void epilogue(const HerkInst& a, const HerkTask& task, const TaskGeom& g,
                                         const int32_t* usum, uint32_t tmem, int quad, int part,
                                         int nparts, int lane, bool first, bool last, int2* scr) {
  const bool stacked = a.rows_per_chan > 0;
  const int p = quad * 32 + lane;
  const int n = a.n_inputs;
  int ch, i, plane;
  bool row_ok;
  // A stacked tile has a power of two (2 .. 64) of rows per channel, so its
  // channel and row splits are masks and shifts (the drain warps share their
  // SMSPs with the busy unpack warps: every instruction of theirs counts).
  if (stacked) {
    const int rpc = a.rows_per_chan;
    ch = task.chan0 + (p >> (31 - __clz(rpc)));
    const int rr = p & (rpc - 1);
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
  const int base_term = F16 ? 0 : 64 * a.tn - 8 * usum[g.a_slot * 128 + p];
  const long long nbl = (long long)n * (n + 1) / 2;
  int64_t* chp = a.acc + (long long)(row_ok ? ch : 0) * nbl * 2;
  const int tri_i = i * (i + 1) / 2;  // baselines per channel stay below 2^30 (inputs <= 32768)
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
  // 16-column chunks of this warp's share.  In a stacked tile a lane's row
  // only meets columns of its own channel: the rows 32 quad .. + 31 of this
  // warp belong to one channel (rows_per_chan >= 32), whose columns are
  // rows_per_chan / 16 chunks, or to channels whose columns are the two
  // chunks 2 quad, 2 quad + 1; the other chunks hold no visibility.
  int c0 = 0, c1 = g.nb * 8;
  if (stacked) {
    const int rpc = a.rows_per_chan;
    c0 = rpc >= 32 ? (rpc == 32 ? quad : quad >> 1) * (rpc >> 4) : 2 * quad;  // rpc <= 64
    c1 = c0 + (rpc >= 32 ? rpc >> 4 : 2);
  }
  const int per = (c1 - c0 + nparts - 1) / nparts;
  const int cbeg = c0 + part * per, cend = min(c1, cbeg + per);
  for (int cc = cbeg; cc < cend; ++cc) {
    int2 prev[4];
    int2* sp = scr + (cc * 4) * 128 + p;
    if (F16 && !first) {
#pragma unroll
      for (int u = 0; u < 4; ++u) prev[u] = sp[u * 128];
    }
    uint32_t r[16];
    tmem_load16(trow + (uint32_t)(cc * 16), r);
    int cs[16];  // 4-bit: the chunk's 16 column sums, in four 16-byte loads
    if constexpr (!F16) {
      const int4* u4 = reinterpret_cast<const int4*>(usum + cc * 16);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int4 v = u4[w];
        cs[4 * w] = v.x, cs[4 * w + 1] = v.y, cs[4 * w + 2] = v.z, cs[4 * w + 3] = v.w;
      }
    }
    int gv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if constexpr (F16)
        gv[k] = __float2int_rn(__uint_as_float(r[k]));
      else
        gv[k] = __float2int_rn(__uint_as_float(r[k]) * 262144.0f) + base_term - 8 * cs[k];
    }
    const int cblk = slot_block(g, cc >> 3);
    const bool upper = !stacked && cblk > task.rb;
    int vre[4], vim[4];
    int off[4];  // element offset of the pair within the channel, -1: not stored
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // columns 2u (lane of row 2i) and 2u + 1 (row 2i + 1)
      const int x0 = plane ? gv[4 * u + 2] : gv[4 * u];
      const int x1 = plane ? gv[4 * u + 3] : gv[4 * u + 1];
      const int y0 = __shfl_xor_sync(0xFFFFFFFFu, plane ? gv[4 * u] : gv[4 * u + 2], 1);
      const int y1 = __shfl_xor_sync(0xFFFFFFFFu, plane ? gv[4 * u + 1] : gv[4 * u + 3], 1);
      // G[2i][2j] + G[2i+1][2j+1] and G[2i+1][2j] - G[2i][2j+1] for this lane's column j
      vre[u] = plane ? y0 + x1 : x0 + y1;
      vim[u] = plane ? x0 - y1 : y0 - x1;
      const int q = (cc & 7) * 16 + 2 * (2 * u + plane);  // real column of input j in its block
      int b;
      bool ok;
      if (stacked) {
        // column q and row p of the tile share a channel when they agree
        // above the rows-per-channel bits
        const int rpc = a.rows_per_chan;
        const int j = (q & (rpc - 1)) >> 1;
        ok = row_ok && (q ^ p) < rpc && j <= i;
        b = tri_i + j;
      } else {
        const int j = (128 * cblk + q) >> 1;
        if (upper) {
          ok = row_ok && j < n;  // baseline (j, i), j > i: the conjugate
          b = j * (j + 1) / 2 + i;
          vim[u] = -vim[u];
        } else {
          ok = row_ok && j <= i;
          b = tri_i + j;
        }
      }
      off[u] = ok ? 2 * b : -1;
    }
    if (F16) {
      if (!first) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          vre[u] += prev[u].x;
          vim[u] += prev[u].y;
        }
      }
      if (!last) {
#pragma unroll
        for (int u = 0; u < 4; ++u) sp[u * 128] = make_int2(vre[u], vim[u]);
        continue;
      }
    }
    if (a.accumulate) {
      // reductions at L2: nothing waits for the old value
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (off[u] >= 0) red_s64x2(chp + off[u], vre[u], vim[u]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (off[u] >= 0) st_s64x2(chp + off[u], vre[u], vim[u]);
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
  alignas(16) int32_t usum[kMaxBlocks * 128];  // read by the drain in 16-byte loads
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

// ------------------------------------------------------------- ring kernel
// Persistent: one CTA per SM walks the tasks blockIdx.x, blockIdx.x + grid,
// ...; stage S counts the stages of all its tasks in order (128 spectra at 4
// bits, 64 at 8 bits, twice that for the double stages of one-block tasks).
// Shared memory is one ring of 32 KB slots, each holding the two units of a
// stage (see kSlotBytes).  Stage S uses slot S mod ns:
//   warp 17 (TMA)     waits until the MMAs of stage S - ns have finished with
//                     the slot, then loads the packed bytes of stage S into
//                     its upper half;
//   group S mod 4     (warps 4g .. 4g + 3) waits for the same MMA completion
//                     and for the bytes, converts unit 0 into the lower half,
//                     reads unit 1 into registers, meets at a group barrier,
//                     and writes unit 1's operands over the packed bytes;
//   warp 16 (MMA)     issues the four (double stage: eight) MMAs of the stage
//                     into one of two 256-column tensor-memory accumulators
//                     (accumulations alternate) and commits the slot back;
//   warps 20..27      (drain) convert accumulation v while accumulation v + 1
//                     is being multiplied (warps 18, 19 only complete the
//                     warpgroup of warps 16, 17).
// An accumulation is a whole task at 4 bits, and at 8 bits up to 1024
// spectra of one (a task of T spectra takes ceil(T / 1024) in a row).
// The unpack warpgroups take registers from the others (setmaxnreg): the
// unpack loop holds a whole stage in registers across the group barrier.
// Every wait on a slot barrier for phase m is preceded by a completed wait
// for phase m - 1 of a barrier whose completion implies it (the MMAs run in
// order), so the parity of a phase two behind can never be mistaken for the
// awaited one, whatever ns >= 4 is.
#ifndef XE_EPI_WARPS
#define XE_EPI_WARPS 8
#endif
#ifndef XE_GROUPS
#define XE_GROUPS 4
#endif
constexpr int kGroups = XE_GROUPS;            // unpack groups (stages S = g mod kGroups)
constexpr int kGroupWarps = 16 / kGroups;
constexpr int kGroupThreads = kGroupWarps * 32;
constexpr int kUnpackWarps = kGroups * kGroupWarps;
// Ring stages.  Every row of Y gets one 128-byte swizzled operand row per
// stage: 128 spectra of E4M3 codes (4-bit samples) or 64 spectra of FP16
// values (8-bit samples).  Either way a 128-row block is 16 KB of operands
// made from 8 KB of packed bytes (64 byte rows x 128 spectra, or 128 byte
// rows x 64 spectra), and a stage takes four MMAs of K = 32 bytes per row.
constexpr int kROpBlock = 128 * 128;  // operands of a 128-row block
constexpr int kRPkBlock = 64 * 128;   // packed bytes of a 128-row block
constexpr int kRKSteps = 4;           // MMAs per 128-row block and time range
// A ring slot holds two units of one stage: the two 128-row blocks of a
// two-block task, or for a one-block task (A = B) the same rows over two
// consecutive time ranges ("double" stages: half the stages, so half the
// per-stage hand-offs, for tasks that would move only 8 KB a stage).
// Operands of unit u at [16 u, 16 u + 16) KB, packed bytes at [16 + 8 u, 24 + 8 u) KB.
constexpr int kSlotBytes = 2 * kROpBlock;
template <bool EIGHT>
__host__ __device__ constexpr int stage_t() {  // spectra per stage
  return EIGHT ? 64 : 128;
}
// 8-bit: spectra per tensor-memory accumulation (FP32 sums of products of at
// most 127^2 stay exact integers: 127^2 * 1024 < 2^24)
constexpr int kPiece8 = 1024;
constexpr int kPieceStages8 = kPiece8 / stage_t<true>();
constexpr int kItems = kMaxBlocks * 4;  // 16-byte packed items per unpack thread and stage
static_assert(kGroupThreads == 128, "an unpack group covers a packed block in four items a thread");
constexpr int kMmaWarp = kUnpackWarps, kTmaWarp = kUnpackWarps + 1, kEpiWarp0 = kUnpackWarps + 4;
constexpr int kEpiWarps = XE_EPI_WARPS;
constexpr int kRingThreads = (kEpiWarp0 + kEpiWarps) * 32;
// registers per thread: launch share, unpack warpgroups, the other warpgroups.
// Chosen per instance from the compiler's spill report and measured times:
// the 8-bit drain, which adds the accumulations' partial sums, takes more,
// the 8-bit unpack less; the low-nibble-real 4-bit unpack needs 88.
constexpr int kRegsLaunch = (65536 / kRingThreads) & ~7;
template <bool LO, bool EIGHT>
__host__ __device__ constexpr int regs_unpack() { return EIGHT ? 72 : (LO ? 88 : 80); }
template <bool LO, bool EIGHT>
__host__ __device__ constexpr int regs_other() { return EIGHT ? 64 : (LO ? 48 : 56); }
static_assert(kRingThreads % 128 == 0, "whole warpgroups");
template <bool LO, bool EIGHT>
constexpr bool regs_fit() {
  return kUnpackWarps * 32 * regs_unpack<LO, EIGHT>() +
             (kRingThreads - kUnpackWarps * 32) * regs_other<LO, EIGHT>() <=
         kRingThreads * kRegsLaunch;
}
static_assert(regs_fit<false, false>() && regs_fit<true, false>() && regs_fit<false, true>(),
              "the register split must fit in the launch allocation");
#ifndef XE_MAX_SLOTS
#define XE_MAX_SLOTS 16
#endif
constexpr int kMaxSlots = XE_MAX_SLOTS;  // ring slots at most (shared memory sets the count)
static_assert(kEpiWarps % 4 == 0, "drain warps cover the four tensor-memory lane quarters");
static_assert(kEpiWarps / 4 <= 2 && 16 * 4 * 128 == kHerkScratchInt2,
              "the 8-bit scratch holds 4 values of 128 rows for each of 16 column chunks");

struct RingCtrl {
  uint64_t full_t[kMaxSlots];    // packed bytes of the slot landed (TMA transaction count)
  uint64_t full_o[kMaxSlots];    // operands of the slot written (one arrival per group warp)
  uint64_t empty[kMaxSlots];     // MMAs of the slot finished (tcgen05.commit)
  uint64_t tmem_full[2];         // accumulator buffer complete
  uint64_t tmem_empty[2];        // accumulator buffer drained
  uint64_t usum_full[2];         // row sums of the task published
  uint64_t usum_empty[2];        // row sums consumed and cleared
  uint64_t done;                 // every MMA finished (before freeing tensor memory)
  uint32_t tmem_base;
  int abort;
  alignas(16) int32_t usum[2][kMaxBlocks * 128];  // read by the drain in 16-byte loads
};

// Task j of this CTA: its explicit list, or round robin over the CTAs.
__device__ __forceinline__ HerkTask my_task(const HerkArgs& a, int j) {
  return a.cta_first ? a.tasks[a.cta_first[blockIdx.x] + j] : a.tasks[blockIdx.x + j * gridDim.x];
}
__device__ __forceinline__ int my_task_count(const HerkArgs& a) {
  if (a.cta_first) return a.cta_first[blockIdx.x + 1] - a.cta_first[blockIdx.x];
  return (a.n_tasks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
}
__device__ __forceinline__ HerkInst task_inst(const HerkArgs& a, const HerkTask& t) {
  return a.insts ? a.insts[t.inst] : a.in;
}
// Stages of a task: stage_t spectra each, twice that for double stages.
template <bool EIGHT>
__device__ __forceinline__ int stages_of(const HerkInst& in, int dbl) {
  const int ts = stage_t<EIGHT>() << dbl;
  return (in.tn + ts - 1) / ts;
}
// Accumulations of a task of nk stages (at least one, so that every role
// counts the same sequence) and the stages of one.
template <bool EIGHT>
__device__ __forceinline__ int piece_stages(int dbl) {
  return kPieceStages8 >> dbl;
}
template <bool EIGHT>
__device__ __forceinline__ int pieces_of(int nk, int dbl) {
  return EIGHT ? max(1, (nk + piece_stages<EIGHT>(dbl) - 1) / piece_stages<EIGHT>(dbl)) : 1;
}

// TCI: the tensor maps describe payload-order blocks ({byte row, channel,
// time}) and the unpack transposes.  EIGHT: 8-bit samples as FP16 operands.
template <bool LO_IS_REAL, bool EIGHT, bool TCI>
__global__ void __launch_bounds__(kRingThreads, 1)
    herk4_ring_kernel(const __grid_constant__ CUtensorMap tmap, const HerkArgs a) {
  constexpr int kT = stage_t<EIGHT>();             // spectra per stage
  constexpr int kPkRowBytes = kT;                  // packed bytes of a byte row in a stage
  extern __shared__ uint8_t dyn_raw[];
  // control block at the end of dynamic shared memory, ring from the first
  // 1024-byte boundary (swizzle atoms) up to it
  RingCtrl& sm = *reinterpret_cast<RingCtrl*>(
      dyn_raw + ((a.smem_bytes - (int)sizeof(RingCtrl)) & ~15));
  uint8_t* ring = align1024(dyn_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_my = my_task_count(a);  // tasks of this CTA; stage counts vary per array
  constexpr int slot_bytes = kSlotBytes;
  int ns = (int)(reinterpret_cast<uint8_t*>(&sm) - ring) / slot_bytes;
  if (ns > kMaxSlots) ns = kMaxSlots;
  if (ns < kGroups) {  // the host sizes shared memory for at least four slots
    if (tid == 0) atomicOr(a.status, kStTimeout);
    return;
  }
  volatile int* abort = &sm.abort;
  // every wait's budget, log2 cycles: w if the fault field sets it (only the
  // fault-injection tests shorten it), read from the parameter space at each wait
#define budget ((!EIGHT && (a.in.fault >> 24)) ? (a.in.fault >> 24) : 31)

  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&sm.full_t[s], 1);
      mbar_init(&sm.full_o[s], kGroupWarps);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.tmem_full[b], 1);
      mbar_init(&sm.tmem_empty[b], kEpiWarps);
      mbar_init(&sm.usum_full[b], kUnpackWarps);
      mbar_init(&sm.usum_empty[b], kEpiWarps);
    }
    mbar_init(&sm.done, 1);
    sm.abort = 0;
  }
  for (int i = tid; i < 2 * kMaxBlocks * 128; i += blockDim.x) (&sm.usum[0][0])[i] = 0;
  if (warp == 0) tmem_alloc(&sm.tmem_base, 512);
  fence_mbar_init();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t ring_addr = smem_addr(ring);
  // Each role branch resizes its registers first: a setmaxnreg whose branches
  // joined again would leave the compiler the smaller budget for all roles.
  if (warp == kTmaWarp) {
    // ------------------------------------------------------------ TMA loader
    regs_shrink<regs_other<LO_IS_REAL, EIGHT>()>();
    if (lane == 0 && n_my > 0) {
      if (!a.tmaps) tma_prefetch_desc(&tmap);
      // fault injection: this stage of CTA 0 is never loaded, so the waits
      // for it run out and the CTA unwinds with a timeout status
      const int skip = (blockIdx.x == 0 && (a.in.fault & 0xFFFFFF) > 0) ? (a.in.fault & 0xFFFFFF) - 1 : -1;
      int s = 0, m = 0, j = 0, k = 0, issued = 0;
      HerkTask task = my_task(a, 0);
      TaskGeom g = task_geom(task);
      HerkInst in = task_inst(a, task);
      const CUtensorMap* tm = a.tmaps ? &a.tmaps[task.inst] : &tmap;
      if (a.tmaps) tensormap_acquire(tm);
      int nk = stages_of<EIGHT>(in, g.dbl);
      bool stacked = in.rows_per_chan > 0;
      for (int S = 0;; ++S, ++k) {
        if (k == nk) {  // next task
          if (++j == n_my) break;
          k = 0;
          task = my_task(a, j);
          g = task_geom(task);
          in = task_inst(a, task);
          tm = a.tmaps ? &a.tmaps[task.inst] : &tmap;
          if (a.tmaps) tensormap_acquire(tm);
          nk = stages_of<EIGHT>(in, g.dbl);
          stacked = in.rows_per_chan > 0;
        }
        if (m > 0 && !mbar_wait(&sm.empty[s], (uint32_t)((m - 1) & 1), abort, budget)) {
          raise_timeout(a.status, abort);
          break;
        }
        const int t = in.t0 + k * (kT << g.dbl);
        const uint32_t dst0 = ring_addr + (uint32_t)(s * slot_bytes + 2 * kRPkBlock);
        if (S != skip) {
          mbar_expect_tx(&sm.full_t[s], (uint32_t)(2 * kRPkBlock));
          for (int u = 0; u < 2; ++u) {
            const uint32_t dst = dst0 + (uint32_t)(u * kRPkBlock);
            // unit u: block u, or the block's second time range
            // (byte rows of a 128-row block: 64 at 4 bits, 128 at 8 bits)
            const int row0 = stacked ? 0 : (kRPkBlock / kPkRowBytes) * slot_block(g, g.dbl ? 0 : u);
            const int tu = t + (g.dbl ? u * kT : 0);
            if (TCI)
              tma_load_3d(dst, tm, row0, task.chan0, tu, &sm.full_t[s]);
            else
              tma_load_3d(dst, tm, tu, row0, task.chan0, &sm.full_t[s]);
          }
        }
        ++issued;
        if (++s == ns) {
          s = 0;
          ++m;
        }
      }
      // never leave with copies in flight: wait for the last loads to land
      int never = 0;
      for (int S = issued - 1; S >= 0 && S >= issued - ns; --S)
        if (S != skip) mbar_wait(&sm.full_t[S % ns], (uint32_t)((S / ns) & 1), &never, budget);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    regs_shrink<regs_other<LO_IS_REAL, EIGHT>()>();
    if (lane == 0) {
      int s = 0, m = 0, v = 0;  // v: accumulations so far (tensor-memory buffer v & 1)
      bool ok = true;
      for (int j = 0; j < n_my && ok; ++j) {
        const HerkTask task = my_task(a, j);
        const TaskGeom g = task_geom(task);
        const int nk = stages_of<EIGHT>(task_inst(a, task), g.dbl);
        const int np = pieces_of<EIGHT>(nk, g.dbl);
        const uint32_t idesc = umma_idesc(0, 128, 128 * g.nb);
        for (int q = 0; q < np && ok; ++q, ++v) {
          const int b = v & 1;
          const int k0 = EIGHT ? q * piece_stages<EIGHT>(g.dbl) : 0;
          const int k1 = EIGHT ? min(nk, k0 + piece_stages<EIGHT>(g.dbl)) : nk;
          if (v >= 2 && !mbar_wait(&sm.tmem_empty[b], (uint32_t)(((v >> 1) - 1) & 1), abort, budget)) {
            raise_timeout(a.status, abort);
            ok = false;
            break;
          }
          tc_after_sync();
          const uint32_t d = tmem + (uint32_t)(b * 256);
          // the stages of this accumulation, DBL a constant (no per-MMA selects)
          auto issue = [&](auto DBL) {
            constexpr bool dbl = decltype(DBL)::value;
            for (int k = k0; k < k1; ++k) {
              if (!mbar_wait(&sm.full_o[s], (uint32_t)(m & 1), abort, budget)) {
                raise_timeout(a.status, abort);
                ok = false;
                break;
              }
              tc_after_sync();
              const uint32_t st = ring_addr + (uint32_t)(s * slot_bytes);
              // two-block task: A in slot a_slot, B in both; double stage:
              // A = B, the second time range in unit 1
              const uint64_t bdesc = umma_desc_sw128(st);
              const uint64_t adesc = dbl ? bdesc : umma_desc_sw128(st + (uint32_t)(g.a_slot * kROpBlock));
#pragma unroll
              for (int kk = 0; kk < (dbl ? 2 : 1) * kRKSteps; ++kk) {
                const uint64_t da = dbl ? bdesc + (uint64_t)((kk >> 2) * (kROpBlock >> 4) + 2 * (kk & 3))
                                        : adesc + 2 * kk;
                const uint64_t db = dbl ? da : bdesc + 2 * kk;
                if (EIGHT)
                  umma_f16(d, da, db, idesc, (k != k0 || kk != 0));
                else
                  umma_f8(d, da, db, idesc, (k != k0 || kk != 0));
              }
              umma_commit(&sm.empty[s]);
              if (++s == ns) {
                s = 0;
                ++m;
              }
            }
          };
          if (g.dbl)
            issue(std::true_type{});
          else
            issue(std::false_type{});
          if (ok) umma_commit(&sm.tmem_full[b]);
        }
      }
      umma_commit(&sm.done);
      int never = 0;
      if (!mbar_wait(&sm.done, 0, &never, budget)) raise_timeout(a.status, abort);
    }
    __syncwarp();
  } else if (warp < kUnpackWarps) {
    // ------------------------------------------------------------ unpackers
    regs_grow<regs_unpack<LO_IS_REAL, EIGHT>()>();
    const int grp = warp / kGroupWarps;
    const int gt = tid - grp * kGroupThreads;
    // Item geometry of this thread (four 16-byte items per packed block).
    //   4-bit, [c][row][t]: byte row g8 + 16 it' of the block, spectra
    //     16 chunk .. + 15 -> operand rows 2 (g8 + 16 it') and + 1, chunk
    //     `chunk`; payload order: rows 4 tq .. + 3, K chunk tc (see tci_t).
    //   8-bit, [c][row][t]: byte row r32 + 32 it', spectra 16 c4 .. + 15 ->
    //     operand row r32 + 32 it', chunks 2 c4 and 2 c4 + 1; payload order:
    //     rows 4 lane .. + 3, spectra 16 c8 .. + 15 gathered with the halves
    //     swapped on odd lanes (sw8), which keeps the stores free of bank
    //     conflicts (the gathers are: a row of 128 bytes per spectrum puts
    //     lane l's word in bank l).
    const int chunk = gt & 7, g8 = gt >> 3;
    const int tq = lane >> 1, tc = (lane + 2 * (gt >> 5)) & 7;
    const int c4 = gt & 3, r32 = gt >> 2;
    const int c8 = ((gt >> 5) + (lane >> 1)) & 3, sw8 = 8 * (lane & 1);
    const uint32_t src0 =
        ring_addr + (uint32_t)(EIGHT ? kPkRowBytes * r32 + 16 * c4 : kPkRowBytes * g8 + 16 * chunk);
    static_assert(kMaxBlocks == 2, "a stage holds at most two 128-row blocks");
    // later items add whole 8-row atoms, so the swizzle position stays the same
    const uint32_t dst_a = ring_addr + (EIGHT ? swz_offset(r32, 2 * c4) : swz_offset(2 * g8, chunk));
    const uint32_t dst_b = ring_addr + (EIGHT ? swz_offset(r32, 2 * c4 + 1) : swz_offset(2 * g8 + 1, chunk));
    bool ok = true;
    // next stage of this group, its slot s = S mod ns and use m = S / ns,
    // advanced by additions (kGroups <= ns)
    int S = grp, s = grp, m = 0;
    uint32_t bad = 0;  // 8-bit: a byte equal to 0x80 (-128) was seen
    int S0 = 0;  // first stage of task j
    for (int j = 0; j < n_my && ok; ++j) {
      const int b = j & 1;
      const HerkTask task = my_task(a, j);
      const TaskGeom g = task_geom(task);
      const int tn = task_inst(a, task).tn;
      const int kTs = kT << g.dbl;  // spectra per stage of this task
      const int S1 = S0 + (tn + kTs - 1) / kTs;
      const int nit = g.nblk * 4;
      int32_t sre[kItems], sim[kItems];
#pragma unroll
      for (int it = 0; it < kItems; ++it) sre[it] = sim[it] = 0;
      // this group's stages of task j: S0 <= S < S1 with S = grp (mod kGroups)
      for (; S < S1; S += kGroups) {
        const int k = S - S0;
        bool got = (m == 0 || mbar_wait(&sm.empty[s], (uint32_t)((m - 1) & 1), abort, budget)) &&
                   mbar_wait(&sm.full_t[s], (uint32_t)(m & 1), abort, budget);
        if (!got) raise_timeout(a.status, abort);
        const uint32_t so = (uint32_t)(s * slot_bytes);
        const bool tail = (k + 1) * kTs > tn;
        // The operands of unit 0 overlap neither unit's packed bytes
        // (operands [0, 16 KB) and [16, 32 KB), packed bytes [16, 32 KB)), so
        // they are written before the group barrier; the barrier then only
        // guards unit 1, whose operands cover packed bytes.
        const uint32_t pk = ring_addr + so + (uint32_t)(2 * kRPkBlock);
        uint32_t wv[16];  // this thread's 64 packed bytes of one block
        // load the items of block it
        auto load = [&](int it) {
          if constexpr (TCI) {  // 4 byte rows x 16 spectra, gathered
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              wv[jj] = lds32(pk + (uint32_t)(it * kRPkBlock) +
                             (uint32_t)(EIGHT ? (16 * c8 + (jj ^ sw8)) * 128 + 4 * lane
                                              : tci_t(tc, jj) * 64 + 4 * tq));
          } else {  // 4 items of 16 bytes: byte rows 16 (4-bit) or 32 (8-bit) apart
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint4 v = lds128(src0 + so + (uint32_t)(2 * kRPkBlock) +
                                     (uint32_t)(2048 * (4 * it + q)));
              wv[4 * q] = v.x, wv[4 * q + 1] = v.y, wv[4 * q + 2] = v.z, wv[4 * q + 3] = v.w;
            }
          }
        };
        // convert unit IT and write its operands (IT a constant: the row
        // sums stay in registers; a double stage's second time range adds to
        // the sums of unit 1 and is folded into unit 0's at the task's end)
        auto store = [&](auto IT) {
          constexpr int it = decltype(IT)::value;
          [[maybe_unused]] const uint32_t ob = ring_addr + so + (uint32_t)(it * kROpBlock);
          // masks of the unit's spectra (off: the unit's first spectrum in the task)
          uint32_t keep[4] = {~0u, ~0u, ~0u, ~0u};
          if (tail) {
            const int off = k * kTs + (it == 1 && g.dbl ? kT : 0);
            if (TCI && EIGHT)
              tci8_keep(c8, sw8, tn - off, keep);
            else if (TCI)
              tci_keep(tc, off, tn, keep);
            else
              time_keep(off + (EIGHT ? c4 : chunk) * 16, tn, keep);
          }
          if constexpr (TCI) {
#pragma unroll
            for (int gg = 0; gg < 4; ++gg)
              transpose4x4b(wv[4 * gg], wv[4 * gg + 1], wv[4 * gg + 2], wv[4 * gg + 3]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // TCI: byte row 4 t + u (t = lane or tq); otherwise item u
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = TCI ? wv[4 * q + u] : wv[4 * u + q];
            if constexpr (EIGHT) {
              uint32_t h[8];
              s8_to_f16(w, keep, h, bad);
              if constexpr (TCI) {
                const int r = 4 * lane + u, sw = sw8 >> 3;
                sts128(ob + swz_offset(r, 2 * c8 + sw), h[0], h[1], h[2], h[3]);
                sts128(ob + swz_offset(r, 2 * c8 + 1 - sw), h[4], h[5], h[6], h[7]);
              } else {
                const uint32_t o = so + (uint32_t)(it * kROpBlock + 4096 * u);  // 32 operand rows on
                sts128(dst_a + o, h[0], h[1], h[2], h[3]);
                sts128(dst_b + o, h[4], h[5], h[6], h[7]);
              }
            } else {
              uint32_t re[4], im[4];
              // always masked (all ones before the last stage): no branch inside the unrolled loop
              unpack16<LO_IS_REAL, true>(w, keep, re, im, sre[4 * it + u], sim[4 * it + u]);
              if constexpr (TCI) {
                const int r = 2 * (4 * tq + u);
                sts128(ob + swz_offset(r, tc), re[0], re[1], re[2], re[3]);
                sts128(ob + swz_offset(r + 1, tc), im[0], im[1], im[2], im[3]);
              } else {
                const uint32_t o = so + (uint32_t)(it * kROpBlock + 4096 * u);
                sts128(dst_a + o, re[0], re[1], re[2], re[3]);
                sts128(dst_b + o, im[0], im[1], im[2], im[3]);
              }
            }
          }
        };
        if (got) {
          load(0);
          store(std::integral_constant<int, 0>{});
          load(1);
        }
        // every packed byte of the stage is in registers or converted before
        // any is overwritten; the group leaves together if any wait failed
        if (!named_bar_and(2 + grp, kGroupThreads, got)) {
          ok = false;
          break;
        }
        store(std::integral_constant<int, 1>{});
        fence_smem_to_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.full_o[s]);
        s += kGroups;
        if (s >= ns) {
          s -= ns;
          ++m;
        }
      }
      if (!ok) break;
      S0 = S1;
      if constexpr (EIGHT) continue;  // signed operands: no row sums
      if (g.dbl) {  // both time ranges of a double stage are block 0's rows
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sre[u] += sre[4 + u];
          sim[u] += sim[4 + u];
        }
      }
      // publish this task's row sums once the buffer is free again
      const bool freed = j < 2 || mbar_wait(&sm.usum_empty[b], (uint32_t)(((j >> 1) - 1) & 1), abort, budget);
      if (!freed) raise_timeout(a.status, abort);
      if (!named_bar_and(2 + grp, kGroupThreads, freed)) break;
      if constexpr (TCI) {
        // the two lanes of a quad in a warp add, then one adds per warp
#pragma unroll
        for (int it = 0; it < kMaxBlocks; ++it) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (it < g.nblk) {
              const int r = sre[4 * it + u] + __shfl_xor_sync(0xFFFFFFFFu, sre[4 * it + u], 1);
              const int mm = sim[4 * it + u] + __shfl_xor_sync(0xFFFFFFFFu, sim[4 * it + u], 1);
              if ((lane & 1) == 0) {
                atomicAdd(&sm.usum[b][it * 128 + 2 * (4 * tq + u)], r);
                atomicAdd(&sm.usum[b][it * 128 + 2 * (4 * tq + u) + 1], mm);
              }
            }
          }
        }
      } else {
        publish_row_sums<kGroupThreads, kItems, 8>(sre, sim, nit, gt, sm.usum[b]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.usum_full[b]);
    }
    if (EIGHT && __any_sync(0xFFFFFFFFu, bad != 0) && lane == 0) atomicOr(a.status, kStRange);
  } else if (warp < kEpiWarp0) {
    regs_shrink<regs_other<LO_IS_REAL, EIGHT>()>();  // the two idle warps of the MMA / TMA warpgroup
  } else {
    // ------------------------------------------------------------ drain
    regs_shrink<regs_other<LO_IS_REAL, EIGHT>()>();
    const int quad = warp & 3, part = (warp - kEpiWarp0) >> 2;
    int2* scr = EIGHT ? a.scratch + (size_t)blockIdx.x * kHerkScratchInt2 : nullptr;
    int v = 0;
    bool ok = true;
    for (int j = 0; j < n_my && ok; ++j) {
      const HerkTask task = my_task(a, j);
      const HerkInst in = task_inst(a, task);
      const TaskGeom g = task_geom(task);
      const int np = pieces_of<EIGHT>(stages_of<EIGHT>(in, g.dbl), g.dbl);
      for (int q = 0; q < np; ++q, ++v) {
        const int b = v & 1;
        const uint32_t par = (uint32_t)((v >> 1) & 1);
        const bool got = mbar_wait(&sm.tmem_full[b], par, abort, budget) &&
                         (EIGHT || mbar_wait(&sm.usum_full[b], par, abort, budget));
        if (!got) raise_timeout(a.status, abort);
        if (!named_bar_and(1, kEpiWarps * 32, got)) {  // the drain warps leave together
          ok = false;
          break;
        }
        tc_after_sync();
        epilogue<EIGHT>(in, task, g, sm.usum[b], tmem + (uint32_t)(b * 256), quad, part,
                        kEpiWarps / 4, lane, q == 0, q == np - 1, scr);
        tc_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.tmem_empty[b]);
        if (!EIGHT) {
          // every drain warp has read the sums: clear them for task j + 2
          named_bar_sync(1, kEpiWarps * 32);
          for (int i = tid - kEpiWarp0 * 32; i < kMaxBlocks * 128; i += kEpiWarps * 32)
            sm.usum[b][i] = 0;
          __syncwarp();
          if (lane == 0) mbar_arrive(&sm.usum_empty[b]);
        }
      }
    }
  }
#undef budget
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 512);
}

// -------------------------------------------------------------- LDG kernel
// Warps 0..3 load, unpack and drain; warp 4 issues MMAs.
constexpr int kLdgThreads = 160;
constexpr int kLdgItems = kMaxBlocks * 4;

template <bool LO_IS_REAL>
__global__ void __launch_bounds__(kLdgThreads, 1) herk4_ldg_kernel(const HerkArgs args) {
  const HerkInst& a = args.in;
  extern __shared__ uint8_t dyn_raw[];
  __shared__ Ctrl sm;
  uint8_t* ops = align1024(dyn_raw);
  const HerkTask task = args.tasks[blockIdx.x];
  const TaskGeom g = task_geom(task);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool stacked = a.rows_per_chan > 0;
  const int stage_bytes = g.nblk * kOpBlockBytes;
  int nst = (args.smem_bytes - 1024) / stage_bytes;
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
               &sm.done, args.status, abort);
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
        raise_timeout(args.status, abort);
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
    if (!good && lane == 0) raise_timeout(args.status, abort);
    tc_after_sync();
    if (good && !*abort)
      epilogue<false>(a, task, g, sm.usum, tmem, warp & 3, 0, 1, lane, true, true, nullptr);
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

int ring_smem() {
  static int m = -1;
  if (m < 0)
    m = std::min(std::min(max_dyn_smem((const void*)herk4_ring_kernel<false, false, false>),
                          max_dyn_smem((const void*)herk4_ring_kernel<true, false, false>)),
                 max_dyn_smem((const void*)herk4_ring_kernel<false, true, false>));
    m = std::min(m, std::min(std::min(max_dyn_smem((const void*)herk4_ring_kernel<false, false, true>),
                                      max_dyn_smem((const void*)herk4_ring_kernel<true, false, true>)),
                             max_dyn_smem((const void*)herk4_ring_kernel<false, true, true>)));
  return m;
}

template <bool LO, bool EIGHT, bool TCI>
cudaError_t ring_launch(const HerkArgs& a, const CUtensorMap* tmap, int grid, cudaStream_t s) {
  // the attribute persists: set it once, so that launches captured into a
  // CUDA graph are plain stream work
  static int set_bytes = -1;
  if (set_bytes != a.smem_bytes) {
    cudaError_t e = set_smem(herk4_ring_kernel<LO, EIGHT, TCI>, a.smem_bytes);
    if (e != cudaSuccess) return e;
    set_bytes = a.smem_bytes;
  }
  herk4_ring_kernel<LO, EIGHT, TCI><<<grid, kRingThreads, a.smem_bytes, s>>>(*tmap, a);
  return cudaGetLastError();
}

}  // namespace

int device_sm_count() {
  static int count[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (count[dev] <= 0) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    count[dev] = nsm > 0 ? nsm : 1;
  }
  return count[dev];
}

int herk_ring_stage(int bits) { return bits == 8 ? stage_t<true>() : stage_t<false>(); }

int herk4_max_smem() {
  int m = max_dyn_smem((const void*)herk4_ldg_kernel<false>);
  m = std::min(m, max_dyn_smem((const void*)herk4_ldg_kernel<true>));
  return std::min(m, ring_smem());
}

cudaError_t herk4_launch(const HerkArgs& args, const CUtensorMap* tmap, int n_tasks,
                         cudaStream_t s, bool tci) {
  cudaError_t e;
  if (tmap || args.tmaps) {
    HerkArgs a = args;
    a.smem_bytes = ring_smem();
    // four slots, the control block and the alignment pad
    if (a.smem_bytes < kGroups * kSlotBytes + (int)sizeof(RingCtrl) + 1024)
      return cudaErrorInvalidConfiguration;
    int grid;
    if (a.cta_first) {
      grid = a.grid;
    } else {
      grid = std::min(n_tasks, device_sm_count());
      if (a.grid > 0) grid = std::min(grid, a.grid);
    }
    if (grid < 1) return cudaSuccess;
    if (a.bits == 8 && (!a.scratch || grid > a.scratch_ctas)) return cudaErrorInvalidValue;
    static const CUtensorMap unused{};  // batched launches read their maps from a.tmaps
    const CUtensorMap* m = tmap ? tmap : &unused;
    if (tci) {
      if (a.bits == 8) return ring_launch<false, true, true>(a, m, grid, s);
      return a.lo_is_real ? ring_launch<true, false, true>(a, m, grid, s)
                          : ring_launch<false, false, true>(a, m, grid, s);
    }
    if (a.bits == 8) return ring_launch<false, true, false>(a, m, grid, s);
    return a.lo_is_real ? ring_launch<true, false, false>(a, m, grid, s)
                        : ring_launch<false, false, false>(a, m, grid, s);
  }
  const HerkArgs& a = args;
  if (a.bits != 4 || tci) return cudaErrorInvalidValue;  // 8-bit rows and payload order take TMA
  if (a.lo_is_real) {
    if ((e = set_smem(herk4_ldg_kernel<true>, a.smem_bytes)) != cudaSuccess) return e;
    herk4_ldg_kernel<true><<<n_tasks, kLdgThreads, a.smem_bytes, s>>>(a);
  } else {
    if ((e = set_smem(herk4_ldg_kernel<false>, a.smem_bytes)) != cudaSuccess) return e;
    herk4_ldg_kernel<false><<<n_tasks, kLdgThreads, a.smem_bytes, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace xe
