// Corner turn (Sec. 2.1, "Transpose": [input, frequency] -> [frequency,
// input]) and FP64 normalisation of the integrated visibilities.
#include "xe_device.cuh"

namespace xe {
namespace {

// ---------------------------------------------------------------- corner turn
// in[t][g][k] -> out[k][g][t] for byte samples, through a 256 (t) x 128 (k)
// shared-memory tile of 32-bit words.  Word w of tile row r is stored at
// r * 32 + (w ^ 4 * (r >> 5)): the 16-byte chunk index is XOR-ed with the
// row's 32-row band, which makes both the row-wise stores and the
// column-wise loads below free of bank conflicts without padding.
constexpr int kTT = 256, kTK = 128;

__device__ __forceinline__ void transpose4x4(uint32_t& a0, uint32_t& a1, uint32_t& a2,
                                             uint32_t& a3) {
  const uint32_t t0 = __byte_perm(a0, a1, 0x5140), t1 = __byte_perm(a0, a1, 0x7362);
  const uint32_t t2 = __byte_perm(a2, a3, 0x5140), t3 = __byte_perm(a2, a3, 0x7362);
  a0 = __byte_perm(t0, t2, 0x5410);
  a1 = __byte_perm(t0, t2, 0x7632);
  a2 = __byte_perm(t1, t3, 0x5410);
  a3 = __byte_perm(t1, t3, 0x7632);
}

__device__ __forceinline__ void ld32B(const uint8_t* p, uint32_t (&r)[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "l"(p));
}
__device__ __forceinline__ void st32B(uint8_t* p, const uint32_t (&r)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

__device__ __forceinline__ int tile_word(int row, int w) { return row * 32 + (w ^ ((row >> 5) << 2)); }

// barrier of one 256-thread group (id 0 is the whole CTA of a 256-thread launch)
__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory");
}

// Store phase of a tile held in `tile`: each thread transposes 4 x 32 bytes
// in registers and writes 32-byte pieces of [k][g][t] rows.
__device__ __forceinline__ void turn_tile_store(uint8_t* __restrict__ out, int T, int K, int G,
                                                long long os, int pair_rows, int t0, int k0,
                                                int g, const uint32_t* tile, int tid, bool full) {
  const int warp = tid >> 5, lane = tid & 31;
  // store: thread = 4 consecutive k (word kq) x 32 consecutive t (segment ts);
  // the eight lanes of a k-quad cover one 256-byte stretch of each output row
  const int kq = 4 * warp + (lane >> 3), ts = lane & 7;
  uint32_t a[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) a[j] = tile[tile_word(ts * 32 + j, kq)];
#pragma unroll
  for (int j = 0; j < 32; j += 4) transpose4x4(a[j], a[j + 1], a[j + 2], a[j + 3]);
  // a[4w + c] now holds t = ts*32 + 4w .. +3 of k = 4 kq + c
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int k = k0 + 4 * kq + c;
    const int tb = t0 + ts * 32;
    const long long row =
        pair_rows ? ((long long)(k >> 1) * G + g) * 2 + (k & 1) : (long long)k * G + g;
    uint8_t* o = out + row * os + tb;
    if (full) {
      const uint32_t r[8] = {a[c], a[4 + c], a[8 + c], a[12 + c],
                             a[16 + c], a[20 + c], a[24 + c], a[28 + c]};
      st32B(o, r);
    } else if (k < K) {
      for (int b = 0; b < 32; ++b)
        if (tb + b < T) o[b] = (uint8_t)(a[4 * (b >> 2) + c] >> ((b & 3) * 8));
    }
  }
}


// One tile: 256 threads (tid 0..255) move spectra t0 .. t0+255 of byte rows
// k0 .. k0+127 of group g through `tile`, meeting at barrier `bar`.  Input
// row (t, g) starts at in + (t G + g) ks: ks = K, or more for a range of
// rows cut from a wider block.
__device__ __forceinline__ void turn_tile(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                          int T, int G, int K, long long ks, long long os, int vec_ok,
                                          int pair_rows, int t0, int k0, int g, uint32_t* tile,
                                          int tid, int bar) {
  const bool full = vec_ok && t0 + kTT <= T && k0 + kTK <= K;
  // load: 256 rows x 128 bytes as 32-byte pieces, four per thread, all
  // issued before any of them is stored
  if (full) {
    uint32_t v[4][8];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = it * 256 + tid, r = e >> 2, p = e & 3;
      ld32B(in + ((long long)(t0 + r) * G + g) * ks + k0 + 32 * p, v[it]);
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = it * 256 + tid, r = e >> 2, p = e & 3;
      // odd rows store their second 16-byte half first: the two rows of a
      // quarter-warp then hit disjoint banks
      const bool odd = r & 1;
      const uint4 lo = make_uint4(v[it][0], v[it][1], v[it][2], v[it][3]);
      const uint4 hi = make_uint4(v[it][4], v[it][5], v[it][6], v[it][7]);
      *reinterpret_cast<uint4*>(&tile[tile_word(r, 8 * p + (odd ? 4 : 0))]) = odd ? hi : lo;
      *reinterpret_cast<uint4*>(&tile[tile_word(r, 8 * p + (odd ? 0 : 4))]) = odd ? lo : hi;
    }
  } else {
    for (int e = tid; e < kTT * 32; e += 256) {
      const int r = e >> 5, w = e & 31;
      uint32_t x = 0;
      if (t0 + r < T) {
        const long long off = ((long long)(t0 + r) * G + g) * ks + k0 + 4 * w;
        for (int b = 0; b < 4; ++b)
          if (k0 + 4 * w + b < K) x |= (uint32_t)in[off + b] << (8 * b);
      }
      tile[tile_word(r, w)] = x;
    }
  }
  group_bar(bar);
  turn_tile_store(out, T, K, G, os, pair_rows, t0, k0, g, tile, tid, full);
}

__global__ void __launch_bounds__(256, 4) turn_kernel(const uint8_t* __restrict__ in,
                                                      uint8_t* __restrict__ out, int T, int G,
                                                      int K, long long ks, long long os,
                                                      int vec_ok, int pair_rows) {
  __shared__ __align__(16) uint32_t tile[kTT * 32];
  turn_tile(in, out, T, G, K, ks, os, vec_ok, pair_rows, blockIdx.x * kTT, blockIdx.y * kTK,
            blockIdx.z, tile, threadIdx.x, 0);
}

// The same tiles from a fixed number of CTAs, one per SM, for a corner turn
// confined to a few SMs while the cross-multiply of the previous block holds
// the others.  Confined to a few SMs, the turn is bound by the bytes each SM
// keeps in flight, not by HBM: each of the kTurnGroups 256-thread groups of a
// CTA walks its own tiles through kTurnBufs 32 KB buffers, with the 16-byte
// cp.async copies of the next kTurnBufs - 1 tiles in flight while one tile is
// transposed and stored.  Edge tiles take the byte path synchronously.
#ifndef XE_TURN_GROUPS
#define XE_TURN_GROUPS 3
#endif
#ifndef XE_TURN_BUFS
#define XE_TURN_BUFS 2
#endif
constexpr int kTurnGroups = XE_TURN_GROUPS;
constexpr int kTurnBufs = XE_TURN_BUFS;
constexpr int kTurnAhead = kTurnBufs - 1;  // tiles in flight per group
constexpr int kTileWords = kTT * 32;
static_assert(kTurnBufs >= 2 && kTurnAhead <= 7, "cp.async.wait_group takes 0..7 here");
static_assert(kTurnGroups * kTurnBufs * kTileWords * 4 <= 227 * 1024,
              "the buffers must fit in one CTA's shared memory");

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t* dst, const uint8_t* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// Issue the copies of a full tile into `tile`, the same word placement as
// the register path of turn_tile: bytes 16c .. 16c+15 of a row go to words
// 4c .. 4c+3.  Consecutive threads take consecutive 16-byte chunks, so each
// warp instruction covers four whole 128-byte rows (every sector requested
// once, not half of it by each of two instructions).
__device__ __forceinline__ void tile_prefetch(const uint8_t* __restrict__ in, int G, long long ks, int t0,
                                              int k0, int g, uint32_t* tile, int tid) {
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int e = it * 256 + tid, r = e >> 3, c = e & 7;
    cp_async16(&tile[tile_word(r, 4 * c)], in + ((long long)(t0 + r) * G + g) * ks + k0 + 16 * c);
  }
}

__global__ void __launch_bounds__(256 * kTurnGroups, 1)
    turn_persist_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int T, int G,
                        int K, long long ks, long long os, int vec_ok, int pair_rows) {
  extern __shared__ __align__(16) uint32_t tiles[];
  const int grp = threadIdx.x >> 8, tid = threadIdx.x & 255, bar = 1 + grp;
  uint32_t* const mine = tiles + kTurnBufs * grp * kTileWords;  // this group's buffers
  // tile indices in 32 bits (the host keeps their count below 2^31): the
  // per-tile index arithmetic is a visible share of this kernel's issue slots
  const unsigned gx = (unsigned)(T + kTT - 1) / kTT, gy = (unsigned)(K + kTK - 1) / kTK;
  const unsigned n = gx * gy * (unsigned)G;
  const unsigned stride = gridDim.x * kTurnGroups;
  auto coords = [&](unsigned w, int& t0, int& k0, int& g) {
    const unsigned r = w / gx, q = r / gy;
    t0 = (int)(w - r * gx) * kTT;
    k0 = (int)(r - q * gy) * kTK;
    g = (int)q;
  };
  auto is_full = [&](int t0, int k0) { return vec_ok && t0 + kTT <= T && k0 + kTK <= K; };
  // copies of full tile w into buffer b; one commit group per tile, empty
  // for edge tiles and past the end, so that group i is always tile i
  auto prefetch = [&](unsigned w, int b) {
    if (w < n) {
      int t0, k0, g;
      coords(w, t0, k0, g);
      if (is_full(t0, k0)) tile_prefetch(in, G, ks, t0, k0, g, mine + b * kTileWords, tid);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  unsigned w = blockIdx.x * kTurnGroups + grp;
#pragma unroll
  for (int d = 0; d < kTurnAhead; ++d) prefetch(w + d * stride, d);
  // tile i sits in buffer i mod kTurnBufs; tile i + kTurnAhead goes into the
  // buffer of tile i - 1, released by the barrier that ended its iteration
  for (int b = 0; w < n; w += stride) {
    const int bn = b == 0 ? kTurnBufs - 1 : b - 1;
    prefetch(w + kTurnAhead * stride, bn);
    cp_async_wait<kTurnAhead>();  // the copies of this tile are in
    int t0, k0, g;
    coords(w, t0, k0, g);
    uint32_t* tile = mine + b * kTileWords;
    if (is_full(t0, k0)) {
      group_bar(bar);
      turn_tile_store(out, T, K, G, os, pair_rows, t0, k0, g, tile, tid, true);
    } else {
      turn_tile(in, out, T, G, K, ks, os, vec_ok, pair_rows, t0, k0, g, tile, tid, bar);
    }
    group_bar(bar);
    if (++b == kTurnBufs) b = 0;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- packet turn
// A block assembled in packet order -- [slot][fid][xid][8 spectra][chans_pkt
// x inputs_pkt bytes] -- becomes the X-engine's [c][i][t] rows.  For one
// (fid, xid) and 128 consecutive bytes k of a packet row, the spectra
// t = 8 slot + tt form a 256 x 128 tile like the corner turn's, except that
// a tile row's address steps by the packet stream stride every 8 spectra and
// each byte k names its own output row: channel xid chans_pkt + k / inputs_pkt,
// input fid inputs_pkt + k mod inputs_pkt.
struct PktGeom {
  int n_fids, inputs_pkt, n_xids, chans_pkt, T;
  long long os;
  int vec_ok;
};

__global__ void __launch_bounds__(256, 4) pkt_turn_kernel(const uint8_t* __restrict__ in,
                                                          uint8_t* __restrict__ out, PktGeom q) {
  __shared__ __align__(16) uint32_t tile[kTT * 32];
  const int rowb = q.chans_pkt * q.inputs_pkt;           // bytes of one spectrum of a packet
  const long long P = 8LL * rowb;                        // payload bytes
  const long long slot_stride = (long long)q.n_fids * q.n_xids * P;
  const int t0 = blockIdx.x * kTT, k0 = blockIdx.y * kTK;
  const int stream = blockIdx.z, fid = stream / q.n_xids, xid = stream % q.n_xids;
  const int N = q.n_fids * q.inputs_pkt;
  const uint8_t* base = in + ((long long)fid * q.n_xids + xid) * P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool full = q.vec_ok && t0 + kTT <= q.T && k0 + kTK <= rowb;
  if (full) {
    uint32_t v[4][8];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = it * 256 + tid, r = e >> 2, p = e & 3, t = t0 + r;
      ld32B(base + (long long)(t >> 3) * slot_stride + (long long)(t & 7) * rowb + k0 + 32 * p, v[it]);
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = it * 256 + tid, r = e >> 2, p = e & 3;
      const bool odd = r & 1;
      const uint4 lo = make_uint4(v[it][0], v[it][1], v[it][2], v[it][3]);
      const uint4 hi = make_uint4(v[it][4], v[it][5], v[it][6], v[it][7]);
      *reinterpret_cast<uint4*>(&tile[tile_word(r, 8 * p + (odd ? 4 : 0))]) = odd ? hi : lo;
      *reinterpret_cast<uint4*>(&tile[tile_word(r, 8 * p + (odd ? 0 : 4))]) = odd ? lo : hi;
    }
  } else {
    for (int e = tid; e < kTT * 32; e += 256) {
      const int r = e >> 5, w = e & 31, t = t0 + r;
      uint32_t x = 0;
      if (t < q.T) {
        const uint8_t* src = base + (long long)(t >> 3) * slot_stride + (long long)(t & 7) * rowb;
        for (int b = 0; b < 4; ++b)
          if (k0 + 4 * w + b < rowb) x |= (uint32_t)src[k0 + 4 * w + b] << (8 * b);
      }
      tile[tile_word(r, w)] = x;
    }
  }
  __syncthreads();
  const int kq = 4 * warp + (lane >> 3), ts = lane & 7;
  uint32_t a[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) a[j] = tile[tile_word(ts * 32 + j, kq)];
#pragma unroll
  for (int j = 0; j < 32; j += 4) transpose4x4(a[j], a[j + 1], a[j + 2], a[j + 3]);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int k = k0 + 4 * kq + c;
    if (k >= rowb) continue;
    const int ch = xid * q.chans_pkt + k / q.inputs_pkt, inp = fid * q.inputs_pkt + k % q.inputs_pkt;
    const int tb = t0 + ts * 32;
    uint8_t* o = out + ((long long)ch * N + inp) * q.os + tb;
    if (full) {
      const uint32_t r[8] = {a[c], a[4 + c], a[8 + c], a[12 + c],
                             a[16 + c], a[20 + c], a[24 + c], a[28 + c]};
      st32B(o, r);
    } else {
      for (int b = 0; b < 32; ++b)
        if (tb + b < q.T) o[b] = (uint8_t)(a[4 * (b >> 2) + c] >> ((b & 3) * 8));
    }
  }
}

// ---------------------------------------------------------------- plane split
// out[r][p][t] = in[r][t][p] for 8-bit complex samples: 16 samples (32 bytes)
// per thread become 16 real and 16 imaginary bytes.
__global__ void split_planes_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                    long long rows, int T, long long os, int vec_ok) {
  const int per_row = (T + 15) / 16;
  const long long total = rows * per_row;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / per_row;
    const int t = (int)(e - r * per_row) * 16;
    const uint8_t* src = in + (r * T + t) * 2;
    uint8_t* dre = out + (2 * r) * os + t;
    uint8_t* dim = dre + os;
    if (vec_ok && t + 16 <= T) {
      const uint4 a = *reinterpret_cast<const uint4*>(src);
      const uint4 b = *reinterpret_cast<const uint4*>(src + 16);
      // even bytes are real parts, odd bytes imaginary parts
      *reinterpret_cast<uint4*>(dre) =
          make_uint4(__byte_perm(a.x, a.y, 0x6420), __byte_perm(a.z, a.w, 0x6420),
                     __byte_perm(b.x, b.y, 0x6420), __byte_perm(b.z, b.w, 0x6420));
      *reinterpret_cast<uint4*>(dim) =
          make_uint4(__byte_perm(a.x, a.y, 0x7531), __byte_perm(a.z, a.w, 0x7531),
                     __byte_perm(b.x, b.y, 0x7531), __byte_perm(b.z, b.w, 0x7531));
    } else {
      for (int k = 0; k < 16 && t + k < T; ++k) {
        dre[k] = src[2 * k];
        dim[k] = src[2 * k + 1];
      }
    }
  }
}

// ---------------------------------------------------------------- normalise
__global__ void normalise_kernel(const int64_t* __restrict__ acc, double* __restrict__ rho,
                                 uint8_t* __restrict__ zero_flag, int n, long long nbl,
                                 long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / nbl, b = e % nbl;
    long long i = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > b) --i;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    const long long j = b - i * (i + 1) / 2;
    const int64_t* v = acc + c * nbl * 2;
    const double pii = (double)v[2 * (i * (i + 1) / 2 + i)];
    const double pjj = (double)v[2 * (j * (j + 1) / 2 + j)];
    const double den2 = pii * pjj;
    double re = 0.0, im = 0.0;
    if (den2 != 0.0) {
      const double den = sqrt(den2);
      re = (double)v[2 * b] / den;
      im = (double)v[2 * b + 1] / den;
    }
    rho[2 * e] = re;
    rho[2 * e + 1] = im;
    if (zero_flag) zero_flag[e] = den2 == 0.0 ? 1 : 0;
  }
  (void)n;
}

}  // namespace

cudaError_t turn_launch(const uint8_t* in, uint8_t* out, int T, int G, int K, long long out_stride,
                        cudaStream_t s, bool pair_rows, int persist_ctas) {
  return turn_launch_strided(in, out, T, G, K, K, out_stride, s, pair_rows, persist_ctas);
}

cudaError_t turn_launch_strided(const uint8_t* in, uint8_t* out, int T, int G, int K,
                                long long in_stride, long long out_stride, cudaStream_t s,
                                bool pair_rows, int persist_ctas) {
  if (in_stride < K) return cudaErrorInvalidValue;
  const int vec_ok = (K % 32 == 0) && (in_stride % 32 == 0) && (T % 32 == 0) && (out_stride % 32 == 0) &&
                     (reinterpret_cast<uintptr_t>(in) % 32 == 0) &&
                     (reinterpret_cast<uintptr_t>(out) % 32 == 0);
  const long long n_tiles = (long long)((T + kTT - 1) / kTT) * ((K + kTK - 1) / kTK) * G;
  if (persist_ctas > 0 && n_tiles + (long long)persist_ctas * kTurnGroups * kTurnBufs < (1LL << 31)) {
    constexpr int smem = kTurnGroups * kTurnBufs * kTileWords * (int)sizeof(uint32_t);
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(turn_persist_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    turn_persist_kernel<<<persist_ctas, 256 * kTurnGroups, smem, s>>>(
        in, out, T, G, K, in_stride, out_stride, vec_ok, pair_rows ? 1 : 0);
    return cudaGetLastError();
  }
  dim3 grid((T + kTT - 1) / kTT, (K + kTK - 1) / kTK, G);
  turn_kernel<<<grid, 256, 0, s>>>(in, out, T, G, K, in_stride, out_stride, vec_ok, pair_rows ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t split_planes_launch(const uint8_t* in, uint8_t* out, long long rows, int T,
                                long long out_stride, cudaStream_t s) {
  const int vec_ok = (T % 16 == 0) && (out_stride % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(out) % 16 == 0);
  const long long total = rows * ((T + 15) / 16);
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  split_planes_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, rows, T, out_stride, vec_ok);
  return cudaGetLastError();
}

cudaError_t pkt_turn_launch(const uint8_t* in, uint8_t* out, int n_fids, int inputs_pkt, int n_xids,
                            int chans_pkt, int T, long long out_stride, cudaStream_t s) {
  PktGeom q{n_fids, inputs_pkt, n_xids, chans_pkt, T, out_stride, 0};
  const int rowb = chans_pkt * inputs_pkt;
  q.vec_ok = rowb % 32 == 0 && out_stride % 32 == 0 && T % 32 == 0 &&
             reinterpret_cast<uintptr_t>(in) % 32 == 0 && reinterpret_cast<uintptr_t>(out) % 32 == 0;
  dim3 grid((T + kTT - 1) / kTT, (rowb + kTK - 1) / kTK, n_fids * n_xids);
  pkt_turn_kernel<<<grid, 256, 0, s>>>(in, out, q);
  return cudaGetLastError();
}

bool needs_turn(int layout, int bits) { return layout != 2 || bits == 8; }

bool turn_can_persist(int layout, int bits) { return needs_turn(layout, bits) && layout != 2; }

cudaError_t turn_rows(const uint8_t* in, uint8_t* out, int layout, int bits, int n_inputs,
                      int n_chans, int n_time, long long out_stride, cudaStream_t s,
                      int persist_ctas) {
  const int N = n_inputs, C = n_chans, T = n_time;
  const bool eight = bits == 8;
  const int R = eight ? 2 * N : N;
  // [t][c][i] is one transpose of a T x (C N) byte matrix, [t][i][c] is N
  // transposes of T x C.  8-bit samples are byte pairs: [t][c][i][p] turns as
  // T x (C 2N); [t][i][c][p] as N transposes of T x 2C with each (c, p) row
  // sent to row (c, i, p); [c][i][t][p] only splits the planes.
  if (layout == 0) return turn_launch(in, out, T, 1, C * R, out_stride, s, false, persist_ctas);
  if (layout == 1)
    return eight ? turn_launch(in, out, T, N, 2 * C, out_stride, s, true, persist_ctas)
                 : turn_launch(in, out, T, N, C, out_stride, s, false, persist_ctas);
  if (eight) return split_planes_launch(in, out, (long long)C * N, T, out_stride, s);
  return cudaSuccess;
}

cudaError_t turn_rows_chans(const uint8_t* in, uint8_t* out, int layout, int bits, int n_inputs,
                            int n_chans, int n_time, int c0, int c1, long long out_stride,
                            cudaStream_t s, int persist_ctas) {
  const int N = n_inputs, C = n_chans, T = n_time;
  if (bits != 4 || c0 < 0 || c1 > C || c0 >= c1) return cudaErrorInvalidValue;
  // channels c0 .. c1-1 are output rows c N + i for c0 <= c < c1
  uint8_t* o = out + (long long)c0 * N * out_stride;
  if (layout == 0)  // [t][c][i]: bytes c0 N .. c1 N of each spectrum
    return turn_launch_strided(in + (long long)c0 * N, o, T, 1, (c1 - c0) * N, (long long)C * N,
                               out_stride, s, false, persist_ctas);
  if (layout == 1)  // [t][i][c]: bytes c0 .. c1 of each (spectrum, input) row
    return turn_launch_strided(in + c0, o, T, N, c1 - c0, C, out_stride, s, false, persist_ctas);
  return cudaErrorInvalidValue;
}

// One thread: copy the status word into a slot of pinned host memory
// (written through its device mapping) and clear it, in stream order.
__global__ void take_status_kernel(int* status, int* host_slot) {
  *host_slot = *status;
  *status = 0;
}

cudaError_t take_status_launch(int* status, int* host_slot, cudaStream_t s) {
  take_status_kernel<<<1, 1, 0, s>>>(status, host_slot);
  return cudaGetLastError();
}

cudaError_t normalise_launch(const int64_t* acc, double* rho, uint8_t* zero_flag, int n_inputs,
                             int n_chans, cudaStream_t s) {
  const long long nbl = (long long)n_inputs * (n_inputs + 1) / 2;
  const long long total = nbl * n_chans;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  normalise_kernel<<<(unsigned)blocks, 256, 0, s>>>(acc, rho, zero_flag, n_inputs, nbl, total);
  return cudaGetLastError();
}

}  // namespace xe
