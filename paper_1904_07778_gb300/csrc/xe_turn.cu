// Corner turn (Sec. 2.1, "Transpose": [input, frequency] -> [frequency,
// input]) and FP64 normalisation of the integrated visibilities.
#include "xe_device.cuh"

namespace xe {
namespace {

// ---------------------------------------------------------------- corner turn
// in[t][g][k] -> out[k][g][t] for byte samples, through a 256 (t) x 128 (k)
// shared-memory tile: 16-byte coalesced loads along k, a 4 x 4 byte
// transpose in registers, 16-byte stores along t.
constexpr int kTT = 256, kTK = 128, kPitch = 36;  // pitch in 32-bit words (16-byte aligned)

__device__ __forceinline__ void transpose4x4(uint32_t& a0, uint32_t& a1, uint32_t& a2,
                                             uint32_t& a3) {
  const uint32_t t0 = __byte_perm(a0, a1, 0x5140), t1 = __byte_perm(a0, a1, 0x7362);
  const uint32_t t2 = __byte_perm(a2, a3, 0x5140), t3 = __byte_perm(a2, a3, 0x7362);
  a0 = __byte_perm(t0, t2, 0x5410);
  a1 = __byte_perm(t0, t2, 0x7632);
  a2 = __byte_perm(t1, t3, 0x5410);
  a3 = __byte_perm(t1, t3, 0x7632);
}

__global__ void __launch_bounds__(256) turn_kernel(const uint8_t* __restrict__ in,
                                                   uint8_t* __restrict__ out, int T, int G, int K,
                                                   long long os, int vec_ok) {
  __shared__ __align__(16) uint32_t tile[kTT * kPitch];
  const int t0 = blockIdx.x * kTT, k0 = blockIdx.y * kTK, g = blockIdx.z;
  const int tid = threadIdx.x;
  const bool full = vec_ok && t0 + kTT <= T && k0 + kTK <= K;
  // load: 256 rows of 128 bytes
#pragma unroll 4
  for (int e = tid; e < kTT * 8; e += 256) {
    const int r = e >> 3, q = e & 7;
    const long long off = ((long long)(t0 + r) * G + g) * K + k0 + 16 * q;
    uint4 v;
    if (full) {
      v = ld_stream16(in + off);
    } else {
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (t0 + r < T)
        for (int b = 0; b < 16; ++b)
          if (k0 + 16 * q + b < K) w[b >> 2] |= (uint32_t)in[off + b] << ((b & 3) * 8);
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    *reinterpret_cast<uint4*>(&tile[r * kPitch + 4 * q]) = v;
  }
  __syncthreads();
  // store: thread = (4 consecutive k, 32 consecutive t)
  const int kq = tid & 31, ts = tid >> 5;
  uint32_t a[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) a[j] = tile[(ts * 32 + j) * kPitch + kq];
#pragma unroll
  for (int j = 0; j < 32; j += 4) transpose4x4(a[j], a[j + 1], a[j + 2], a[j + 3]);
  // after the transposes a[4w + c] holds t = ts*32 + 4w .. +3 of k = 4 kq + c
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int k = k0 + 4 * kq + c;
    const int tb = t0 + ts * 32;
    uint8_t* o = out + ((long long)k * G + g) * os + tb;
    if (full) {
      *reinterpret_cast<uint4*>(o) = make_uint4(a[c], a[4 + c], a[8 + c], a[12 + c]);
      *reinterpret_cast<uint4*>(o + 16) = make_uint4(a[16 + c], a[20 + c], a[24 + c], a[28 + c]);
    } else if (k < K) {
      for (int b = 0; b < 32; ++b)
        if (tb + b < T) o[b] = (uint8_t)(a[4 * (b >> 2) + c] >> ((b & 3) * 8));
    }
  }
}

// ---------------------------------------------------------------- normalise
__global__ void normalise_kernel(const int64_t* __restrict__ acc, double* __restrict__ rho,
                                 int n, long long nbl, long long total) {
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
  }
  (void)n;
}

}  // namespace

cudaError_t turn_launch(const uint8_t* in, uint8_t* out, int T, int G, int K, long long out_stride,
                        cudaStream_t s) {
  const int vec_ok = (K % 16 == 0) && (T % 16 == 0) && (out_stride % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(out) % 16 == 0);
  dim3 grid((T + kTT - 1) / kTT, (K + kTK - 1) / kTK, G);
  turn_kernel<<<grid, 256, 0, s>>>(in, out, T, G, K, out_stride, vec_ok);
  return cudaGetLastError();
}

cudaError_t normalise_launch(const int64_t* acc, double* rho, int n_inputs, int n_chans,
                             cudaStream_t s) {
  const long long nbl = (long long)n_inputs * (n_inputs + 1) / 2;
  const long long total = nbl * n_chans;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  normalise_kernel<<<(unsigned)blocks, 256, 0, s>>>(acc, rho, n_inputs, nbl, total);
  return cudaGetLastError();
}

}  // namespace xe
