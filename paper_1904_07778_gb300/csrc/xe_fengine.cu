// GPU F-engine (Sec. 2.1): polyphase filter bank, the FFT of two real
// inputs as one complex transform with the Eq. 2 separation, the 18-bit
// output, and the equaliser / requantiser to packed fix_4_3 codes -- one
// fused kernel whose output is the X-engine's input.
//
// A CTA takes one input pair (2k, 2k+1) and a group of 32 consecutive
// spectra.  Per spectrum, M/8 threads (an "FFT unit"; a CTA holds
// 2048/M units for M <= 2048) filter 8 consecutive samples each, store
// z[n] = y_2k[n] + j y_2k+1[n] in padded shared memory, and run an in-place
// Stockham FFT (radix-8 passes, then one radix-2 or radix-4 pass).  The
// separated spectra are rounded to 18 bits, equalised, packed, and staged
// as [channel][input][spectrum] so that the group leaves as 32-byte runs of
// the X-engine's [c][i][t] order: the corner turn happens here.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fengine.h"
#include "xe_internal.h"
#include "xengine.h"

struct fe_ctx {
  int n_inputs = 0, n_chans = 0, taps = 0, shift = 0;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* h = nullptr;         // [taps * M] prototype filter
  float2* w = nullptr;        // [M] exp(-2 pi j n / M)
  uint32_t* gain = nullptr;   // [C][N]
};

namespace xe {
namespace {

constexpr int kFeGroup = 32;  // spectra per CTA
// spectra a unit transforms side by side (they share the pass barriers);
// three measured no faster than two
__host__ __device__ constexpr int fe_nb(int) { return 2; }

struct FeArgs {
  const int8_t* adc;
  long long adc_stride;
  const float* h;
  const float2* w;
  const uint32_t* gain;
  uint8_t* out;
  long long out_stride;
  int32_t* v18;
  float* spec;
  unsigned long long* power;
  int n_inputs, n_spectra, taps, layout;
  int lo_is_real, vec_in, vec_out;
  float scale;  // 2^-(shift + 1): Eq. 2's halving and the 18-bit scaling
};

__host__ __device__ constexpr int fe_threads(int logm) {
  return (1 << logm) / 8 > 256 ? (1 << logm) / 8 : 256;
}
// one float2 of padding per 16: consecutive runs of 16 (half a warp's
// 8-byte accesses) stay contiguous, stride-8 runs spread over the banks
__host__ __device__ constexpr int fe_pad(int n) { return n + (n >> 4); }
// Twiddles of the radix-8 passes at Ns = 8 and Ns = 64 in shared memory,
// [k][j-1] for k < Ns: they depend only on lt mod Ns, so the table is small
// (threads with equal k read the same entry) and frees the registers they
// would take.
constexpr int kTwTable = (8 + 64) * 7;
template <int LOGM>
constexpr size_t fe_smem_bytes() {
  constexpr int M = 1 << LOGM;
  constexpr int units = fe_threads(LOGM) / (M / 8);
  return (size_t)fe_nb(LOGM) * units * fe_pad(M) * sizeof(float2) + (size_t)(M / 2) * 2 * kFeGroup +
         kTwTable * sizeof(float2);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_mj(float2 a) { return make_float2(a.y, -a.x); }  // a * (-j)

// Y[k] = sum_n x[n] (-j)^(nk)
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_mj(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

// X[k] = sum_n a[n] W8^(nk), W8 = exp(-j pi / 4): two DFT4s of the even and
// odd samples, joined with W8^k.
__device__ __forceinline__ void dft8(float2 (&a)[8]) {
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  o1 = make_float2(r * (o1.x + o1.y), r * (o1.y - o1.x));    // * (1 - j) / sqrt2
  o2 = mul_mj(o2);                                           // * -j
  o3 = make_float2(r * (o3.y - o3.x), -r * (o3.x + o3.y));   // * (-1 - j) / sqrt2
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1);
  a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3);
  a[7] = csub(e3, o3);
}

// Twiddles of one Stockham pass for one thread: butterfly b = lt + r M/8
// multiplies its input j by exp(-2 pi j (b mod Ns) j / (Ns R)), for
// j = 1 .. R-1.  They do not depend on the spectrum, so a thread loads them
// once (from the FP64-rounded table) and keeps them in registers.
template <int M, int R>
__device__ __forceinline__ void load_twiddles(float2 (&tw)[7], int lt, int Ns,
                                              const float2* __restrict__ w) {
  constexpr int B = 8 / R;
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const int k = (lt + r * (M / 8)) & (Ns - 1);
    const int step = k * (M / (R * Ns));
#pragma unroll
    for (int j = 1; j < R; ++j) tw[r * (R - 1) + j - 1] = __ldg(&w[j * step]);
  }
}

// One Stockham pass of radix R over NB independent M-point transforms held
// in zs[] (padded indices): butterfly b reads z[b + j M/R], applies its
// twiddles, and writes the R outputs to (b div Ns) Ns R + (b mod Ns) + r Ns.
// Each of the M/8 threads of a unit runs 8/R butterflies per transform;
// loads and stores are separated by a CTA barrier that the NB transforms
// share.
template <int M, int R, int NB, bool STW = false>
__device__ __forceinline__ void fft_pass(float2* const (&zs)[NB], int lt, int Ns,
                                         const float2 (&tw)[7], const float2* stw = nullptr) {
  constexpr int B = 8 / R;       // butterflies per thread
  constexpr int S = M / R;       // input stride
  float2 v[NB][8];
#pragma unroll
  for (int e = 0; e < NB; ++e) {
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int b = lt + r * (M / 8);
#pragma unroll
      for (int j = 0; j < R; ++j) v[e][r * R + j] = zs[e][fe_pad(b + j * S)];
      if (Ns > 1) {
        if constexpr (STW) {  // radix 8, one butterfly per thread: this thread's row of the table
          const float2* row = stw + (b & (Ns - 1)) * 7;
#pragma unroll
          for (int j = 1; j < R; ++j) v[e][r * R + j] = cmul(v[e][r * R + j], row[j - 1]);
        } else {
#pragma unroll
          for (int j = 1; j < R; ++j) v[e][r * R + j] = cmul(v[e][r * R + j], tw[r * (R - 1) + j - 1]);
        }
      }
    }
    if constexpr (R == 8) {
      dft8(v[e]);
    } else if constexpr (R == 4) {
      dft4(v[e][0], v[e][1], v[e][2], v[e][3]);
      dft4(v[e][4], v[e][5], v[e][6], v[e][7]);
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 a0 = v[e][2 * r], a1 = v[e][2 * r + 1];
        v[e][2 * r] = cadd(a0, a1);
        v[e][2 * r + 1] = csub(a0, a1);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < NB; ++e) {
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int b = lt + r * (M / 8);
      const int k = b & (Ns - 1);
      const int base = (b - k) * R + k;
#pragma unroll
      for (int j = 0; j < R; ++j) zs[e][fe_pad(base + j * Ns)] = v[e][r * R + j];
    }
  }
  __syncthreads();
}

// The equaliser in FP32, exactly: with |v| below vsat = ceil(7.5 2^21 / g)
// the fix_36_24 product p = v g is an integer below 7.5 2^21 < 2^24, so
// v (g 2^-21) is exact in FP32, and one fused multiply-add with 1.5 2^23
// rounds it half to even; the sum's low four bits are the fix_4_3 code in
// two's complement.  At or above vsat, |p| rounds to 8 or more and the code
// saturates at +-7.
__host__ __device__ inline float saturation_threshold(uint32_t g) {
  return g == 0 ? 3.0e38f : (float)((15728640u + g - 1) / g);  // 7.5 2^21 = 15728640
}
__device__ __forceinline__ int equalise_nibble(float vf, float gs, float vsat) {
  const int code = __float_as_int(fmaf(vf, gs, 12582912.0f)) & 0xF;
  return fabsf(vf) >= vsat ? (vf < 0.f ? 0x9 : 0x7) : code;
}

// clamp(rne(x), -2^17, 2^17 - 1): clamping first keeps |x| < 2^22, where
// adding 1.5 2^23 rounds x to the nearest integer, ties to even.  Returns
// the sum; its low bits hold the integer, and subtracting 1.5 2^23 gives it
// back exactly as a float.
__device__ __forceinline__ float round18_biased(float x) {
  const float c = fminf(fmaxf(x, -131072.0f), 131071.0f);
  return c + 12582912.0f;
}

// Byte r of w (biased: w holds x ^ 0x80 per byte, x the int8 sample) as the
// float x, exactly: the byte becomes the low mantissa bits of 1.5 * 2^23,
// and subtracting 1.5 * 2^23 + 128 leaves x (every step exact below 2^24).
__device__ __forceinline__ float biased_byte_to_float(uint32_t w, int r) {
  return __int_as_float((int)__byte_perm(w, 0x4B400000u, 0x7650u + (unsigned)r)) - 12583040.0f;
}

// Taps 0..3 of the filter for 8 consecutive samples of both inputs of a
// pair, with aligned 8-byte rows: every tap's loads are issued before any
// arithmetic (taps past `taps` load nothing and add nothing), then
// y += h x in FP32 fused multiply-adds.
__device__ __forceinline__ void fir_taps4(float (&y0)[8], float (&y1)[8], const float (&h)[4][8],
                                          const int8_t* x0, const int8_t* x1, long long M,
                                          int taps, bool has1) {
  uint32_t w[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int2 a = make_int2(0, 0), b = make_int2(0, 0);
    if (q < taps) {
      a = __ldg(reinterpret_cast<const int2*>(x0 + q * M));
      if (has1) b = __ldg(reinterpret_cast<const int2*>(x1 + q * M));
    }
    w[q][0] = (uint32_t)a.x ^ 0x80808080u;
    w[q][1] = (uint32_t)a.y ^ 0x80808080u;
    w[q][2] = (uint32_t)b.x ^ 0x80808080u;
    w[q][3] = (uint32_t)b.y ^ 0x80808080u;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q >= taps) break;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      y0[r] = fmaf(h[q][r], biased_byte_to_float(w[q][r >> 2], r & 3), y0[r]);
      y1[r] = fmaf(h[q][r], biased_byte_to_float(w[q][2 + (r >> 2)], r & 3), y1[r]);
    }
  }
}

// One tap of the filter for 8 consecutive samples of both inputs of a pair:
// y += h x, in FP32 fused multiply-adds.
__device__ __forceinline__ void fir_tap(float (&y0)[8], float (&y1)[8], const float (&h)[8],
                                        const int8_t* x0, const int8_t* x1, bool has1, int vec_in) {
  if (vec_in) {
    const int2 w0 = __ldg(reinterpret_cast<const int2*>(x0));
    const int2 w1 = has1 ? __ldg(reinterpret_cast<const int2*>(x1)) : make_int2(0, 0);
    const uint32_t b0[2] = {(uint32_t)w0.x ^ 0x80808080u, (uint32_t)w0.y ^ 0x80808080u};
    const uint32_t b1[2] = {(uint32_t)w1.x ^ 0x80808080u, (uint32_t)w1.y ^ 0x80808080u};
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      y0[r] = fmaf(h[r], biased_byte_to_float(b0[r >> 2], r & 3), y0[r]);
      y1[r] = fmaf(h[r], biased_byte_to_float(b1[r >> 2], r & 3), y1[r]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      y0[r] = fmaf(h[r], (float)x0[r], y0[r]);
      y1[r] = fmaf(h[r], has1 ? (float)x1[r] : 0.f, y1[r]);
    }
  }
}

// Two CTAs per SM where 256-thread CTAs fit twice (registers capped at 128,
// with a few spills): measured 10% faster than one CTA at 217 registers.
__host__ __device__ constexpr int fe_min_blocks(int logm) { return logm <= 11 ? 2 : 1; }

// POWER: accumulate Eq. 3's power sums (a separate instance, so that the
// common launch without them keeps those registers free).
template <int LOGM, bool POWER>
__global__ void __launch_bounds__(fe_threads(LOGM), fe_min_blocks(LOGM)) fengine_kernel(FeArgs a) {
  constexpr int M = 1 << LOGM, C = M / 2;
  constexpr int TPU = M / 8;                 // threads per FFT unit
  constexpr int NT = fe_threads(LOGM);
  constexpr int U = NT / TPU;                // units per CTA
  constexpr int PM = fe_pad(M);
  constexpr int P8 = LOGM / 3, REM = LOGM % 3;
  extern __shared__ __align__(16) uint8_t fe_smem[];
  const int tid = threadIdx.x, u = tid / TPU, lt = tid % TPU;
  constexpr int kFeNB = fe_nb(LOGM);
  float2* zs[kFeNB];
#pragma unroll
  for (int e = 0; e < kFeNB; ++e) zs[e] = reinterpret_cast<float2*>(fe_smem) + (e * U + u) * PM;
  uint8_t* codes = fe_smem + (size_t)kFeNB * U * PM * sizeof(float2);  // [kFeGroup][C][2]
  float2* ttab = reinterpret_cast<float2*>(codes + (size_t)C * 2 * kFeGroup);  // [Ns=8 | Ns=64][k][7]
  const int i0 = 2 * blockIdx.y;
  const bool has1 = i0 + 1 < a.n_inputs;
  const int N = a.n_inputs;
  const int t0 = blockIdx.x * kFeGroup;
  const int ng = min(kFeGroup, a.n_spectra - t0);

  // per-thread constants: the filter taps of its 8 samples (up to 4 taps in
  // registers) and the twiddles of every pass
  float hr[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < a.taps) {
      const float4 hA = __ldg(reinterpret_cast<const float4*>(a.h + q * M + 8 * lt));
      const float4 hB = __ldg(reinterpret_cast<const float4*>(a.h + q * M + 8 * lt + 4));
      hr[q][0] = hA.x; hr[q][1] = hA.y; hr[q][2] = hA.z; hr[q][3] = hA.w;
      hr[q][4] = hB.x; hr[q][5] = hB.y; hr[q][6] = hB.z; hr[q][7] = hB.w;
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) hr[q][r] = 0.f;
    }
  }
  // passes at Ns = 8 and 64 read the shared table (filled here, first read
  // after the filter's barrier); a pass at Ns = 512 (M = 4096) keeps registers
  for (int e = tid; e < kTwTable; e += NT) {
    const int big = e >= 56, q = big ? e - 56 : e, k = q / 7, j = q % 7 + 1;
    const int Ns = big ? 64 : 8;
    if (M >= 8 * Ns) ttab[e] = __ldg(&a.w[j * k * (M / (8 * Ns))]);
  }
  float2 tw[1][7], twl[7];
  if constexpr (P8 >= 4) load_twiddles<M, 8>(tw[0], lt, 512, a.w);
  if constexpr (REM == 2) load_twiddles<M, 4>(twl, lt, 1 << (3 * P8), a.w);
  if constexpr (REM == 1) load_twiddles<M, 2>(twl, lt, 1 << (3 * P8), a.w);

  float gs[4][2], vsat[4][2];  // gain as g 2^-21 (exact) and its saturation threshold
  unsigned long long pw[4][2];  // only used by the POWER instance
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int nu = lt + k * TPU;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t gj = (j == 0 || has1) ? a.gain[(long long)nu * N + i0 + j] : 0u;
      gs[k][j] = (float)gj * 4.76837158203125e-07f;  // 2^-21
      vsat[k][j] = saturation_threshold(gj);
      pw[k][j] = 0ull;
    }
  }

  for (int sb = 0; sb < ng; sb += kFeNB * U) {
    // ---- polyphase filter: y[n] = sum_q h[q M + n] x[(t + q) M + n]
    if (U == 1 && a.vec_in && a.taps <= 4) {
      // One unit per CTA: the unit's spectra sb, sb + 1, ... are adjacent and
      // share frames, so each frame is loaded and converted once and added
      // into every spectrum that uses it (static tap indices).
      constexpr int NF = kFeNB + 3;  // frames of kFeNB spectra at up to 4 taps
      const int8_t* xb = a.adc + (long long)i0 * a.adc_stride + (long long)(t0 + sb) * M + 8 * lt;
      const int last = min(ng - 1 - sb, kFeNB - 1);  // last active spectrum of the iteration
      float y[kFeNB][2][8];
#pragma unroll
      for (int e = 0; e < kFeNB; ++e)
#pragma unroll
        for (int r = 0; r < 8; ++r) y[e][0][r] = y[e][1][r] = 0.f;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (f > last + a.taps - 1) break;  // frames past the last active spectrum's taps
        const int2 w0 = __ldg(reinterpret_cast<const int2*>(xb + (long long)f * M));
        const int2 w1 = has1 ? __ldg(reinterpret_cast<const int2*>(xb + a.adc_stride + (long long)f * M))
                             : make_int2(0, 0);
        const uint32_t b[4] = {(uint32_t)w0.x ^ 0x80808080u, (uint32_t)w0.y ^ 0x80808080u,
                               (uint32_t)w1.x ^ 0x80808080u, (uint32_t)w1.y ^ 0x80808080u};
        float x[2][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          x[0][r] = biased_byte_to_float(b[r >> 2], r & 3);
          x[1][r] = biased_byte_to_float(b[2 + (r >> 2)], r & 3);
        }
#pragma unroll
        for (int e = 0; e < kFeNB; ++e) {
          const int q = f - e;  // this frame is tap q of spectrum e
          if (q < 0 || q > 3 || q >= a.taps || e > last) continue;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            y[e][0][r] = fmaf(hr[q][r], x[0][r], y[e][0][r]);
            y[e][1][r] = fmaf(hr[q][r], x[1][r], y[e][1][r]);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < kFeNB; ++e) {
#pragma unroll
        for (int r = 0; r < 8; ++r) zs[e][fe_pad(8 * lt + r)] = make_float2(y[e][0][r], y[e][1][r]);
      }
      // the next iteration's newest frames come from DRAM: ask for those of
      // its active spectra now
#pragma unroll
      for (int e = 0; e < kFeNB; ++e) {
        if (sb + kFeNB + e >= ng) break;
        const int8_t* nx = xb + (long long)(kFeNB + e + a.taps - 1) * M;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(nx));
        if (has1) asm volatile("prefetch.global.L1 [%0];" ::"l"(nx + a.adc_stride));
      }
    } else {
#pragma unroll
    for (int e = 0; e < kFeNB; ++e) {
      const int s = sb + e * U + u;
      const bool active = s < ng;
      const long long t = t0 + s;
      float y0[8], y1[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) y0[r] = y1[r] = 0.f;
      if (active) {
        const int8_t* x0 = a.adc + (long long)i0 * a.adc_stride + t * M + 8 * lt;
        const int8_t* x1 = x0 + a.adc_stride;
        // taps 0..3 with their coefficients in registers (static indices),
        // then any further taps with coefficients from the table
        if (a.vec_in) {
          fir_taps4(y0, y1, hr, x0, x1, M, a.taps, has1);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < a.taps)
              fir_tap(y0, y1, hr[q], x0 + (long long)q * M, x1 + (long long)q * M, has1, 0);
        }
        for (int q = 4; q < a.taps; ++q) {
          float hq[8];
          const float4 hA = __ldg(reinterpret_cast<const float4*>(a.h + q * M + 8 * lt));
          const float4 hB = __ldg(reinterpret_cast<const float4*>(a.h + q * M + 8 * lt + 4));
          hq[0] = hA.x; hq[1] = hA.y; hq[2] = hA.z; hq[3] = hA.w;
          hq[4] = hB.x; hq[5] = hB.y; hq[6] = hB.z; hq[7] = hB.w;
          fir_tap(y0, y1, hq, x0 + (long long)q * M, x1 + (long long)q * M, has1, a.vec_in);
        }
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) zs[e][fe_pad(8 * lt + r)] = make_float2(y0[r], y1[r]);
      // the next iteration's newest frame comes from DRAM: ask for it now
      if (active && s + kFeNB * U < ng) {
        const int8_t* nx =
            a.adc + (long long)i0 * a.adc_stride + (t + kFeNB * U + a.taps - 1) * M + 8 * lt;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(nx));
        if (has1) asm volatile("prefetch.global.L1 [%0];" ::"l"(nx + a.adc_stride));
      }
    }
    }
    __syncthreads();
    // ---- FFTs of y_2k + j y_2k+1 (natural order out), kFeNB side by side
    fft_pass<M, 8, kFeNB>(zs, lt, 1, twl);  // first pass: no twiddles
    if constexpr (P8 >= 2) fft_pass<M, 8, kFeNB, true>(zs, lt, 8, twl, ttab);
    if constexpr (P8 >= 3) fft_pass<M, 8, kFeNB, true>(zs, lt, 64, twl, ttab + 56);
    if constexpr (P8 >= 4) fft_pass<M, 8, kFeNB>(zs, lt, 512, tw[0]);
    if constexpr (REM == 2) fft_pass<M, 4, kFeNB>(zs, lt, 1 << (3 * P8), twl);
    if constexpr (REM == 1) fft_pass<M, 2, kFeNB>(zs, lt, 1 << (3 * P8), twl);
    // ---- Eq. 2 separation, 18-bit rounding, equaliser
#pragma unroll
    for (int e = 0; e < kFeNB; ++e) {
      const int s = sb + e * U + u;
      if (s >= ng) continue;
      const long long t = t0 + s;
      const float2* z = zs[e];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nu = lt + k * TPU;
        const float2 zp = z[fe_pad(nu)], zm = z[fe_pad((M - nu) & (M - 1))];
        const float X[2][2] = {{(zp.x + zm.x) * a.scale, (zp.y - zm.y) * a.scale},
                               {(zp.y + zm.y) * a.scale, (zm.x - zp.x) * a.scale}};
        uint32_t pair = 0;  // the codes of inputs i0 and i0 + 1: one 16-bit store
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (j == 1 && !has1) break;
          const float sr = round18_biased(X[j][0]), si = round18_biased(X[j][1]);
          const int vr = __float_as_int(sr) - 0x4B400000, vi = __float_as_int(si) - 0x4B400000;
          if (a.spec || a.v18) {
            const long long ei = ((t * C + nu) * N + i0 + j) * 2;
            if (a.spec) *reinterpret_cast<float2*>(a.spec + ei) = make_float2(X[j][0], X[j][1]);
            if (a.v18) *reinterpret_cast<int2*>(a.v18 + ei) = make_int2(vr, vi);
          }
          if constexpr (POWER) pw[k][j] += (unsigned long long)((long long)vr * vr + (long long)vi * vi);
          const int qr = equalise_nibble(sr - 12582912.0f, gs[k][j], vsat[k][j]);
          const int qi = equalise_nibble(si - 12582912.0f, gs[k][j], vsat[k][j]);
          pair |= (uint32_t)(a.lo_is_real ? (qi << 4) | qr : (qr << 4) | qi) << (8 * j);
        }
        *reinterpret_cast<uint16_t*>(codes + (s * C + nu) * 2) = (uint16_t)pair;
      }
    }
    __syncthreads();
  }

  // ---- codes out.  Staging is [spectrum][channel][input], so a thread
  // gathers one (channel, input) row of 32 spectra with conflict-free byte
  // loads (consecutive threads, consecutive rows) and stores it as two
  // 16-byte pieces of the [c][i][t] output.
  const int nj = has1 ? 2 : 1;
  if (a.out) {
    if (a.layout == CORR_L_CIT) {
      for (int row = tid; row < 2 * C; row += NT) {
        const int nu = row >> 1, j = row & 1;
        if (j >= nj) continue;
        uint8_t* o = a.out + ((long long)nu * N + i0 + j) * a.out_stride + t0;
        if (a.vec_out && ng == kFeGroup) {
          uint32_t wv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            wv[q] = (uint32_t)codes[(4 * q) * 2 * C + row] |
                    ((uint32_t)codes[(4 * q + 1) * 2 * C + row] << 8) |
                    ((uint32_t)codes[(4 * q + 2) * 2 * C + row] << 16) |
                    ((uint32_t)codes[(4 * q + 3) * 2 * C + row] << 24);
          *reinterpret_cast<uint4*>(o) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
          *reinterpret_cast<uint4*>(o + 16) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
        } else {
          for (int s = 0; s < ng; ++s) o[s] = codes[s * 2 * C + row];
        }
      }
    } else {  // [t][c][i]
      for (int e = tid; e < ng * C; e += NT) {
        const int s = e / C, nu = e - s * C;
        uint8_t* o = a.out + ((long long)(t0 + s) * C + nu) * N + i0;
        o[0] = codes[(s * C + nu) * 2];
        if (has1) o[1] = codes[(s * C + nu) * 2 + 1];
      }
    }
  }
  if constexpr (POWER) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int nu = lt + k * TPU;
      // every unit of the CTA summed its own spectra: add them all
      atomicAdd(a.power + (long long)nu * N + i0, pw[k][0]);
      if (has1) atomicAdd(a.power + (long long)nu * N + i0 + 1, pw[k][1]);
    }
  }
}

template <int LOGM, bool POWER>
cudaError_t fe_launch_one(const FeArgs& a, int n_pairs, cudaStream_t s) {
  constexpr size_t smem = fe_smem_bytes<LOGM>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fengine_kernel<LOGM, POWER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((a.n_spectra + kFeGroup - 1) / kFeGroup, n_pairs);
  fengine_kernel<LOGM, POWER><<<grid, fe_threads(LOGM), smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGM>
cudaError_t fe_launch(const FeArgs& a, int n_pairs, cudaStream_t s) {
  return a.power ? fe_launch_one<LOGM, true>(a, n_pairs, s) : fe_launch_one<LOGM, false>(a, n_pairs, s);
}

bool fe_is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void fe_free(fe_ctx* f) {
  if (!f) return;
  if (f->stream) cudaStreamSynchronize(f->stream);
  cudaFree(f->h);
  cudaFree(f->w);
  cudaFree(f->gain);
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  delete f;
}

}  // namespace
}  // namespace xe

using namespace xe;

extern "C" {

int fe_create(int n_inputs, int n_chans, int taps, int shift, unsigned flags, void* stream,
              fe_ctx** out) {
  TraceRange trace_("fe_create");
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_inputs < 1 || n_inputs > 131070 || n_chans < 16 || n_chans > 2048 ||
      (n_chans & (n_chans - 1)) || taps < 1 || taps > 16 || shift < 0 || shift > 24 ||
      (flags & ~FE_F_LO_IS_REAL))
    return CORR_EINVAL;
  fe_ctx* f = new (std::nothrow) fe_ctx;
  if (!f) return CORR_ENOMEM;
  f->n_inputs = n_inputs;
  f->n_chans = n_chans;
  f->taps = taps;
  f->shift = shift;
  f->flags = flags;
  const int M = 2 * n_chans;
  const long long L = (long long)taps * M;
  // prototype: Hamming window times sinc, in FP64, rounded to FP32
  std::vector<float> h(L);
  const double pi = 3.14159265358979323846;
  for (long long m = 0; m < L; ++m) {
    const double win = 0.54 - 0.46 * std::cos(2.0 * pi * (double)m / (double)(L - 1));
    const double x = ((double)m - (double)(L - 1) / 2.0) / (double)M;
    const double sinc = x == 0.0 ? 1.0 : std::sin(pi * x) / (pi * x);
    h[m] = (float)(win * sinc);
  }
  std::vector<float2> w(M);
  for (int n = 0; n < M; ++n) {
    const double ang = -2.0 * pi * (double)n / (double)M;
    w[n] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  int st = CORR_OK;
  do {
    if (stream) {
      f->stream = (cudaStream_t)stream;
    } else {
      if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) { st = CORR_ECUDA; break; }
      f->own_stream = true;
    }
    if (cudaMalloc(&f->h, L * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&f->w, M * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&f->gain, (size_t)n_chans * n_inputs * sizeof(uint32_t)) != cudaSuccess) {
      st = CORR_ENOMEM;
      break;
    }
    if (cudaMemcpy(f->h, h.data(), L * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(f->w, w.data(), M * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(f->gain, 0, (size_t)n_chans * n_inputs * sizeof(uint32_t)) != cudaSuccess) {
      st = CORR_ECUDA;
      break;
    }
  } while (0);
  if (st != CORR_OK) {
    fe_free(f);
    return st;
  }
  *out = f;
  return CORR_OK;
}

int fe_set_gains(fe_ctx* f, const uint32_t* gain) {
  if (!f || !gain) return CORR_EINVAL;
  const size_t n = (size_t)f->n_chans * f->n_inputs;
  if (fe_is_device(gain)) {
    // checked on the host: a device table is copied back once
    std::vector<uint32_t> hg(n);
    if (cudaMemcpy(hg.data(), gain, n * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return CORR_ECUDA;
    for (uint32_t v : hg)
      if (v >= (1u << 18)) return CORR_EINVAL;
  } else {
    for (size_t k = 0; k < n; ++k)
      if (gain[k] >= (1u << 18)) return CORR_EINVAL;
  }
  if (cudaMemcpyAsync(f->gain, gain, n * sizeof(uint32_t), cudaMemcpyDefault, f->stream) != cudaSuccess ||
      cudaStreamSynchronize(f->stream) != cudaSuccess)
    return CORR_ECUDA;
  return CORR_OK;
}

int fe_channelise(fe_ctx* f, const int8_t* adc, long long adc_stride, int n_spectra, uint8_t* out,
                  int layout, long long out_stride, int32_t* v18, float* spec, int64_t* power) {
  TraceRange trace_("fe_channelise");
  if (!f || !adc || n_spectra < 1) return CORR_EINVAL;
  const int M = 2 * f->n_chans;
  if (adc_stride < (long long)(n_spectra + f->taps - 1) * M) return CORR_EINVAL;
  if (layout != CORR_L_CIT && layout != CORR_L_TCI) return CORR_EINVAL;
  if (out && layout == CORR_L_CIT && out_stride < n_spectra) return CORR_EINVAL;
  if (!fe_is_device(adc) || (out && !fe_is_device(out)) || (v18 && !fe_is_device(v18)) ||
      (spec && !fe_is_device(spec)) || (power && !fe_is_device(power)))
    return CORR_EINVAL;
  if ((v18 && reinterpret_cast<uintptr_t>(v18) % 8) || (spec && reinterpret_cast<uintptr_t>(spec) % 8) ||
      (power && reinterpret_cast<uintptr_t>(power) % 8))
    return CORR_EINVAL;
  FeArgs a{};
  a.adc = adc;
  a.adc_stride = adc_stride;
  a.h = f->h;
  a.w = f->w;
  a.gain = f->gain;
  a.out = out;
  a.out_stride = out_stride;
  a.v18 = v18;
  a.spec = spec;
  a.power = reinterpret_cast<unsigned long long*>(power);
  a.n_inputs = f->n_inputs;
  a.n_spectra = n_spectra;
  a.taps = f->taps;
  a.layout = layout;
  a.lo_is_real = (f->flags & FE_F_LO_IS_REAL) ? 1 : 0;
  a.vec_in = reinterpret_cast<uintptr_t>(adc) % 8 == 0 && adc_stride % 8 == 0;
  a.vec_out = out && layout == CORR_L_CIT && reinterpret_cast<uintptr_t>(out) % 16 == 0 &&
              out_stride % 16 == 0;
  a.scale = std::ldexp(1.0f, -(f->shift + 1));
  const int pairs = (f->n_inputs + 1) / 2;
  cudaError_t e;
  switch (M) {
    case 32: e = fe_launch<5>(a, pairs, f->stream); break;
    case 64: e = fe_launch<6>(a, pairs, f->stream); break;
    case 128: e = fe_launch<7>(a, pairs, f->stream); break;
    case 256: e = fe_launch<8>(a, pairs, f->stream); break;
    case 512: e = fe_launch<9>(a, pairs, f->stream); break;
    case 1024: e = fe_launch<10>(a, pairs, f->stream); break;
    case 2048: e = fe_launch<11>(a, pairs, f->stream); break;
    case 4096: e = fe_launch<12>(a, pairs, f->stream); break;
    default: return CORR_EINVAL;
  }
  return e == cudaSuccess ? CORR_OK : CORR_ECUDA;
}

int fe_gains_from_power(const int64_t* power, int n_chans, int n_inputs, long long n_spectra,
                        double target_rms, uint32_t* gain) {
  if (!power || !gain || n_chans < 1 || n_inputs < 1 || n_spectra < 1 || !(target_rms > 0.0))
    return CORR_EINVAL;
  const long long n = (long long)n_chans * n_inputs;
  for (long long k = 0; k < n; ++k) {
    if (power[k] < 0) return CORR_EINVAL;
    if (power[k] == 0) {
      gain[k] = 0;
      continue;
    }
    const double rms = std::sqrt((double)power[k] / (2.0 * (double)n_spectra));
    const double g = std::nearbyint(target_rms * 2097152.0 / rms);
    gain[k] = g < 1.0 ? 1u : (g > 262143.0 ? 262143u : (uint32_t)g);
  }
  return CORR_OK;
}

int fe_sync(fe_ctx* f) {
  if (!f) return CORR_EINVAL;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? CORR_OK : CORR_ECUDA;
}

void fe_destroy(fe_ctx* f) { fe_free(f); }

}  // extern "C"
