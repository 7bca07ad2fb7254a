// Internal interfaces between the X-engine's translation units (kernels and
// the C-ABI runtime).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace xe {

// Device status word bits (OR-ed by kernels, read and cleared by the host).
enum : int {
  kStTimeout = 1,   // a bounded device-side wait expired
  kStRange = 2,     // an 8-bit sample equal to -128 was seen
};

// One tile-row task of the Hermitian rank-k update.  The real Gram matrix of
// a channel is G = Y Y^T with Y the (2N x T) matrix whose row 2i holds Re x_i
// and row 2i+1 holds Im x_i.  A task owns output rows [128 rb, 128 rb + 128)
// of G against column blocks [128 cb0, 128 cb1) (cb1 <= rb + 1, at most four
// blocks), for channel chan0.  When 2N < 128, several channels are stacked in
// one 128-row tile (rows_per_chan = 2N rounded up to a power of two) and the
// task covers channels chan0 .. chan0 + 128 / rows_per_chan - 1.
struct HerkTask {
  int chan0;
  int rb;
  int cb0;
  int cb1;
};

struct HerkArgs {
  const uint8_t* x;          // samples, [channel][input][time] order
  int64_t* acc;              // int64 visibilities [C][N(N+1)/2][2]
  const HerkTask* tasks;
  int* status;
  long long chan_stride;     // bytes between channels of x
  long long row_stride;      // bytes between inputs of x
  int n_inputs, n_chans;
  int t0, tn;                // time range [t0, t0 + tn) of this launch, samples
  int rows_per_chan;         // stacked mode: rows per channel in a tile; 0 = not stacked
  int accumulate;            // 0: store into acc, 1: add into acc
  int lo_is_real;            // 4-bit: real part in the low nibble
  int vec_ok;                // 16-byte loads are aligned everywhere
  int smem_bytes;            // dynamic shared memory of the launch
};

// Largest number of spectra integrated in one tensor-memory accumulation:
// with 4-bit offset codes u <= 15 a partial sum is at most 225 per spectrum,
// and FP32 holds every integer below 2^24 exactly (225 * 65536 < 2^24).
constexpr int kMaxChunk4 = 65536;

int herk4_max_smem();
cudaError_t herk4_launch(const HerkArgs& a, int n_tasks, cudaStream_t s);

// Corner turn of byte samples: in[t][g][k] -> out[k][g][t] (out row = T bytes).
cudaError_t turn_launch(const uint8_t* in, uint8_t* out, int T, int G, int K, cudaStream_t s);

// FP64 correlation coefficients from int64 visibilities.
cudaError_t normalise_launch(const int64_t* acc, double* rho, int n_inputs, int n_chans,
                             cudaStream_t s);

}  // namespace xe
