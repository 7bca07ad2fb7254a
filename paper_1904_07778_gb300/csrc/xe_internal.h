// Internal interfaces between the X-engine's translation units (kernels and
// the C-ABI runtime).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace xe {

// A named NVTX range for the scope (visible in a profiler's timeline; free
// when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Device status word bits (OR-ed by kernels, read and cleared by the host).
enum : int {
  kStTimeout = 1,   // a bounded device-side wait expired
  kStRange = 2,     // an 8-bit sample equal to -128 was seen
};

// One task of the Hermitian rank-k update.  The real Gram matrix of a
// channel is G = Y Y^T with Y the (2N x T) matrix whose row 2i holds Re x_i
// and row 2i+1 holds Im x_i; it is cut into 128 x 128 blocks.  A task owns
// the rows of block rb against one or two column blocks cb[0], cb[1]
// (cb[1] = -1 for one): the MMA is 128 x 128 or 128 x 256.  Because G is
// symmetric, block (rb, c) with c > rb stands for block (c, rb) of the lower
// triangle and is written transposed.  When 2N <= 64, several channels are
// stacked in one 128-row block (rows_per_chan = 2N rounded up to a power of
// two) and the task covers channels chan0 .. chan0 + 128 / rows_per_chan - 1.
//
// 8-bit samples have the same Y: the block is first laid out as
// [channel][input][re/im byte][time] (byte row 2i + p), each byte is one
// FP16 operand, and the blocks above count 2N rows as at 4 bits.
struct HerkTask {
  int chan0;
  int rb;
  int cb[2];
  int inst;  // array (instance) of a batched launch; 0 for a single array
};

// One array's block as the cross-multiply sees it.
struct HerkInst {
  const uint8_t* x;          // samples, [channel][byte row][time] order
  int64_t* acc;              // int64 visibilities [C][N(N+1)/2][2]
  long long chan_stride;     // bytes between channels of x
  long long row_stride;      // bytes between byte rows of x
  int n_inputs, n_chans;
  int t0, tn;                // time range [t0, t0 + tn) of this launch, samples
  int rows_per_chan;         // stacked mode: rows per channel in a tile; 0 = not stacked
  int accumulate;            // 0: store into acc, 1: add into acc
  int vec_ok;                // 16-byte loads are aligned everywhere
  // Fault injection for the tests of the bounded waits, read from the
  // single-array launch's instance only (0 = off): bits 0..23 = s > 0 makes
  // the TMA loader of CTA 0 skip its stage s - 1, so the waits for it run
  // out; bits 24..30 = w > 0 limits every wait to 2^w cycles.
  int fault;
};

struct HerkArgs {
  HerkInst in;               // the array of a single-array launch
  const HerkInst* insts;     // batched launch: per-array parameters (device memory), else null
  const CUtensorMap* tmaps;  // batched launch: per-array tensor maps (device, 64-byte aligned)
  const HerkTask* tasks;
  const int* cta_first;      // if set, CTA b runs tasks [cta_first[b], cta_first[b + 1]);
                             // otherwise task j of CTA b is b + j * gridDim.x
  int* status;
  int lo_is_real;            // 4-bit: real part in the low nibble (whole launch)
  int bits;                  // 4, or 8 (byte rows: 2 per input, each one row of Y)
  // 8-bit: per-CTA partial sums of tasks longer than one accumulation,
  // kHerkScratchInt2 int2 for each of scratch_ctas CTAs (the launch's grid
  // must not exceed it)
  int2* scratch;
  int scratch_ctas;
  int smem_bytes;            // dynamic shared memory of the launch
  int n_tasks;               // tasks in `tasks`
  int grid;                  // CTAs of a launch with cta_first; otherwise, if > 0,
                             // the most CTAs (SMs) a single-array launch may use
};

// Largest number of spectra integrated in one tensor-memory accumulation:
// with 4-bit offset codes u <= 15 a partial sum is at most 225 per spectrum,
// and FP32 holds every integer below 2^24 exactly (225 * 65536 < 2^24).
constexpr int kMaxChunk4 = 65536;
// Largest number of 8-bit spectra per launch.  The kernel accumulates 1024
// spectra at a time in FP32 (127^2 * 1024 < 2^24) and adds the pieces in
// int32, which holds |V| <= 2 * 127^2 * 32768 < 2^31.
constexpr int kMaxChunk8 = 32768;
// int2 partial sums per CTA of an 8-bit launch (a 128 x 256 task: 64 x 128
// visibilities).
constexpr int kHerkScratchInt2 = 8192;

int herk4_max_smem();
// Spectra per stage of the ring kernel (128 at 4 bits, 64 at 8 bits): the
// time extent of its TMA boxes.
int herk_ring_stage(int bits);
// Launch the cross-multiply.  Batched (a.insts and a.tmaps set): the ring
// kernel over every array's tasks in one persistent launch.  Otherwise tmap
// (make_herk_tmap) describes a.in.x for the ring kernel, or is null for the
// 4-bit kernel that loads with plain global loads (any alignment).
// With tci the tensor maps describe payload-order ([t][c][i]) blocks and the
// kernel transposes while it unpacks.  8-bit launches need a.scratch for
// every CTA of the grid (cudaErrorInvalidValue otherwise).
cudaError_t herk4_launch(const HerkArgs& a, const CUtensorMap* tmap, int n_tasks, cudaStream_t s,
                         bool tci = false);

// Tensor map of one block for the ring kernel, R byte rows per channel
// (N at 4 bits, 2N at 8 bits), rpc = rows_per_chan of the task plan.  A box
// is one 128-row operand block of one stage: herk_ring_stage(bits) spectra
// of 128 * bits / 8 byte rows, or for stacked arrays rpc * bits / 8 byte rows
// of 128 / rpc channels.
//   tci = false: x is [channel][byte row][time] with rows row_stride bytes
//     apart (a multiple of 16, base 16-byte aligned); dims {T, R, C}.
//   tci = true: x is the payload order [time][channel][byte row] (R a
//     multiple of 16, base 16-byte aligned); dims {R, C, T}.
// Returns false if the driver rejects it.
bool make_herk_tmap(CUtensorMap* m, const uint8_t* x, bool tci, int bits, int R, int n_chans,
                    int n_time, long long row_stride, int rpc);
// Device scratch for the 8-bit partial sums of a launch on this device: one
// kHerkScratchInt2 region per SM (*ctas = the SM count).
cudaError_t herk_scratch_alloc(int2** p, int* ctas);
// Whether a block of this layout and width can be read in payload order
// (no corner turn): [t][c][i] with R = N bits / 4 byte rows a multiple of 16.
bool tci_direct(int layout, int bits, int n_inputs);

// Corner turn of byte samples: in[t][g][k] -> out[k][g][t], output rows of
// out_stride >= T bytes (32-byte aligned rows take the fast path).
// With pair_rows, k = 2 c + p counts (c, p) pairs and output row (k, g) goes
// to row (c G + g) 2 + p instead of k G + g: 8-bit [t][i][c][re/im] becomes
// [c][i][re/im][t].
// With persist_ctas > 0 the turn runs as that many persistent CTAs, one per
// SM (for overlapping it with a cross-multiply on the remaining SMs).
cudaError_t turn_launch(const uint8_t* in, uint8_t* out, int T, int G, int K, long long out_stride,
                        cudaStream_t s, bool pair_rows = false, int persist_ctas = 0);
// The same with input rows in_stride >= K bytes apart: a range of K bytes cut
// out of each row of a wider block.
cudaError_t turn_launch_strided(const uint8_t* in, uint8_t* out, int T, int G, int K,
                                long long in_stride, long long out_stride, cudaStream_t s,
                                bool pair_rows = false, int persist_ctas = 0);

// A block in packet order, [slot][fid][xid][8][chans_pkt][inputs_pkt] bytes,
// becomes [c][i][t] rows of out_stride bytes (c = xid chans_pkt + cc,
// i = fid inputs_pkt + ii, t = 8 slot + tt).
cudaError_t pkt_turn_launch(const uint8_t* in, uint8_t* out, int n_fids, int inputs_pkt, int n_xids,
                            int chans_pkt, int T, long long out_stride, cudaStream_t s);

// 8-bit samples already in [row][t][re/im] order (row = channel x input):
// out[row][p][t] = in[row][t][p], output rows of out_stride bytes.
cudaError_t split_planes_launch(const uint8_t* in, uint8_t* out, long long rows, int T,
                                long long out_stride, cudaStream_t s);

// Lay one block out as [channel][byte row][time] with rows of out_stride
// bytes (byte rows: one per input at 4 bits, re and im bytes at 8 bits).
// Returns false without launching when the layout is already that one
// (4-bit [c][i][t]): the block itself is then the cross-multiply's input.
bool needs_turn(int layout, int bits);
// turn_rows runs turn_launch (and so can take persist_ctas) for this layout
bool turn_can_persist(int layout, int bits);
cudaError_t turn_rows(const uint8_t* in, uint8_t* out, int layout, int bits, int n_inputs,
                      int n_chans, int n_time, long long out_stride, cudaStream_t s,
                      int persist_ctas = 0);
// turn_rows for channels c0 .. c1-1 only (4-bit [t][c][i] or [t][i][c]):
// their rows of the whole block's output.  cudaErrorInvalidValue otherwise.
cudaError_t turn_rows_chans(const uint8_t* in, uint8_t* out, int layout, int bits, int n_inputs,
                            int n_chans, int n_time, int c0, int c1, long long out_stride,
                            cudaStream_t s, int persist_ctas = 0);

// Tasks of one array of n_inputs inputs (2 n_inputs rows of Y; see
// HerkTask): rows_per_chan is set for stacked arrays.  With singles, every
// task has one column block (128 x 128).
std::vector<HerkTask> plan_tasks(int n_inputs, int n_chans, int* rows_per_chan, bool singles = false);

// Snapshot the device status word into host_slot (pinned host memory, written
// by the device through its mapping; read it once the stream has passed this
// point) and clear it.
cudaError_t take_status_launch(int* status, int* host_slot, cudaStream_t s);
// SM count of the current device (queried once per device).
int device_sm_count();
// FP64 correlation coefficients from int64 visibilities; zero_flag (may be
// null) gets 1 per baseline whose denominator V_ii V_jj is zero, else 0.
cudaError_t normalise_launch(const int64_t* acc, double* rho, uint8_t* zero_flag, int n_inputs,
                             int n_chans, cudaStream_t s);

}  // namespace xe
