/*
 * xengine.h -- C ABI of the GB300 X-engine (FX correlator, cross-multiply
 * and integrate stage) of Niu et al., arXiv:1904.07778.
 *
 * What the library computes (Sec. 2, System Design; Sec. 2.2, X-engine):
 * for every frequency channel c and every pair of inputs j <= i,
 *
 *     V[c][i][j] = sum over pushed spectra t of  x_i(c,t) * conj(x_j(c,t))
 *
 * i.e. all cross- and auto-correlations of the same frequency (the CMAC
 * "multiply and accumulation" of Sec. 2), integrated over a caller-chosen
 * number of blocks ("integrated for some pre-specified duration", Sec. 2).
 * Results are exact integers (int64); the GPU result is bit-identical to
 * the plain definition above.
 *
 * Conventions shared by every call:
 *  - Status: every int-returning call returns CORR_OK (0) or a negative
 *    CORR_E* code; nothing throws across the ABI.  corr_strerror() names it.
 *  - Output order: baseline index b(i,j) = i*(i+1)/2 + j for i >= j (lower
 *    triangle incl. autos; the upper triangle is the conjugate).  A
 *    visibility array is int64 vis[n_chans][n_baselines][2], [..][0] = Re,
 *    [..][1] = Im.  The paper's delay-test visibility V = I1* . I2 (Sec. 3,
 *    Eq. 5) conjugates the first input; that quantity is this library's
 *    V[i=2][j=1] = x_2 conj(x_1).
 *  - Pointers: any buffer argument may be host memory (pageable or pinned)
 *    or device memory of the current CUDA device; the library detects which.
 *    The caller owns every buffer it passes.
 *  - Streams: all device work of a context runs on the stream given to
 *    corr_create (a cudaStream_t passed as void*), or on a private stream if
 *    NULL was given.  Calls on one context are not thread-safe; use one
 *    context per thread.
 */
#ifndef XENGINE_H
#define XENGINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define CORR_OK 0
#define CORR_EINVAL (-1)    /* bad argument: shape, bits, layout, size, pointer   */
#define CORR_ENOMEM (-2)    /* device or host allocation failed                  */
#define CORR_EBUSY (-3)     /* request does not fit the memory budget now         */
#define CORR_ERANGE (-4)    /* an 8-bit sample equal to -128 was pushed           */
#define CORR_ESEQ (-5)      /* block sequence number is a gap or a duplicate      */
#define CORR_ETIMEDOUT (-6) /* a bounded device-side wait expired                 */
#define CORR_ECUDA (-7)     /* a CUDA runtime call failed                         */
#define CORR_ESTATE (-8)    /* call not valid in the context's current state      */
#define CORR_ECORRUPT (-9)  /* a packet failed its CRC check (ingest.h)           */

/* ---- sample layouts of a pushed block -------------------------------- */
/* [time][channel][input]: the F-engine payload order of Sec. 2.3 (packets
 * hold "[time, (fixed) channel, (run) input channel]").                    */
#define CORR_L_TCI 0
/* [time][input][channel]: spectra grouped by receiver input, before the
 * corner turn of Sec. 2.1 ("Transpose" block: [input, frequency] ->
 * [frequency, input]); the library performs the corner turn on the GPU.    */
#define CORR_L_TIC 1
/* [channel][input][time]: already corner-turned and time-contiguous.       */
#define CORR_L_CIT 2

/* ---- create flags ---------------------------------------------------- */
/* 4-bit samples: the real part is in the LOW nibble (default: high nibble).
 * Sec. 2.1 only says two 4-bit numbers are re-packed into one byte.        */
#define CORR_F_LO_IS_REAL 0x1u

/* Pass as seq to corr_push to skip the sequence check.                    */
#define CORR_SEQ_ANY UINT64_MAX

typedef struct corr_ctx corr_ctx; /* opaque, owned by the library */

/*
 * corr_create -- make a correlator context for one array.
 *   n_inputs : number of inputs N (receiver channels; 2 per dual-pol dish,
 *              Sec. 1), 1 <= N <= 1024.
 *   n_chans  : frequency channels C held by this context (the F/N channels a
 *              GPU node processes, Sec. 2), C >= 1.
 *   n_time   : spectra per pushed block T, T >= 1.
 *   bits     : 4 -> one byte per complex sample, two 4-bit two's-complement
 *              numbers (the equaliser output of Sec. 2.1, values -7..7; code
 *              0x8 decodes to -8);  8 -> two int8 bytes (re, im) per sample,
 *              symmetric range -127..127.  A -128 is still integrated
 *              exactly, and the next corr_sync / corr_dump / corr_normalise
 *              returns CORR_ERANGE (once; the flag is then cleared).  In the
 *              layouts an 8-bit sample is the byte pair (re, im) in place of
 *              the 4-bit byte.  CORR_F_LO_IS_REAL is invalid with 8 bits.
 *   layout   : CORR_L_TCI, CORR_L_TIC or CORR_L_CIT.
 *   flags    : CORR_F_* bits.
 *   stream   : cudaStream_t to run on, or NULL for a private stream.
 *   out      : receives the context.
 * Allocates the context's device state (accumulators, staging, corner-turn
 * buffers) on the current device.  Returns CORR_EINVAL for a bad shape,
 * CORR_ENOMEM when an allocation fails, CORR_ECUDA when no usable device.
 */
int corr_create(int n_inputs, int n_chans, int n_time, int bits, int layout, unsigned flags,
                void* stream, corr_ctx** out);

/*
 * corr_push -- add one block of T spectra to the running integration.
 *   block  : packed samples in the context's layout, host or device memory.
 *   nbytes : must equal N * C * T * bits / 4, else CORR_EINVAL.
 *   seq    : block sequence number; the first push after create or a reset
 *            may carry any value, each later push must carry previous + 1
 *            (the packet-counter gap check of Sec. 2.3).  A gap or duplicate
 *            returns CORR_ESEQ and the block is NOT integrated.
 *            CORR_SEQ_ANY disables the check for this push.
 * Asynchronous and stream-ordered.  A device block is read in place and
 * must stay unchanged until corr_sync or corr_dump returns; a host block is
 * copied to device staging (pinned memory makes the copy asynchronous and
 * double-buffered against compute) and must stay unchanged until the same
 * point.  8-bit samples equal to -128 are detected on the device and
 * reported as CORR_ERANGE by the next corr_sync / corr_dump.
 */
int corr_push(corr_ctx* ctx, const void* block, size_t nbytes, uint64_t seq);

/*
 * corr_push_many -- add n_blocks blocks of T spectra each to the running
 * integration: the accumulation of Sec. 2.2 over the spectra of several
 * blocks, the same result as n_blocks corr_push calls in order.
 *   blocks   : n_blocks pointers to packed blocks in the context's layout.
 *   n_blocks : 1 <= n_blocks <= CORR_MAX_PUSH_MANY, else CORR_EINVAL.
 *   nbytes   : bytes of ONE block, N * C * T * bits / 4, else CORR_EINVAL.
 *   seq      : sequence number of the first block (the others follow it), or
 *              CORR_SEQ_ANY; checked as for corr_push, and a gap returns
 *              CORR_ESEQ with no block integrated.
 * When every block is device memory with 16-byte aligned rows and needs no
 * corner turn (CORR_L_CIT, or CORR_L_TCI where the cross-multiply reads the
 * payload order itself), and the context is not pipelined, all blocks run
 * as ONE persistent cross-multiply launch: the tasks of all blocks are spread
 * over the SMs together, so the last, partly filled wave of tasks is paid
 * once instead of once per block.  Every block then adds its partial sums
 * with reductions at L2 into an accumulator that a new integration zeroes
 * first.  Otherwise the call pushes the blocks one by one, and on an error
 * the blocks before the failing one stay integrated.  Stream order and the
 * lifetime of the blocks are as for corr_push.  The context keeps two small
 * device tables of the blocks' parameters; a call with the same blocks and
 * integration buffer as one of the last two reuses its table.
 */
#define CORR_MAX_PUSH_MANY 4096
int corr_push_many(corr_ctx* ctx, const void* const* blocks, int n_blocks, size_t nbytes,
                   uint64_t seq);

/*
 * corr_set_pipeline -- overlap the corner turn of each block with the
 * cross-multiply of the block pushed before it.
 *   turn_sms : > 0 -> each push's corner turn runs as turn_sms persistent
 *              CTAs (one per SM) on an internal stream, and its cross-multiply
 *              on the other SMs of a second internal stream, so that the turn
 *              of block k+1 overlaps the cross-multiply of block k; the context
 *              keeps a second corner-turned buffer (allocated here).
 *              0 -> one stream again.  Must be below the device's SM count.
 * Only for configurations that turn their blocks (4-bit and 8-bit CORR_L_TCI,
 * CORR_L_TIC), else CORR_EINVAL.  Waits for the context's work first.
 * Stream order while pipelined: work queued on the context's stream after a
 * corr_push waits for that block's corner turn (the only reader of the
 * block), not for its cross-multiply; corr_dump, corr_dump_async, corr_sync,
 * corr_normalise and corr_restore wait for every cross-multiply.
 */
int corr_set_pipeline(corr_ctx* ctx, int turn_sms);

/*
 * corr_dump -- copy the integrated visibilities out.
 *   vis   : int64 [C][N(N+1)/2][2], host or device memory; may be NULL to
 *           only reset.
 *   reset : nonzero -> the integration restarts from zero afterwards.
 * Waits for all pushed work.  Returns the first deferred device error
 * (CORR_ERANGE, CORR_ETIMEDOUT) if one occurred since the last check.
 */
int corr_dump(corr_ctx* ctx, int64_t* vis, int reset);

/*
 * corr_dump_async -- overlapped dump: queue the copy of the integrated
 * visibilities into vis and return without waiting.
 *   vis   : int64 [C][N(N+1)/2][2], device or host memory (pinned host memory
 *           keeps the call asynchronous; a pageable buffer makes it wait).
 *           vis holds the sums once the matching corr_dump_wait returns.
 *   reset : nonzero -> the next integration starts from zero at once, in a
 *           second accumulator (allocated on the first such call), so pushes
 *           after this call overlap the copy; zero -> pushes after this call
 *           wait for the copy and then keep adding to the same sums.
 * At most CORR_MAX_ASYNC_DUMPS dumps may be outstanding (CORR_EBUSY beyond).
 * The deferred device status of the blocks in the dumped integration
 * (CORR_ERANGE, CORR_ETIMEDOUT) is returned by its corr_dump_wait, not by a
 * later corr_sync / corr_dump.  A host block pushed before this call may be
 * changed once the matching corr_dump_wait returns.  CORR_EINVAL for a null
 * argument.
 */
#define CORR_MAX_ASYNC_DUMPS 4
int corr_dump_async(corr_ctx* ctx, int64_t* vis, int reset);

/*
 * corr_dump_wait -- wait for the oldest outstanding corr_dump_async (dumps
 * complete in the order they were queued) and return its status.
 * CORR_ESTATE when no dump is outstanding.
 */
int corr_dump_wait(corr_ctx* ctx);

/*
 * corr_bind -- integrate in place in the caller's device buffer.  The next
 * integration is accumulated directly in vis instead of the context's own
 * accumulator, so that a dump into vis copies nothing: the long integration
 * of Sec. 2 lands where the caller reads it.
 *   vis : int64 [C][N(N+1)/2][2] in device memory (the layout corr_dump
 *         writes), owned by the caller, who must neither read nor write it
 *         until the integration's dump (corr_dump, or the corr_dump_wait of
 *         a corr_dump_async) has returned.  Work queued on the context's
 *         stream before the first push is ordered before the first write.
 * Call between integrations: after corr_create, or after a dump with reset
 * and before the next push.  corr_dump / corr_dump_async into vis itself
 * then copy nothing (with reset = 0, vis simply goes on accumulating); a dump
 * into another buffer copies from vis as usual.  The binding ends with the
 * next dump with reset; corr_restore and corr_normalise act on vis while it
 * is bound.  CORR_EINVAL for NULL or a host pointer, CORR_ESTATE after a
 * push into the current integration.
 */
int corr_bind(corr_ctx* ctx, int64_t* vis);

/*
 * corr_normalise -- correlation coefficients of the current integration:
 * rho_ij = V_ij / sqrt(V_ii * V_jj) computed in FP64 on the GPU as
 * double(V_ij) / sqrt(double(V_ii) * double(V_jj)); rho = 0 where
 * V_ii * V_jj == 0.  (Not defined by the paper; provided for monitoring.)
 *   rho : double [C][N(N+1)/2][2], host or device memory.
 * Does not reset the integration.
 */
int corr_normalise(corr_ctx* ctx, double* rho);

/*
 * corr_normalise_flags -- corr_normalise that also reports where the
 * coefficient is undefined.  The paper defines no normalisation; the rule is
 * the one above: rho = 0 where V_ii * V_jj == 0 (an input that was silent
 * over the whole integration), and then zero_flag = 1 for that baseline.
 *   rho       : double [C][N(N+1)/2][2], host or device memory.
 *   zero_flag : uint8 [C][N(N+1)/2], host or device memory, or NULL (then
 *               this is corr_normalise): 1 where V_ii * V_jj == 0, else 0.
 * Synchronous for host buffers, stream-ordered for device buffers.  Errors
 * as corr_normalise; CORR_ENOMEM if a host buffer's staging copy cannot be
 * allocated.
 */
int corr_normalise_flags(corr_ctx* ctx, double* rho, uint8_t* zero_flag);

/* corr_sync -- wait for all pushed work and queued dumps; returns any deferred
 * device error not already returned by corr_dump_wait. */
int corr_sync(corr_ctx* ctx);

/* corr_destroy -- free the context (waits for its work first).  NULL is ok. */
int corr_destroy(corr_ctx* ctx);

/* corr_strerror -- static description of a status code. */
const char* corr_strerror(int status);

/* corr_n_baselines -- N(N+1)/2, or 0 for N < 1. */
int64_t corr_n_baselines(int n_inputs);

/*
 * corr_restore -- resume an integration from a saved state (checkpoint /
 * resume: a corr_dump with reset = 0 is the snapshot).
 *   vis : int64 [C][N(N+1)/2][2], host or device, as corr_dump wrote it.
 * The context's running integration becomes vis; later pushes add to it.
 * The sequence check restarts (any seq is accepted next).  Stream-ordered;
 * vis is read before the call returns.  CORR_EINVAL for a null argument.
 */
int corr_restore(corr_ctx* ctx, const int64_t* vis);

/*
 * Run-time counters of a context, in the spirit of the per-thread key/value
 * status buffer of the paper's pipeline manager (Sec. 2.2, Hashpipe status).
 * Device times are summed over launches since the context was created and
 * are only collected while timing is on (corr_set_timing): each timed
 * kernel or copy is bracketed by CUDA events on the context's stream.
 */
typedef struct corr_stats {
  uint64_t blocks;          /* blocks integrated                              */
  uint64_t seq_rejects;     /* pushes rejected with CORR_ESEQ                 */
  uint64_t dumps;           /* corr_dump calls                                */
  uint64_t turn_launches;   /* corner-turn kernels launched                   */
  uint64_t herk_launches;   /* cross-multiply kernels launched                */
  uint64_t norm_launches;   /* normalisation kernels launched                 */
  double turn_ms;           /* device time in corner-turn kernels (timed)     */
  double herk_ms;           /* device time in cross-multiply kernels (timed)  */
  double copy_in_ms;        /* device time of host-to-device block copies     */
  double dump_ms;           /* device time of visibility copies out           */
  double norm_ms;           /* device time in normalisation kernels           */
  uint64_t timed_turn;      /* launches included in turn_ms                   */
  uint64_t timed_herk;      /* launches included in herk_ms                   */
} corr_stats;

/*
 * corr_set_fault_injection -- test hook for the failure detection of the
 * device-side waits (the paper has no counterpart; its pipeline monitor of
 * Sec. 2.2 only reports status).  Every wait inside the cross-multiply is
 * bounded; when one runs out the kernel records CORR_ETIMEDOUT in the
 * context's status word, lets every role of the CTA leave (no copy or MMA
 * left in flight, tensor memory freed) and returns, so the context stays
 * usable.  This call makes that happen on purpose:
 *   stage       : >= 0: the first CTA of every later cross-multiply never
 *                 loads its stage `stage` (128-spectrum steps of its task
 *                 list), so the waits for it run out; -1 turns it off.
 *   wait_log2   : 1 .. 40 limits every wait to 2^wait_log2 SM cycles
 *                 instead of the default budget of 2^31 (about a second);
 *                 0 restores the default.
 * The visibilities of a push made with a fault are undefined and its dump
 * returns CORR_ETIMEDOUT.  Only the 4-bit TMA path of corr_push (row
 * strides that are multiples of 16 bytes) reads the hook.  Waits for the
 * context's work first.  CORR_EINVAL for stage outside -1 .. 2^24 - 2 or
 * wait_log2 outside 0 .. 40.
 */
int corr_set_fault_injection(corr_ctx* ctx, int stage, int wait_log2);

/* corr_set_timing -- turn per-phase device timing on (1) or off (0). */
int corr_set_timing(corr_ctx* ctx, int on);

/* corr_get_stats -- wait for the context's work and fill *out. */
int corr_get_stats(corr_ctx* ctx, corr_stats* out);

/*
 * corr_correlate_noalloc -- the visibilities of ONE block, for callers that
 * cannot allocate device memory (an allocator owned by another framework,
 * allocation frozen after start-up, or a real-time loop where a cudaMalloc
 * could stall).  The paper has no counterpart: it is a packaging of the
 * corr_create/corr_push/corr_dump path that allocates nothing.
 *
 * The library keeps every intermediate (work list, status word, the
 * corner-turned copy of the block) in one fixed device array of
 * CORR_NOALLOC_SCRATCH_BYTES that exists on every device that loads the
 * library, for the life of the process.  The call itself allocates nothing
 * and frees nothing, on host or device.
 *   block   : device pointer on the current device, N * C * T * bits / 4
 *             bytes in `layout` (4-bit; corr_correlate_noalloc_bits below
 *             takes 8-bit blocks too).
 *   vis     : device pointer on the current device, int64 [C][N(N+1)/2][2];
 *             overwritten with this block's visibilities (not added to).
 *   status  : optional device int on the current device; receives the device
 *             status bits of this call (0 ok, 1 a bounded device-side wait ran
 *             out, 2 an 8-bit sample equal to -128 was integrated).  The call returns before the GPU has run the work, so a
 *             device-side failure is reported only here: a caller that passes
 *             NULL does not learn of it.
 *   stream  : cudaStream_t to run on (NULL: the legacy default stream).
 * Limits: 256 + 20 * tasks (rounded up to 256) + (8-bit: 65536 * SMs) +
 * (turned ? R * C * ceil32(T) : 0) bytes must fit the scratch, where tasks is
 * C / (128 / 2^ceil(log2 2N)) rounded up for 2N <= 64, else C times the tasks
 * of one channel, R = N (4-bit) or 2N (8-bit) byte rows, and a block is
 * turned unless it is 4-bit CORR_L_CIT or a payload-order (CORR_L_TCI) block
 * whose rows the cross-multiply reads in place (R a multiple of 16 and at
 * least 64 (4-bit) or 128 (8-bit) byte rows, or R = 16 or 32, or R = 64 at
 * 8 bits; 16-byte aligned); larger requests return CORR_EINVAL.  Host pointers, and device
 * pointers of another GPU, return CORR_EINVAL.  CORR_ECUDA if the device
 * lacks the shared memory the cross-multiply needs.  Asynchronous: returns
 * once the work is queued.
 * Set-up: the first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.
 * Concurrency: every call shares the one scratch array, which keeps the last
 * call's contents.  Calls that overlap on the GPU (other streams, other host
 * threads on the same device) race and corrupt each other; issue them in
 * order on one stream.
 */
#define CORR_NOALLOC_SCRATCH_BYTES (16u << 20)
int corr_correlate_noalloc(const void* block, int n_inputs, int n_chans, int n_time, int layout,
                           unsigned flags, int64_t* vis, int* status, void* stream);

/*
 * corr_correlate_noalloc_bits -- corr_correlate_noalloc with the sample width
 * of corr_create: bits = 4 (the call above) or 8 (two int8 bytes, re and im,
 * per complex sample, symmetric range -127..127; a -128 is integrated exactly
 * and reported as status bit 2; CORR_F_LO_IS_REAL is invalid with 8 bits).
 * The 8-bit cross-multiply keeps per-SM partial sums in the scratch (64 KB a
 * streaming multiprocessor), which leaves less room for a turned block.
 * Everything else is as for corr_correlate_noalloc.
 */
int corr_correlate_noalloc_bits(const void* block, int n_inputs, int n_chans, int n_time, int bits,
                                int layout, unsigned flags, int64_t* vis, int* status, void* stream);

/*
 * Batches: several arrays correlated in one persistent launch.
 *
 * A correlator node may serve several arrays (or subarrays) at once, each
 * with its own input count, channel count and block length (the paper's
 * Sec. 2 node takes F/N channels of M m inputs; here the shapes differ).
 * A batch holds every array's device state and correlates one block of
 * every array per run: the corner turns, then ONE persistent cross-multiply
 * launch over all arrays' tasks, replayed from a CUDA graph.  The task
 * schedule (tile grouping, assignment of tasks to SMs) can be autotuned at
 * creation by timing candidate schedules on the device.
 */
typedef struct corr_shape {
  int n_inputs;   /* N, 1 <= N <= 1024                                      */
  int n_chans;    /* C >= 1                                                 */
  int n_time;     /* T spectra per block, 1 <= T <= 65536 (4-bit), 32768 (8-bit) */
  int bits;       /* 4 or 8 (the same for every array of a batch)           */
  int layout;     /* CORR_L_*                                               */
  unsigned flags; /* CORR_F_* (the same for every array of a batch)         */
} corr_shape;

typedef struct corr_batch corr_batch; /* opaque, owned by the library */

/* Schedules an autotuned batch can choose from (corr_batch_info.schedule). */
#define CORR_SCHED_PAIRS_LPT 0   /* 128x256 tasks, longest-first onto the least loaded SM */
#define CORR_SCHED_SINGLES_LPT 1 /* 128x128 tasks, longest-first                      */
#define CORR_SCHED_PAIRS_RR 2    /* 128x256 tasks, round robin in list order           */

/* schedule, n_tasks and n_ctas describe the single-launch form;
 * launches_per_run counts the graph corr_batch_run replays now (more once
 * corr_batch_set_pipeline has split the run). */
typedef struct corr_batch_info {
  int schedule;          /* CORR_SCHED_* in use                                  */
  int n_tasks;           /* tasks of one cross-multiply launch                   */
  int n_ctas;            /* CTAs (one per SM)                                    */
  int launches_per_run;  /* kernels one corr_batch_run launches                  */
  double tuned_ms[3];    /* median run time of each schedule (autotune), else 0  */
  int tune_source;       /* 0 default schedule, 1 timed now, 2 from the tune cache */
} corr_batch_info;

/*
 * corr_batch_create -- device state for n arrays (inputs, corner-turn
 * copies, int64 visibilities) and the run's CUDA graph.
 *   shapes : n array shapes; every array must have the same bits and flags.
 *   stream : cudaStream_t for the runs; NULL or a default stream (legacy,
 *            per-thread), on which no graph can be captured, gives a private
 *            stream (the caller then orders its own work with corr_batch_sync).
 *   tune   : 0 uses CORR_SCHED_PAIRS_LPT; 1 times every schedule on the
 *            device (on the current contents of the input buffers) and keeps
 *            the fastest.  If the environment variable XE_TUNE_CACHE names a
 *            file, a result for the same GPU (name, SM count) and the same
 *            shapes is taken from it instead of timing, and new results are
 *            appended to it (JSON lines: key, schedule, tuned_ms).
 * Returns CORR_EINVAL for a bad shape or mixed bits/flags, CORR_ENOMEM,
 * CORR_ECUDA.
 */
int corr_batch_create(const corr_shape* shapes, int n, void* stream, int tune, corr_batch** out);

/* Device buffer of array k's input block (N C T bits/4 bytes, the array's
 * layout); the caller fills it before corr_batch_run.  NULL if k is invalid. */
void* corr_batch_input(corr_batch* b, int k);

/* Device int64 [C][N(N+1)/2][2] visibilities of array k's last block, valid
 * after the run completes (corr_batch_sync).  NULL if k is invalid. */
int64_t* corr_batch_output(corr_batch* b, int k);

/* Copy array k's block in (host or device src, exactly N C T bits/4 bytes),
 * or its visibilities out (host or device dst, N(N+1)/2 C 2 int64), ordered
 * on the batch's stream; CORR_EINVAL for a bad k, pointer or size. */
int corr_batch_set_input(corr_batch* b, int k, const void* src, size_t nbytes);
int corr_batch_get_output(corr_batch* b, int k, int64_t* dst);

/* corr_batch_run -- correlate the current block of every array (the outputs
 * are overwritten, not accumulated): replays the batch's CUDA graph on its
 * stream.  Asynchronous. */
int corr_batch_run(corr_batch* b);

/* corr_batch_run_plain -- the same work as one corner turn and one
 * cross-multiply launch per array, without a graph (the comparison form).
 * Asynchronous. */
int corr_batch_run_plain(corr_batch* b);

/*
 * corr_batch_set_pipeline -- overlap the corner turn with the cross-multiply
 * inside each run.  The array with the most bytes to turn (4-bit, [t][c][i]
 * or [t][i][c], more than 32 inputs) is turned in n_chunks channel ranges on
 * turn_sms SMs of a second stream, while the other SMs cross-multiply the
 * other arrays and then each range as soon as it is turned.  The graph that
 * corr_batch_run replays is re-captured in that form (a few launches per
 * run instead of one).  turn_sms = 0 restores the single-launch form.
 * Waits for the batch's stream.  CORR_EINVAL for turn_sms outside
 * 0 .. SMs - 1, n_chunks < 1, or no array that can be split so.
 */
int corr_batch_set_pipeline(corr_batch* b, int turn_sms, int n_chunks);

/* Wait for the batch's stream; returns a pending device status (CORR_ERANGE,
 * CORR_ETIMEDOUT) once, else CORR_OK. */
int corr_batch_sync(corr_batch* b);

int corr_batch_info_get(corr_batch* b, corr_batch_info* out);
void corr_batch_destroy(corr_batch* b);

/*
 * corr_plan_schedule -- longest-processing-time-first assignment of tasks to
 * CTAs (host only; no device needed).
 *   cost      : n_tasks task costs (any positive unit).
 *   order     : out, n_tasks task indices grouped by CTA, each CTA's tasks in
 *               decreasing cost.
 *   cta_first : out, n_ctas + 1 offsets into order (CTA b runs
 *               order[cta_first[b] .. cta_first[b + 1]) ).
 * Tasks are taken in decreasing cost and each goes to the CTA with the least
 * total so far (ties: lowest index).  Returns CORR_EINVAL for bad arguments.
 */
int corr_plan_schedule(const double* cost, int n_tasks, int n_ctas, int* order, int* cta_first);

/*
 * Streaming service: continuous batching of integration requests.
 *
 * The paper's pipeline integrates for a pre-set duration and then dumps
 * (Sec. 2, Sec. 2.2).  The service generalises that to many concurrent
 * integrations of different arrays and lengths sharing one GPU: each request
 * asks for n_blocks blocks of block_spectra spectra of one array.  Requests
 * are admitted in arrival order while their device state (int64 accumulator,
 * two ingest buffers, the corner-turn buffer) fits in a fixed HBM budget,
 * carved out of one allocation made at creation.  Every tick correlates the
 * pending block of every active request in one persistent launch (one per
 * sample width), so requests that arrive while others run join the next
 * tick; a request's blocks are copied in on a second stream while the
 * previous tick computes.  When its last block is integrated the request is
 * done; corr_svc_fetch copies its visibilities out and frees its memory,
 * which admits queued requests.  Latency = submit to done (host clock, the
 * completion observed by a host callback on the stream).
 *
 * Not thread-safe: one host thread drives a service.
 */
typedef struct corr_svc corr_svc; /* opaque, owned by the library */

typedef struct corr_req {
  int n_inputs;       /* N, 1 <= N <= 1024                              */
  int n_chans;        /* C >= 1                                         */
  int bits;           /* 4 or 8                                         */
  int layout;         /* CORR_L_*                                       */
  unsigned flags;     /* CORR_F_*                                       */
  int block_spectra;  /* spectra per block, <= 65536 (4-bit), 32768 (8-bit); for CORR_L_CIT
                         at 4 bits a multiple of 16 */
  int64_t n_blocks;   /* blocks to integrate, >= 1                      */
} corr_req;

#define CORR_SVC_DRY_RUN 1u /* host logic only: no device memory, no kernels (tests) */

#define CORR_REQ_QUEUED 0   /* waiting for memory                        */
#define CORR_REQ_ACTIVE 1   /* admitted: accepts blocks                  */
#define CORR_REQ_DONE 2     /* every block integrated; fetch the result  */
#define CORR_REQ_FETCHED 3  /* result copied out, memory released        */

typedef struct corr_svc_stats {
  uint64_t submitted, admitted, completed, fetched;
  uint64_t ticks;            /* corr_svc_tick calls that launched work    */
  uint64_t launches;         /* kernels launched by ticks                  */
  uint64_t blocks;           /* blocks integrated                          */
  double chan_spectra;       /* sum over integrated blocks of C x spectra  */
  double ops;                /* correlator ops integrated (8 N(N+1)/2 C T) */
  double p50_ms, p99_ms, max_ms; /* submit-to-done latency of done requests */
  uint64_t budget, in_use, peak_in_use; /* bytes of the HBM budget         */
  int active, queued;
} corr_svc_stats;

/* corr_svc_create -- a service with hbm_budget bytes of device state (one
 * allocation now).  flags: CORR_SVC_DRY_RUN or 0.  stream as for batches. */
int corr_svc_create(size_t hbm_budget, unsigned flags, void* stream, corr_svc** out);

/* corr_svc_submit -- queue a request; it is admitted at once if its state
 * fits.  *id receives its handle.  CORR_EINVAL for a bad shape, CORR_EBUSY if
 * it could never fit the budget. */
int corr_svc_submit(corr_svc* s, const corr_req* r, int64_t* id);

/* corr_svc_state -- CORR_REQ_* of a request.  CORR_EINVAL for an unknown id. */
int corr_svc_state(corr_svc* s, int64_t id, int* state);

/* corr_svc_push -- the request's next block (host or device memory, N C T
 * bits/4 bytes in its layout), copied in on the ingest stream.  The copy is
 * ordered after nothing the caller queued: a device block must be complete
 * when the call is made (synchronize its producer first).  The block may be
 * reused once the tick that integrates it has completed (corr_svc_wait).
 * CORR_ESTATE unless the request is active and still expects blocks;
 * CORR_EBUSY while two pushed blocks are waiting for ticks. */
int corr_svc_push(corr_svc* s, int64_t id, const void* block, size_t nbytes);

/* corr_svc_tick -- correlate the oldest waiting block of every active
 * request in one launch per sample width.  *n_requests (optional) receives
 * how many requests took part.  Asynchronous. */
int corr_svc_tick(corr_svc* s, int* n_requests);

/* corr_svc_fetch -- for a done request: copy its visibilities (int64
 * [C][N(N+1)/2][2], host or device; NULL to discard), release its memory and
 * admit queued requests.  CORR_ESTATE if it is not done yet. */
int corr_svc_fetch(corr_svc* s, int64_t id, int64_t* vis);

/* corr_svc_wait -- wait for the work queued so far; returns a pending device
 * status once (CORR_ERANGE, CORR_ETIMEDOUT), else CORR_OK. */
int corr_svc_wait(corr_svc* s);

int corr_svc_stats_get(corr_svc* s, corr_svc_stats* out);
void corr_svc_destroy(corr_svc* s);

#ifdef __cplusplus
}
#endif
#endif /* XENGINE_H */
