/*
 * fengine.h -- C ABI of the GPU F-engine front end (arXiv:1904.07778,
 * Sec. 2.1 "F-engine"): polyphase filter bank, FFT of two real inputs in one
 * complex transform (Eq. 2), 18-bit spectra, and the equaliser / requantiser
 * to 4-bit fix_4_3 codes packed as the X-engine's input (xengine.h).
 *
 * What one spectrum is.  With M = 2C real samples per spectrum and L = taps M
 * filter coefficients h[m] = w[m] sinc((m - (L-1)/2) / M), w the Hamming
 * window 0.54 - 0.46 cos(2 pi m / (L-1)), spectrum t of input i is
 *   y[n] = sum_{q < taps} h[q M + n] x_i[(t + q) M + n],   n = 0 .. M-1
 *   X[c] = sum_n y[n] exp(-2 pi j c n / M),                 c = 0 .. C-1
 * computed in FP32 on the GPU (two inputs per complex FFT, separated with
 * Eq. 2).  The 18-bit PFB output (Sec. 2.1) is v = clamp(rne(X / 2^shift),
 * -2^17, 2^17 - 1) per component (rne = round half to even).  The equaliser
 * multiplies v by an unsigned 18-bit gain g (fix_18_7) into a fix_36_24
 * product p and keeps q = clamp(rne(p / 2^21), -7, 7), the fix_4_3 code;
 * the real and imaginary codes share one byte, real in the high nibble
 * unless FE_F_LO_IS_REAL.
 *
 * Conventions as in xengine.h: int status returns (FE_* = CORR_* codes),
 * stream-ordered asynchronous calls, caller-owned buffers.
 */
#pragma once
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ctx fe_ctx;

#define FE_F_LO_IS_REAL 0x1u /* real part in the low nibble of each byte */

/*
 * fe_create -- a channeliser for one array.
 *   n_inputs : >= 1 real input streams (inputs 2k, 2k+1 share one FFT; an odd
 *              last input is paired with zeros).
 *   n_chans  : C, a power of two in [16, 2048]; M = 2C samples per spectrum.
 *   taps     : PFB taps, 1 .. 16.
 *   shift    : 0 .. 24, the power of two divided out before the 18-bit
 *              rounding (the FFT's scaling).
 *   flags    : FE_F_* bits.
 *   stream   : cudaStream_t to run on, or NULL for a private stream.
 * Builds the coefficient and twiddle tables on the host (FP64 rounded to
 * FP32) and copies them to the current device.  All gains start at 0.
 * CORR_EINVAL for a bad argument, CORR_ENOMEM, CORR_ECUDA.
 */
int fe_create(int n_inputs, int n_chans, int taps, int shift, unsigned flags, void* stream,
              fe_ctx** out);

/*
 * fe_set_gains -- equaliser gains, uint32 [C][n_inputs] (host or device),
 * each < 2^18 (fix_18_7, value g / 128).  CORR_EINVAL if one is larger.
 * Stream-ordered; the buffer is read before the call returns.
 */
int fe_set_gains(fe_ctx* ctx, const uint32_t* gain);

/*
 * fe_channelise -- T spectra of every input.
 *   adc        : int8 samples, device memory, input i's stream at
 *                adc + i * adc_stride, at least (T + taps - 1) M samples per
 *                input (spectrum t starts at sample t M; the first taps - 1
 *                frames are the previous block's history).
 *   adc_stride : samples between inputs.
 *   n_spectra  : T >= 1.
 *   out        : packed codes, device memory, or NULL.
 *   layout     : CORR_L_CIT (2): out[(c N + i) out_stride + t], the
 *                X-engine's pre-turned order (out_stride >= T);
 *                CORR_L_TCI (0): out[(t C + c) N + i], the payload order of
 *                Sec. 2.3 (out_stride ignored).
 *   v18        : NULL or int32 [T][C][N][2] (device): the 18-bit spectra.
 *   spec       : NULL or float [T][C][N][2] (device): X / 2^shift before
 *                rounding, as the GPU computed it.
 *   power      : NULL or int64 [C][N] (device): sum over the T spectra of
 *                v_re^2 + v_im^2 is ADDED to it (Eq. 3's P).
 * CORR_EINVAL for a bad argument or a host pointer.
 */
int fe_channelise(fe_ctx* ctx, const int8_t* adc, long long adc_stride, int n_spectra,
                  uint8_t* out, int layout, long long out_stride, int32_t* v18, float* spec,
                  int64_t* power);

/*
 * fe_gains_from_power -- Eq. 3 on the host: RMS = sqrt(P / (2 T)) per
 * (channel, input) from the summed power of T spectra, and the gain that
 * brings it to target_rms: g = rne(target_rms 2^21 / RMS) clamped to
 * 1 .. 2^18 - 1, g = 0 where P = 0.  power and gain are host arrays of
 * n_chans * n_inputs.  Pure host code (no device work).
 */
int fe_gains_from_power(const int64_t* power, int n_chans, int n_inputs, long long n_spectra,
                        double target_rms, uint32_t* gain);

/* fe_sync -- wait for the context's work. */
int fe_sync(fe_ctx* ctx);

/* fe_destroy -- free the context (waits for its work first).  NULL is ok. */
void fe_destroy(fe_ctx* ctx);

#ifdef __cplusplus
}
#endif
