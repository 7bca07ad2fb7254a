"""F-engine oracle -- TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of the F-engine front end of arXiv:1904.07778
(Sec. 2.1, "F-engine"): polyphase filter bank with a Hamming-windowed
prototype, FFT of 2C real samples per spectrum, the two-real-signals-in-one-
complex-FFT separation (Eq. 2), the 18-bit PFB output, and the equaliser /
requantiser to 4-bit fix_4_3 codes with its RMS gain rule (Eq. 3).  numpy in
float64 for the filter bank and the DFT (numpy.fft as the library step);
plain integer arithmetic for the equaliser.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; it shares nothing with the CUDA package.

Readings of the paper (it leaves these open):
  * prototype filter: h[m] = w[m] sinc((m - (L-1)/2) / M), m = 0 .. L-1,
    L = taps * M, M = 2C real samples per spectrum (critically sampled real
    FFT), w the Hamming window 0.54 - 0.46 cos(2 pi m / (L-1));
  * spectrum t of input i: y[n] = sum_q h[q M + n] x[(t + q) M + n],
    X[c] = sum_n y[n] exp(-2 pi j c n / M) for c = 0 .. C-1 (the Nyquist bin
    is dropped);
  * 18-bit output (fix_18_17 as an integer): v = clamp(rne(X / 2^shift),
    -2^17, 2^17 - 1) per component, rne = round half to even;
  * equaliser: gain g an unsigned 18-bit integer (fix_18_7), p = v g is
    fix_36_24; "rounded even from the 21st bit, then the 22nd to 25th bits"
    counts bits from the least significant one: q = rne(p / 2^21), kept in
    the symmetric fix_4_3 range -7 .. 7 by saturation;
  * packing: real part in the high nibble, imaginary in the low nibble
    (or swapped with lo_is_real);
  * gain rule (Eq. 3): RMS = sqrt(P / (2 n)) with P the summed power
    v_re^2 + v_im^2 of n spectra; g = rne(target 2^21 / RMS) clamped to
    1 .. 2^18 - 1, and g = 0 for a silent input (P = 0).
"""
from __future__ import annotations

import numpy as np

FIX18_MIN, FIX18_MAX = -(1 << 17), (1 << 17) - 1
GAIN_MAX = (1 << 18) - 1


def pfb_coeffs(n_chans: int, taps: int) -> np.ndarray:
    """Prototype filter of the PFB (Sec. 2.1: Hamming window times sinc),
    length taps * 2C, float64."""
    M = 2 * n_chans
    L = taps * M
    m = np.arange(L, dtype=np.float64)
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * m / (L - 1))
    return w * np.sinc((m - (L - 1) / 2.0) / M)


def pfb_frames(x: np.ndarray, n_chans: int, taps: int, n_spectra: int,
               h: np.ndarray | None = None) -> np.ndarray:
    """Filtered frames y[t][n] of one input's samples x (at least
    (n_spectra + taps - 1) * 2C of them), float64 [T][2C]."""
    M = 2 * n_chans
    if h is None:
        h = pfb_coeffs(n_chans, taps)
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros((n_spectra, M), dtype=np.float64)
    for q in range(taps):
        y += h[q * M:(q + 1) * M][None, :] * x[q * M:(q + n_spectra) * M].reshape(n_spectra, M)
    return y


def spectra(adc: np.ndarray, n_chans: int, taps: int, n_spectra: int) -> tuple[np.ndarray, np.ndarray]:
    """Channelised spectra of every input.

    adc: int8 [n_inputs][n_samples], n_samples >= (n_spectra + taps - 1) 2C.
    Returns (X, absum): X complex128 [T][C][n_inputs], and absum float64
    [T][n_inputs] = sum_n |y[n]| of each filtered frame (for error bounds).
    """
    n_inputs = adc.shape[0]
    h = pfb_coeffs(n_chans, taps)
    X = np.empty((n_spectra, n_chans, n_inputs), dtype=np.complex128)
    absum = np.empty((n_spectra, n_inputs), dtype=np.float64)
    for i in range(n_inputs):
        y = pfb_frames(adc[i], n_chans, taps, n_spectra, h)
        X[:, :, i] = np.fft.fft(y, axis=1)[:, :n_chans]
        absum[:, i] = np.abs(y).sum(axis=1)
    return X, absum


def separate(S: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 2: from S = DFT(x1 + j x2) of two real sequences (last axis, length
    M) recover DFT(x1) and DFT(x2)."""
    M = S.shape[-1]
    neg = S[..., (-np.arange(M)) % M]          # S[-nu]
    Sr, Si, Sr_n, Si_n = S.real, S.imag, neg.real, neg.imag
    X1 = (Sr + Sr_n) / 2 + 1j * (Si - Si_n) / 2
    X2 = (Si + Si_n) / 2 - 1j * (Sr - Sr_n) / 2
    return X1, X2


def rne(a: np.ndarray) -> np.ndarray:
    """Round half to even, float64 -> int64."""
    return np.rint(a).astype(np.int64)


def to_fix18(X: np.ndarray, shift: int = 0) -> np.ndarray:
    """18-bit PFB output: int64 [..., 2] (re, im), saturated."""
    v = np.stack([rne(np.ldexp(X.real, -shift)), rne(np.ldexp(X.imag, -shift))], axis=-1)
    return np.clip(v, FIX18_MIN, FIX18_MAX)


def rne_shift(p: np.ndarray, s: int) -> np.ndarray:
    """Integer round-half-to-even of p / 2^s (p int64)."""
    p = np.asarray(p, dtype=np.int64)
    fl = p >> s                                  # floor
    rem = p - (fl << s)                          # 0 .. 2^s - 1
    half = np.int64(1) << (s - 1)
    up = (rem > half) | ((rem == half) & ((fl & 1) == 1))
    return fl + up.astype(np.int64)


def equalise(v: np.ndarray, gain: np.ndarray) -> np.ndarray:
    """Equaliser / requantiser: 18-bit v (int64 [..., C, N, 2]) times the
    fix_18_7 gain (integer [C, N]) -> fix_4_3 codes int64 [..., C, N, 2] in
    -7 .. 7."""
    g = np.asarray(gain, dtype=np.int64)[..., None]
    p = np.asarray(v, dtype=np.int64) * g        # fix_36_24, |p| < 2^35
    return np.clip(rne_shift(p, 21), -7, 7)


def pack(q: np.ndarray, lo_is_real: bool = False) -> np.ndarray:
    """Two 4-bit two's complement codes [..., 2] -> one byte."""
    re = q[..., 0].astype(np.int64) & 0xF
    im = q[..., 1].astype(np.int64) & 0xF
    return ((im << 4) | re if lo_is_real else (re << 4) | im).astype(np.uint8)


def power(v: np.ndarray) -> np.ndarray:
    """Summed power of 18-bit spectra [T][C][N][2] -> int64 [C][N]."""
    v = np.asarray(v, dtype=np.int64)
    return (v[..., 0] ** 2 + v[..., 1] ** 2).sum(axis=0)


def gains_from_power(P: np.ndarray, n_spectra: int, target_rms: float = 2.5) -> np.ndarray:
    """Eq. 3 gain rule: RMS = sqrt(P / (2 n)); g = rne(target 2^21 / RMS),
    clamped to 1 .. 2^18 - 1; 0 where P == 0.  int64 [C][N]."""
    P = np.asarray(P, dtype=np.int64)
    g = np.zeros(P.shape, dtype=np.int64)
    live = P > 0
    rms = np.sqrt(P[live].astype(np.float64) / (2.0 * n_spectra))
    g[live] = np.clip(np.rint(target_rms * 2097152.0 / rms), 1, GAIN_MAX).astype(np.int64)
    return g


def fengine(adc: np.ndarray, n_chans: int, taps: int, n_spectra: int, gain: np.ndarray,
            shift: int = 0, lo_is_real: bool = False) -> dict:
    """The whole front end: 18-bit spectra, fix_4_3 codes, packed bytes in
    [t][c][i] order (the payload order of Sec. 2.3) and the summed power."""
    X, absum = spectra(adc, n_chans, taps, n_spectra)
    v = to_fix18(X, shift)
    q = equalise(v, gain)
    return {"X": X, "absum": absum, "v": v, "q": q, "bytes": pack(q, lo_is_real),
            "power": power(v)}
