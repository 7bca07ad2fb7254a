"""Pins of the F-engine oracle (oracle/fengine.py) against hand derivations,
closed forms and invariants -- never against the oracle's own formula.

What each group pins:
  * prototype values at C = 1 and C = 2 derived by hand with exact
    trigonometric values: window length L - 1, sinc scale M = 2C, centre
    (L - 1) / 2;
  * an impulse through the filter bank: which frame meets which tap, the
    sign of the DFT exponent, the dropped Nyquist bin;
  * the paper's Eq. 2 on a hand example and against separate DFTs;
  * rounding ties and saturation of the 18-bit output and of the
    equaliser (bit 20 rounds, bits 21..24 kept, symmetric -7..7);
  * nibble packing through the X-engine oracle's own decoder;
  * Eq. 3 on constant inputs, and the RMS the rule produces on noise.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fengine as fe

SQ2 = math.sqrt(2.0)


def test_prototype_c1_taps2_by_hand():
    # L = 4, M = 2.  Window: 0.54 - 0.46 cos(2 pi m / 3) = 0.08, 0.77, 0.77, 0.08
    # (cos(2 pi / 3) = cos(4 pi / 3) = -1/2).  sinc((m - 1.5) / 2) at -0.75,
    # -0.25, 0.25, 0.75 = (sqrt2 / 2) / (0.75 pi), (sqrt2 / 2) / (0.25 pi), ...
    want = [0.08 * 2 * SQ2 / (3 * math.pi), 0.77 * 2 * SQ2 / math.pi,
            0.77 * 2 * SQ2 / math.pi, 0.08 * 2 * SQ2 / (3 * math.pi)]
    assert np.allclose(fe.pfb_coeffs(1, 2), want, rtol=1e-14, atol=0)


def test_prototype_c2_taps1_by_hand():
    # L = 4, M = 4: same window; sinc((m - 1.5) / 4) at -3/8, -1/8, 1/8, 3/8 with
    # sin(3 pi / 8) = sqrt(2 + sqrt2) / 2 and sin(pi / 8) = sqrt(2 - sqrt2) / 2.
    s38 = math.sqrt(2 + SQ2) / 2 / (3 * math.pi / 8)
    s18 = math.sqrt(2 - SQ2) / 2 / (math.pi / 8)
    want = [0.08 * s38, 0.77 * s18, 0.77 * s18, 0.08 * s38]
    assert np.allclose(fe.pfb_coeffs(2, 1), want, rtol=1e-14, atol=0)


def test_prototype_symmetric_and_peaked():
    h = fe.pfb_coeffs(64, 4)
    assert h.size == 4 * 128
    assert np.allclose(h, h[::-1], rtol=0, atol=1e-15)
    assert np.argmax(h) in (255, 256) and h.max() < 1.0


@pytest.mark.parametrize("s,taps", [(0, 4), (3 * 16 + 5, 4), (7 * 16 + 15, 3), (40, 1)])
def test_impulse_through_filter_bank(s, taps):
    """x = delta[s]: spectrum t sees it through tap q = s // M - t at
    n0 = s % M only, so X_t[c] = h[q M + n0] exp(-2 pi j c n0 / M)."""
    C, T = 8, 6
    M = 2 * C
    adc = np.zeros((1, (T + taps - 1) * M), dtype=np.int8)
    adc[0, s] = 1
    X, _ = fe.spectra(adc, C, taps, T)
    h = fe.pfb_coeffs(C, taps)
    n0 = s % M
    for t in range(T):
        q = s // M - t
        amp = h[q * M + n0] if 0 <= q < taps else 0.0
        for c in range(C):
            want = amp * complex(math.cos(2 * math.pi * c * n0 / M), -math.sin(2 * math.pi * c * n0 / M))
            assert abs(X[t, c, 0] - want) < 1e-12, (t, c)


def test_linear_in_inputs():
    rng = np.random.default_rng(1)
    a = rng.integers(-100, 100, (2, 5 * 32), dtype=np.int64).astype(np.int8)
    b = rng.integers(-20, 20, (2, 5 * 32), dtype=np.int64).astype(np.int8)
    Xa, _ = fe.spectra(a, 16, 3, 3)
    Xb, _ = fe.spectra(b, 16, 3, 3)
    Xab, _ = fe.spectra((a.astype(np.int16) + b).astype(np.int8), 16, 3, 3)
    assert np.allclose(Xab, Xa + Xb, rtol=0, atol=1e-9)


def test_eq2_hand_example():
    # x1 = delta[0] -> X1 = 1 1 1 1; x2 = delta[1] -> X2 = 1 -j -1 j;
    # S = X1 + j X2 = (1+j) 2 (1-j) 0.
    S = np.array([1 + 1j, 2, 1 - 1j, 0], dtype=np.complex128)
    X1, X2 = fe.separate(S)
    assert np.allclose(X1, [1, 1, 1, 1]) and np.allclose(X2, [1, -1j, -1, 1j])


def test_eq2_matches_separate_transforms():
    rng = np.random.default_rng(2)
    x1, x2 = rng.normal(size=(2, 5, 64))
    X1, X2 = fe.separate(np.fft.fft(x1 + 1j * x2, axis=-1))
    assert np.allclose(X1, np.fft.fft(x1, axis=-1), rtol=0, atol=1e-12)
    assert np.allclose(X2, np.fft.fft(x2, axis=-1), rtol=0, atol=1e-12)


def test_fix18_ties_and_saturation():
    X = np.array([2.5, 3.5, -2.5, -3.5, 0.5, -0.5, 1.49999, 131071.4, 131072.0, -131072.6])
    v = fe.to_fix18(X + 0j)[..., 0]
    assert v.tolist() == [2, 4, -2, -4, 0, 0, 1, 131071, 131071, -131072]
    v1 = fe.to_fix18(np.array([5.0 + 7j, -5.0 - 3j]), shift=1)
    assert v1.tolist() == [[2, 4], [-2, -2]]   # 2.5 -> 2, 3.5 -> 4, -2.5 -> -2, -1.5 -> -2


# (v, g, q): with g = 2^11, p = v 2^11 and q = rne(v / 2^10)
EQ_CASES = [
    (1024, 2048, 1), (1536, 2048, 2), (2560, 2048, 2), (512, 2048, 0), (1535, 2048, 1),
    (1537, 2048, 2), (-1536, 2048, -2), (-2560, 2048, -2), (-512, 2048, 0), (-513, 2048, -1),
    (7168, 2048, 7), (8192, 2048, 7), (-8192, 2048, -7), (-131072, 2048, -7),
    # fractional gains: p = v g, q = rne(p / 2^21)
    (131071, 1, 0),            # 0.0625
    (8, 262143, 1),            # 0.999996
    (4, 262143, 0),            # 0.499998
    (-4, 262143, 0),           # -0.499998
    (12, 262144 - 1, 1),       # 1.499994
    (3, 349525 // 2, 0),       # 3 * 174762 / 2^21 = 0.249999
    (0, 262143, 0),
]


@pytest.mark.parametrize("v,g,q", EQ_CASES)
def test_equaliser_hand_cases(v, g, q):
    got = fe.equalise(np.array([[[[v, -v]]]]), np.array([[g]]))
    assert got[0, 0, 0].tolist() == [q, -q]     # rounding and saturation are symmetric


def test_equaliser_never_emits_minus_eight():
    v = np.arange(-(1 << 17), 1 << 17, 97, dtype=np.int64)
    q = fe.equalise(np.stack([v, v], -1)[:, None, None, :], np.array([[(1 << 18) - 1]]))
    assert q.min() == -7 and q.max() == 7


def test_pack_nibbles_through_xengine_decoder():
    """Packed codes decode, in the X-engine oracle, to the same integers:
    the autocorrelation of one input is sum(re^2 + im^2) and the cross term
    with a second input holds re/im in the right places."""
    assert fe.pack(np.array([-1, 3])) == 0xF3
    assert fe.pack(np.array([-1, 3]), lo_is_real=True) == 0x3F
    assert fe.pack(np.array([-7, 7])) == 0x97
    rng = np.random.default_rng(3)
    q = rng.integers(-7, 8, (50, 1, 2, 2))       # [t][c][i][re/im]
    blk = fe.pack(q)                              # [t][c][i], the payload order
    vis = oracle.correlate(blk.reshape(-1), 2, 1, 50, bits=4, layout=oracle.L_TCI)
    x = q[..., 0] + 1j * q[..., 1]
    v10 = np.sum(x[:, 0, 1] * np.conj(x[:, 0, 0]))
    assert vis[0, 0, 0] == np.sum(np.abs(x[:, 0, 0]) ** 2) and vis[0, 0, 1] == 0
    assert vis[0, 1, 0] == v10.real and vis[0, 1, 1] == v10.imag


def test_gain_rule_constant_inputs():
    # v = (100, 100) for 10 spectra: P = 200000, RMS = sqrt(P / 20) = 100,
    # g = rne(2.5 * 2^21 / 100) = rne(52428.8) = 52429.
    P = np.array([[200000, 10 * 2 * 1024 ** 2, 0, 1]])
    g = fe.gains_from_power(P, 10)
    assert g[0, 0] == 52429
    assert g[0, 1] == 5120                      # RMS 1024: 2.5 * 2048 exactly
    assert g[0, 2] == 0                          # silent input
    assert g[0, 3] == (1 << 18) - 1              # RMS 0.22: clamped
    assert fe.gains_from_power(np.array([[200000]]), 10, target_rms=2.0)[0, 0] == 41943  # 41943.04


def test_gain_rule_sets_output_rms():
    """Eq. 3's factor 2: after the rule, Gaussian 18-bit spectra come out of
    the equaliser with per-component RMS near the target (rounding adds
    1/12 to the variance; saturation at 7 = 2.8 sigma removes a little)."""
    rng = np.random.default_rng(4)
    n = 200000
    v = np.rint(rng.normal(0, 900.0, (n, 1, 1, 2))).astype(np.int64)
    g = fe.gains_from_power(fe.power(v), n)
    q = fe.equalise(v, g)
    rms = math.sqrt(np.mean(q.astype(np.float64) ** 2))
    assert abs(rms - math.sqrt(2.5 ** 2 + 1 / 12)) < 0.03


def test_fengine_composes_the_steps():
    rng = np.random.default_rng(5)
    C, taps, T, N = 16, 4, 5, 3
    adc = rng.integers(-60, 61, (N, (T + taps - 1) * 2 * C)).astype(np.int8)
    gain = rng.integers(1, 1 << 18, (C, N))
    out = fe.fengine(adc, C, taps, T, gain, shift=1)
    X, _ = fe.spectra(adc, C, taps, T)
    assert np.array_equal(out["v"], fe.to_fix18(X, 1))
    assert np.array_equal(out["bytes"], fe.pack(fe.equalise(out["v"], gain)))
    assert out["bytes"].shape == (T, C, N)
