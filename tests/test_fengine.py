"""Parity of the GPU F-engine (include/fengine.h) with the F-engine oracle.

The spectra are FP32 on the GPU and FP64 in the oracle, so parity has three
layers:
  1. |spec_gpu - X / 2^shift| <= E elementwise, E the a-priori bound of the
     arithmetic (below);
  2. decisions taken in the GPU's precision are bit-exact: v18 = clamp(rne(
     spec)), the codes = the oracle equaliser applied to v18, and the power
     = the oracle's sum over v18;
  3. v18 equals the oracle's 18-bit value wherever X / 2^shift is farther
     than E from a rounding tie (it is unique there), and is one of the two
     neighbours elsewhere.

The bound E (per spectrum and input pair, u = 2^-24): the filter's FP32 fused
multiply-adds and the FP32 coefficients cost at most (taps + 1) u sum_q |h x|
per sample; every one of the log2 M radix-2 levels of the FFT (radix-8 and
radix-4 passes are three and two such levels) rounds a twiddle product and a
sum, at most 4 u times the largest partial sum, which sum_n |z[n]| bounds;
Eq. 2 adds one rounding of the result.  Summed over the samples:
E = u ((taps + 1) sum_n sum_q |h x| + (4 log2 M + 1) sum_n |z[n]|) / 2^shift.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import fengine as ofe  # noqa: E402
from paper_1904_07778_gb300 import synth  # noqa: E402

U = 2.0 ** -24


@pytest.fixture(scope="module")
def fe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300 import fengine
    return fengine


def _bound(adc, C, taps, T, shift):
    """E [T][pairs] of the module docstring, from the oracle's filter."""
    N = adc.shape[0]
    h = np.abs(ofe.pfb_coeffs(C, taps))
    afir = np.stack([ofe.pfb_frames(np.abs(adc[i].astype(np.float64)), C, taps, T, h).sum(axis=1)
                     for i in range(N)], axis=1)                     # [T][N]
    _, absum = ofe.spectra(adc, C, taps, T)                          # [T][N]
    P = (N + 1) // 2
    pad = lambda a: np.concatenate([a, np.zeros((T, 2 * P - N))], axis=1) if N % 2 else a
    afir, absum = pad(afir), pad(absum)
    afir_p = afir[:, 0::2] + afir[:, 1::2]
    ay_p = absum[:, 0::2] + absum[:, 1::2]
    logm = math.log2(2 * C)
    return U * ((taps + 1) * afir_p + (4 * logm + 1) * ay_p) / 2.0 ** shift


def _run(fe, adc, C, taps, T, shift, gain, layout=2, lo_is_real=False, out_stride=None,
         adc_stride=None, with_power=True):
    N = adc.shape[0]
    dev = torch.device("cuda")
    S = adc_stride or adc.shape[1]
    a = torch.zeros((N, S), dtype=torch.int8, device=dev)
    a[:, :adc.shape[1]] = torch.from_numpy(adc).to(dev)
    if layout == 2:
        os_ = out_stride or T
        out = torch.full((C * N * os_,), 0xEE, dtype=torch.uint8, device=dev)
    else:
        os_ = 0
        out = torch.full((T * C * N,), 0xEE, dtype=torch.uint8, device=dev)
    v18 = torch.zeros((T, C, N, 2), dtype=torch.int32, device=dev)
    spec = torch.zeros((T, C, N, 2), dtype=torch.float32, device=dev)
    power = torch.zeros((C, N), dtype=torch.int64, device=dev) if with_power else None
    with fe.FEngine(N, C, taps, shift, lo_is_real=lo_is_real) as f:
        f.set_gains(gain)
        f.channelise(a.view(-1), T, out=out, layout=layout, out_stride=os_, v18=v18, spec=spec,
                     power=power, adc_stride=S)
        f.sync()
    out = out.cpu().numpy()
    if layout == 2:
        codes = out.reshape(C, N, os_)[:, :, :T].transpose(2, 0, 1)  # -> [t][c][i]
        pad = out.reshape(C, N, os_)[:, :, T:]
    else:
        codes, pad = out.reshape(T, C, N), np.zeros(0)
    return {"codes": codes, "pad": pad, "v18": v18.cpu().numpy().astype(np.int64),
            "spec": spec.cpu().numpy().astype(np.float64),
            "power": power.cpu().numpy() if power is not None else None}


def _check(got, adc, C, taps, T, shift, gain, lo_is_real=False):
    N = adc.shape[0]
    X, _ = ofe.spectra(adc, C, taps, T)
    Xs = np.stack([X.real, X.imag], axis=-1) / 2.0 ** shift              # [T][C][N][2]
    E = np.repeat(_bound(adc, C, taps, T, shift), 2, axis=1)[:, :N]      # [T][N]
    E = E[:, None, :, None]
    err = np.abs(got["spec"] - Xs)
    assert np.all(err <= E), float((err / E).max())
    # decisions in the GPU's precision
    v = got["v18"]
    assert np.array_equal(v, np.clip(np.rint(got["spec"]), -(1 << 17), (1 << 17) - 1).astype(np.int64))
    assert np.array_equal(got["codes"], ofe.pack(ofe.equalise(v, gain), lo_is_real))
    if got["power"] is not None:
        assert np.array_equal(got["power"], ofe.power(v))
    # the 18-bit values against the oracle's where they are unique
    vo = ofe.to_fix18(X, shift)
    frac = Xs - np.floor(Xs)
    unique = (np.abs(frac - 0.5) > E) | (np.abs(Xs) > (1 << 17) + 1)
    assert np.array_equal(v[unique], vo[unique])
    assert np.all(np.abs(v - vo) <= 1)
    return float(np.mean(v == vo))


def _gains(rng, C, N, lo=2000, hi=60000):
    return rng.integers(lo, hi, (C, N)).astype(np.uint32)


CASES = [  # (N, C, taps, T, shift)
    (2, 16, 1, 32, 0), (2, 16, 4, 33, 0), (3, 32, 4, 40, 1), (4, 64, 2, 64, 0),
    (5, 128, 8, 17, 2), (8, 256, 4, 96, 0), (6, 512, 4, 70, 1), (4, 1024, 4, 64, 0),
    (2, 2048, 4, 33, 3), (1, 64, 3, 5, 0),
    # one FFT unit per CTA (frame-major filter) with fewer taps and ragged groups
    (3, 1024, 2, 41, 0), (2, 2048, 1, 9, 1), (4, 1024, 3, 35, 0),
]


@pytest.mark.parametrize("N,C,taps,T,shift", CASES)
def test_fengine_parity(fe, N, C, taps, T, shift):
    rng = np.random.default_rng(N * 1000 + C + taps + T)
    adc = synth.adc(N * 31 + C, N, (T + taps - 1) * 2 * C, sigma=20.0,
                    tones=[(30.0, 5.25 / (2 * C), 0.4)], common=8.0)
    gain = _gains(rng, C, N)
    # the kernel has an instance with Eq. 3's power sums and one without
    got = _run(fe, adc, C, taps, T, shift, gain, with_power=T % 2 == 0)
    assert _check(got, adc, C, taps, T, shift, gain) > 0.99


@pytest.mark.parametrize("layout", [0, 2])
def test_layouts_and_nibble_order(fe, layout):
    N, C, taps, T = 6, 64, 4, 45
    rng = np.random.default_rng(11)
    adc = synth.adc(12, N, (T + taps - 1) * 2 * C)
    gain = _gains(rng, C, N)
    for lo in (False, True):
        got = _run(fe, adc, C, taps, T, 0, gain, layout=layout, lo_is_real=lo)
        _check(got, adc, C, taps, T, 0, gain, lo_is_real=lo)


def test_unaligned_input_and_output_strides(fe):
    """Odd input stride (byte loads) and an output row stride that is not a
    multiple of 16 (byte stores); the gap after each row stays untouched."""
    N, C, taps, T = 4, 32, 4, 64
    rng = np.random.default_rng(12)
    adc = synth.adc(13, N, (T + taps - 1) * 2 * C)
    gain = _gains(rng, C, N)
    got = _run(fe, adc, C, taps, T, 0, gain, out_stride=T + 5, adc_stride=adc.shape[1] + 3)
    _check(got, adc, C, taps, T, 0, gain)
    assert np.all(got["pad"] == 0xEE)


@pytest.mark.parametrize("phase,edge", [(0.0, (1 << 17) - 1), (np.pi, -(1 << 17))])
def test_saturation(fe, phase, edge):
    """A full-scale tone at a bin centre of a 2048-channel transform (|X|
    near 63 x 4096): the real part of that bin saturates at the 18-bit edge
    and the codes reach +-7, never -8."""
    N, C, taps, T = 2, 2048, 4, 32
    adc = synth.adc(14, N, (T + taps - 1) * 2 * C, sigma=1.0, tones=[(126.0, 100 / (2 * C), phase)])
    gain = np.full((C, N), 262143, dtype=np.uint32)
    got = _run(fe, adc, C, taps, T, 0, gain)
    _check(got, adc, C, taps, T, 0, gain)
    v = got["v18"]
    assert np.all(v[:, 100, :, 0] == edge)
    q = ofe.equalise(v, gain)
    assert q.max() == 7 and q.min() == -7


def test_gain_loop_sets_output_rms(fe):
    """Power from the GPU, gains from Eq. 3 in the C ABI, then codes whose
    RMS is the target (the equaliser's purpose, Sec. 2.1)."""
    N, C, taps, T = 8, 256, 4, 256
    adc = synth.adc(15, N, (T + taps - 1) * 2 * C, sigma=12.0, common=6.0)
    ones = np.ones((C, N), dtype=np.uint32)
    first = _run(fe, adc, C, taps, T, 0, ones)
    g = fe.fe_gains_from_power(first["power"], T, 2.5)
    assert np.array_equal(g.astype(np.int64), ofe.gains_from_power(first["power"], T, 2.5))
    got = _run(fe, adc, C, taps, T, 0, g)
    _check(got, adc, C, taps, T, 0, g)
    q = ofe.equalise(got["v18"], g)
    rms = math.sqrt(np.mean(q.astype(np.float64) ** 2))
    assert abs(rms - 2.5) < 0.15


def test_fengine_feeds_the_xengine(fe):
    """The [c][i][t] codes go straight into a correlator context (no corner
    turn) and give the X-engine oracle's visibilities of the same codes."""
    from paper_1904_07778_gb300 import xengine as xe
    N, C, taps, T = 12, 128, 4, 256
    rng = np.random.default_rng(16)
    adc = synth.adc(17, N, (T + taps - 1) * 2 * C, sigma=14.0, common=10.0)
    gain = _gains(rng, C, N, 20000, 40000)
    dev = torch.device("cuda")
    a = torch.from_numpy(adc).to(dev)
    out = torch.empty(C * N * T, dtype=torch.uint8, device=dev)
    with fe.FEngine(N, C, taps, 0) as f, xe.Correlator(N, C, T, bits=4, layout=xe.CORR_L_CIT) as cor:
        f.set_gains(gain)
        f.channelise(a, T, out=out, layout=xe.CORR_L_CIT)
        f.sync()
        cor.push(out)
        vis = cor.dump()
    codes = out.cpu().numpy()
    assert np.array_equal(vis, oracle.correlate(codes, N, C, T, bits=4, layout=oracle.L_CIT))
    # the delay test of Sec. 3: input 1 sees the common source one sample
    # after input 0, so V_10(c) = sum x_1 conj(x_0) turns by -2 pi c / M
    v10 = vis[:, 1, 0] + 1j * vis[:, 1, 1]
    c = np.arange(C)
    rot = np.sum(v10 * np.exp(2j * np.pi * c / (2 * C)))
    coh = np.abs(rot) / np.sum(np.sqrt(vis[:, 0, 0] * vis[:, 2, 0].astype(np.float64)))
    assert abs(np.angle(rot)) < 0.1 and coh > 0.15


def test_full_size_sampled(fe):
    """192 inputs x 1024 channels x 8192 spectra (the cylinder block) in
    one launch; sampled pairs and spectra against the oracle, codes exact
    where the 18-bit value is unique and a neighbour's code elsewhere."""
    N, C, taps, T = 192, 1024, 4, 8192
    M = 2 * C
    S = (T + taps - 1) * M
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    a = torch.empty((N, S), dtype=torch.int8, device=dev)
    for i in range(0, N, 16):
        a[i:i + 16] = torch.clamp(torch.round(torch.randn((16, S), generator=g, device=dev) * 16), -127, 127).to(torch.int8)
    rng = np.random.default_rng(18)
    gain = _gains(rng, C, N, 1500, 3000)
    out = torch.empty(C * N * T, dtype=torch.uint8, device=dev)
    with fe.FEngine(N, C, taps, 0) as f:
        f.set_gains(gain)
        f.channelise(a, T, out=out)
        f.sync()
    codes = out.view(C, N, T)
    for pair, t0 in ((0, 0), (37, 4000), (95, T - 40)):
        i0, nt = 2 * pair, 40
        adc = a[i0:i0 + 2, t0 * M:(t0 + nt + taps - 1) * M].cpu().numpy()
        X, _ = ofe.spectra(adc, C, taps, nt)
        E = np.repeat(_bound(adc, C, taps, nt, 0), 2, axis=1)[:, None, :, None]
        Xs = np.stack([X.real, X.imag], axis=-1)
        lo = np.clip(np.floor(Xs), -(1 << 17), (1 << 17) - 1).astype(np.int64)
        hi = np.clip(lo + 1, -(1 << 17), (1 << 17) - 1)
        gsub = gain[:, i0:i0 + 2]
        got = codes[:, i0:i0 + 2, t0:t0 + nt].cpu().numpy().transpose(2, 0, 1)
        want = ofe.pack(ofe.equalise(ofe.to_fix18(X), gsub))
        unique = np.all((np.abs(Xs - np.floor(Xs) - 0.5) > E), axis=-1)
        assert np.array_equal(got[unique], want[unique])
        alt = [ofe.pack(ofe.equalise(np.stack([r, i], -1), gsub))
               for r in (lo[..., 0], hi[..., 0]) for i in (lo[..., 1], hi[..., 1])]
        assert np.all(np.any(np.stack([got == x for x in alt]), axis=0))
