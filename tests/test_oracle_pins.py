"""Pins of the X-engine oracle against values fixed by the paper and by
mathematics (not against the oracle itself).

Each test names what it pins.  A plausible mistake in the oracle -- swapped
conjugation, a wrong nibble, a transposed layout index, a dropped term in the
real or imaginary part, a wrong baseline index -- fails at least one test.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1904_07778_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bidx(i, j):
    return i * (i + 1) // 2 + j


def _full_matrix(vis_c, n):
    """Hermitian N x N complex matrix from one channel's lower triangle."""
    m = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        for j in range(i + 1):
            v = vis_c[_bidx(i, j), 0] + 1j * vis_c[_bidx(i, j), 1]
            m[i, j] = v
            m[j, i] = np.conj(v)
    return m


# --- golden fixtures (hand-evaluated) ------------------------------------------

def test_golden_nibble_decode():
    """Sec. 2.1 equaliser output: two 4-bit two's-complement numbers per byte."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "nibble_decode.txt"))
            if l.strip() and not l.startswith("#")]
    blk = np.array([int(r[0], 16) for r in rows], dtype=np.uint8)
    re, im = oracle.decode(blk, 1, 1, len(rows), bits=4, layout=oracle.L_CIT)
    assert re[0, 0].tolist() == [int(r[1]) for r in rows]
    assert im[0, 0].tolist() == [int(r[2]) for r in rows]
    # the other nibble order swaps the parts
    re2, im2 = oracle.decode(blk, 1, 1, len(rows), bits=4, layout=oracle.L_CIT, hi_is_real=False)
    assert re2.tolist() == im.tolist() and im2.tolist() == re.tolist()


def test_golden_hand_visibilities():
    """Hand-evaluated sum_t x_i conj(x_j) for 4-bit and 8-bit examples."""
    for line in open(os.path.join(GOLDEN, "vis_hand.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        left, right = line.split("|")
        f = left.split()
        bits, n, t = int(f[1]), int(f[2]), int(f[3])
        blk = np.array([int(x, 16) for x in f[4:]], dtype=np.uint8)
        want = np.array([int(x) for x in right.split()], dtype=np.int64).reshape(1, -1, 2)
        got = oracle.correlate(blk, n, 1, t, bits=bits, layout=oracle.L_TCI)
        assert np.array_equal(got, want), (f[0], got, want)


# --- brute force on tiny inputs ------------------------------------------------

def _brute(re, im):
    """Definition evaluated with Python complex numbers, one term at a time."""
    C, N, T = re.shape
    out = np.zeros((C, N * (N + 1) // 2, 2), dtype=np.int64)
    for c in range(C):
        for i in range(N):
            for j in range(i + 1):
                s = 0j
                for t in range(T):
                    xi = complex(int(re[c, i, t]), int(im[c, i, t]))
                    xj = complex(int(re[c, j, t]), int(im[c, j, t]))
                    s += xi * xj.conjugate()
                out[c, _bidx(i, j)] = (int(s.real), int(s.imag))
    return out


@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("hi", [True, False])
def test_brute_force_tiny(bits, layout, hi):
    """Decode + layout indexing + conjugation vs brute force (N, T, C tiny)."""
    clip = 8 if bits == 4 else 127
    rng = np.random.default_rng(100 + bits + 10 * layout + hi)
    for N, T, C in [(1, 1, 1), (2, 2, 3), (3, 7, 2), (5, 2, 1), (4, 5, 3)]:
        re = rng.integers(-clip, clip + (0 if bits == 4 else 1), size=(C, N, T)).astype(np.int8)
        im = rng.integers(-clip, clip + (0 if bits == 4 else 1), size=(C, N, T)).astype(np.int8)
        blk = synth.pack(re, im, bits=bits, layout=layout, hi_is_real=hi)
        got = oracle.correlate(blk, N, C, T, bits=bits, layout=layout, hi_is_real=hi, threads=2)
        assert np.array_equal(got, _brute(re, im)), (N, T, C)


def test_exhaustive_byte_pairs():
    """Every pair of 4-bit complex codes (256 x 256), T = 1, against complex
    products evaluated from an independent numpy decode of the nibbles."""
    b0, b1 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    C = 65536
    blk = np.stack([b0.reshape(-1), b1.reshape(-1)], axis=-1).astype(np.uint8).reshape(-1)
    # layout [t][c][i] with T = 1: bytes ordered (c, i)
    got = oracle.correlate(blk, 2, C, 1, bits=4, layout=oracle.L_TCI)

    def dec(b):
        hi = (b >> 4).astype(np.int64)
        lo = (b & 15).astype(np.int64)
        return np.where(hi >= 8, hi - 16, hi) + 1j * np.where(lo >= 8, lo - 16, lo)

    x0, x1 = dec(b0.reshape(-1)), dec(b1.reshape(-1))
    for b, v in ((0, x0 * np.conj(x0)), (1, x1 * np.conj(x0)), (2, x1 * np.conj(x1))):
        assert np.array_equal(got[:, b, 0], v.real.astype(np.int64))
        assert np.array_equal(got[:, b, 1], v.imag.astype(np.int64))


# --- closed forms --------------------------------------------------------------

@pytest.mark.parametrize("bits", [4, 8])
def test_constant_input_closed_form(bits):
    """x_i(t) = a_i + i b_i for all t gives V_ij = T (a_i a_j + b_i b_j) +
    i T (b_i a_j - a_i b_j)."""
    N, C, T = 6, 3, 37
    a = np.array([1, -3, 7, 0, -8 if bits == 4 else -127, 5])
    b = np.array([2, 4, -7, 0, 3, -1 if bits == 4 else 126])
    re = np.broadcast_to(a[None, :, None], (C, N, T)).astype(np.int8)
    im = np.broadcast_to(b[None, :, None], (C, N, T)).astype(np.int8)
    for layout in (0, 1, 2):
        got = oracle.correlate(synth.pack(re, im, bits=bits, layout=layout), N, C, T, bits=bits,
                               layout=layout)
        for i in range(N):
            for j in range(i + 1):
                assert got[1, _bidx(i, j), 0] == T * (a[i] * a[j] + b[i] * b[j])
                assert got[1, _bidx(i, j), 1] == T * (b[i] * a[j] - a[i] * b[j])


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_impulse_lights_one_row(layout):
    """A single nonzero sample at (c0, i0, t0) contributes only to the
    auto-correlation of input i0 in channel c0 (pins layout indexing)."""
    N, C, T = 5, 4, 9
    for (c0, i0, t0) in [(0, 0, 0), (3, 4, 8), (2, 1, 5), (1, 3, 0)]:
        re = np.zeros((C, N, T), np.int8)
        im = np.zeros((C, N, T), np.int8)
        re[c0, i0, t0], im[c0, i0, t0] = 3, -2
        got = oracle.correlate(synth.pack(re, im, layout=layout), N, C, T, layout=layout)
        want = np.zeros_like(got)
        want[c0, _bidx(i0, i0)] = (13, 0)
        assert np.array_equal(got, want)
        # with a constant companion input the impulse lights exactly row/column i0
        re[c0, :, t0] = 1
        re[c0, i0, t0] = 3
        got = oracle.correlate(synth.pack(re, im, layout=layout), N, C, T, layout=layout)
        for i in range(N):
            for j in range(i + 1):
                v = got[c0, _bidx(i, j)]
                xi = complex(re[c0, i, t0], im[c0, i, t0])
                xj = complex(re[c0, j, t0], im[c0, j, t0])
                e = xi * xj.conjugate()
                assert (v[0], v[1]) == (int(e.real), int(e.imag))
        other = [c for c in range(C) if c != c0]
        assert not got[other].any()


# --- invariants ----------------------------------------------------------------

def test_invariants_random():
    """Autos real and non-negative; Cauchy-Schwarz |V_ij|^2 <= V_ii V_jj;
    linearity in time; permuting inputs permutes V."""
    N, C, T = 7, 5, 64
    blk = synth.random_bytes(5, N * C * T)
    v = oracle.correlate(blk, N, C, T, layout=2)
    for i in range(N):
        assert (v[:, _bidx(i, i), 1] == 0).all()
        assert (v[:, _bidx(i, i), 0] >= 0).all()
    for c in range(C):
        for i in range(N):
            for j in range(i):
                p = int(v[c, _bidx(i, j), 0]) ** 2 + int(v[c, _bidx(i, j), 1]) ** 2
                assert p <= int(v[c, _bidx(i, i), 0]) * int(v[c, _bidx(j, j), 0])
    # linearity in time: two half blocks add up to the whole
    x = blk.reshape(C, N, T)
    v1 = oracle.correlate(np.ascontiguousarray(x[:, :, :20]).reshape(-1), N, C, 20, layout=2)
    v2 = oracle.correlate(np.ascontiguousarray(x[:, :, 20:]).reshape(-1), N, C, T - 20, layout=2)
    assert np.array_equal(v1 + v2, v)
    # accumulate-into form gives the same
    acc = oracle.correlate(np.ascontiguousarray(x[:, :, :20]).reshape(-1), N, C, 20, layout=2)
    oracle.correlate(np.ascontiguousarray(x[:, :, 20:]).reshape(-1), N, C, T - 20, layout=2, out=acc)
    assert np.array_equal(acc, v)
    # permutation of inputs
    perm = np.random.default_rng(1).permutation(N)
    vp = oracle.correlate(np.ascontiguousarray(x[:, perm, :]).reshape(-1), N, C, T, layout=2)
    for c in range(C):
        m, mp = _full_matrix(v[c], N), _full_matrix(vp[c], N)
        assert np.array_equal(mp, m[np.ix_(perm, perm)])
    # channel subset equals the matching rows of the full result
    sub = oracle.correlate(blk, N, C, T, layout=2, chans=[4, 0, 2])
    assert np.array_equal(sub, v[[4, 0, 2]])


def test_total_power_identity():
    """sum_i V_ii = sum_t sum_i |x_i|^2."""
    N, C, T = 9, 3, 50
    blk = synth.random_bytes(8, N * C * T)
    v = oracle.correlate(blk, N, C, T, layout=0)
    nib = lambda n: np.where(n >= 8, n - 16, n)
    x = blk.reshape(T, C, N).astype(np.int64)
    p = (nib(x >> 4) ** 2 + nib(x & 15) ** 2).sum(axis=(0, 2))
    autos = sum(v[:, _bidx(i, i), 0] for i in range(N))
    assert np.array_equal(autos, p)


def test_projected_power_is_quadratic_form():
    """sum_t |sum_i conj(w_i) x_i|^2 == w^H V w (Hermitian quadratic form)."""
    N, C, T = 6, 4, 40
    for bits in (4, 8):
        blk = synth.random_bytes(11 + bits, N * C * T * bits // 4)
        if bits == 8:
            blk[blk == 0x80] = 0x7F
        v = oracle.correlate(blk, N, C, T, bits=bits, layout=1)
        rng = np.random.default_rng(2)
        w = rng.integers(-1, 2, size=(5, N)) + 1j * rng.integers(-1, 2, size=(5, N))
        pp = oracle.projected_power(blk, N, C, T, w, bits=bits, layout=1)
        for c in range(C):
            m = _full_matrix(v[c], N)
            for k in range(5):
                q = np.conj(w[k]) @ m @ w[k]
                assert q.imag == 0 and int(q.real) == pp[c, k]


def test_projected_power_brute_force_every_layout_and_thread_count():
    """The projected power against a direct numpy evaluation of its
    definition (decode by hand, then sum over time of |w^H x(t)|^2), for every
    layout, a channel subset and one or several threads."""
    N, C, T = 5, 7, 33
    rng = np.random.default_rng(31)
    w = rng.integers(-2, 3, size=(3, N)) + 1j * rng.integers(-2, 3, size=(3, N))
    nib = lambda n: np.where(n >= 8, n - 16, n)
    for layout in (0, 1, 2):
        blk = synth.random_bytes(40 + layout, N * C * T)
        shape = {0: (T, C, N), 1: (T, N, C), 2: (C, N, T)}[layout]
        perm = {0: (1, 2, 0), 1: (2, 1, 0), 2: (0, 1, 2)}[layout]
        b = blk.reshape(shape).transpose(perm).astype(np.int64)   # [C][N][T]
        x = nib(b >> 4) + 1j * nib(b & 15)
        want = np.array([[int(np.rint((np.abs(np.conj(wv) @ x[c]) ** 2).sum())) for wv in w]
                         for c in range(C)])
        for threads in (1, 3):
            got = oracle.projected_power(blk, N, C, T, w, layout=layout, threads=threads)
            assert np.array_equal(got, want), (layout, threads)
        sub = [6, 0, 3]
        got = oracle.projected_power(blk, N, C, T, w, layout=layout, chans=sub, threads=2)
        assert np.array_equal(got, want[sub])


def test_minus_128_rejected():
    """8-bit -128 lies outside the symmetric quantiser and is an error."""
    blk = np.array([0x80, 0x00, 0x01, 0x02], dtype=np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.correlate(blk, 2, 1, 1, bits=8)


# --- the paper's own identities ------------------------------------------------

def test_fx_equals_xf():
    """Sec. 2: multiplying in frequency equals convolving (correlating) in
    time, so FX and XF correlators agree.  XF: circular lagged correlation
    r_ij[l] = sum_n x_i[n+l] conj(x_j[n]), then DFT over l.  FX: DFT of each
    series, then the oracle's cross-multiply over blocks."""
    rng = np.random.default_rng(3)
    N, L, nblk = 4, 16, 5
    xs = rng.integers(-7, 8, size=(nblk, N, L)) + 1j * rng.integers(-7, 8, size=(nblk, N, L))
    # XF side, written with explicit loops
    xf = np.zeros((L, N, N), dtype=np.complex128)
    for b in range(nblk):
        for i in range(N):
            for j in range(N):
                r = np.array([sum(xs[b, i, (n + l) % L] * np.conj(xs[b, j, n]) for n in range(L))
                              for l in range(L)])
                xf[:, i, j] += np.array([sum(r[l] * np.exp(-2j * np.pi * k * l / L) for l in range(L))
                                         for k in range(L)])
    # FX side: spectra per block are the "samples" of each frequency channel
    X = np.fft.fft(xs, axis=2)  # [blk][N][k]
    fx = oracle.correlate_complex(X.transpose(2, 1, 0))  # [C=k][N][T=blk]
    for k in range(L):
        for i in range(N):
            for j in range(i + 1):
                assert abs(fx[k, _bidx(i, j)] - xf[k, i, j]) <= 1e-9 * max(1.0, abs(xf[k, i, j]))


def test_complex_and_integer_paths_agree():
    """The FP64 complex form of the definition equals the int64 form exactly."""
    N, C, T = 5, 3, 30
    blk = synth.random_bytes(21, N * C * T)
    v = oracle.correlate(blk, N, C, T, layout=0)
    re, im = oracle.decode(blk, N, C, T, layout=0)
    vc = oracle.correlate_complex(re + 1j * im)
    assert np.array_equal(vc.real.astype(np.int64), v[..., 0])
    assert np.array_equal(vc.imag.astype(np.int64), v[..., 1])


@pytest.mark.parametrize("amp", [0.5, 2.0])
def test_delay_phase_slope(amp):
    """Sec. 3, Eq. 5: a common signal seen with a relative delay gives a
    visibility phase linear in frequency.  With the sky model x_i =
    Q(amp s e^{j phi_i(c)} + n_i), arg V_ij(c) = phi_i(c) - phi_j(c), so the
    channel-to-channel phase step is 2 pi (tau_i - tau_j) / C (sign fixed by
    the conjugation convention)."""
    N, C, T = 4, 64, 4096
    re, im = synth.sky(9, N, C, T, amp=amp)
    v = oracle.correlate(synth.pack(re, im, layout=2), N, C, T, layout=2)
    tau, phi0 = synth.sky_params(9, N, C)
    for i in range(N):
        for j in range(i):
            z = v[:, _bidx(i, j), 0] + 1j * v[:, _bidx(i, j), 1]
            step = np.angle(np.sum(z[1:] * np.conj(z[:-1])))
            want = 2 * np.pi * (tau[i] - tau[j]) / C
            d = (step - want + np.pi) % (2 * np.pi) - np.pi
            assert abs(d) < 0.05, (i, j, step, want)
            # absolute phase at channel 0 matches phi0_i - phi0_j
            d0 = (np.angle(z[0]) - (phi0[i] - phi0[j]) + np.pi) % (2 * np.pi) - np.pi
            assert abs(d0) < (0.6 if amp < 1 else 0.2)


def test_autocorrelation_statistics():
    """E[V_ii] = T * 2 E[Q(X)^2] for X ~ N(0, sigma^2) rounded and clipped to
    +-7 (the equaliser target RMS 2-3, Sec. 2.1); checked within 5 sigma
    using the exact discretised-Gaussian moments."""
    sigma, N, C, T = 2.5, 8, 16, 2048
    Phi = lambda z: 0.5 * (1 + math.erf(z / math.sqrt(2)))
    p = {}
    for k in range(-7, 8):
        lo = -math.inf if k == -7 else (k - 0.5) / sigma
        hi = math.inf if k == 7 else (k + 0.5) / sigma
        p[k] = (Phi(hi) if hi != math.inf else 1.0) - (Phi(lo) if lo != -math.inf else 0.0)
    m2 = sum(k * k * q for k, q in p.items())
    m4 = sum(k ** 4 * q for k, q in p.items())
    mean = T * 2 * m2
    sd = math.sqrt(T * 2 * (m4 - m2 * m2))
    blk = synth.block("gauss", 4, N, C, T, layout=0)
    v = oracle.correlate(blk, N, C, T, layout=0)
    autos = np.array([v[:, _bidx(i, i), 0] for i in range(N)], dtype=np.float64)
    assert np.all(np.abs(autos - mean) < 5 * sd)
    # the RMS of the quantised output lands in the paper's 2..3 target band
    rms = math.sqrt(autos.mean() / (2 * T))
    assert 2.0 < rms < 3.0


# --- normalisation -------------------------------------------------------------

def test_normalise_properties():
    """rho_ii = 1; |rho_ij| <= 1; x_j = i x_i gives rho_ji = +i; x_j = -x_i
    gives rho_ji = -1; an all-zero input gives rho = 0 with the flag set;
    rho is invariant to scaling an input."""
    N, C, T = 5, 2, 33
    rng = np.random.default_rng(4)
    re = rng.integers(-5, 6, size=(C, N, T)).astype(np.int8)
    im = rng.integers(-5, 6, size=(C, N, T)).astype(np.int8)
    re[:, 1], im[:, 1] = -im[:, 0], re[:, 0]  # x1 = i x0
    re[:, 2], im[:, 2] = -re[:, 0], -im[:, 0]  # x2 = -x0
    re[:, 4], im[:, 4] = 0, 0
    v = oracle.correlate(synth.pack(re, im, bits=8, layout=2), N, C, T, bits=8, layout=2)
    rho, flags = oracle.normalise(v, N)
    for c in range(C):
        for i in range(4):
            assert rho[c, _bidx(i, i), 0] == 1.0 and rho[c, _bidx(i, i), 1] == 0.0
        assert np.allclose(rho[c, _bidx(1, 0)], [0.0, 1.0], rtol=0, atol=1e-15)
        assert np.allclose(rho[c, _bidx(2, 0)], [-1.0, 0.0], rtol=0, atol=1e-15)
        for j in range(5):
            b = _bidx(4, j)
            assert rho[c, b].tolist() == [0.0, 0.0] and flags[c, b] == 1
    assert np.all(np.hypot(rho[..., 0], rho[..., 1]) <= 1 + 1e-15)
    re3, im3 = re.copy(), im.copy()
    re3[:, 3] *= 3
    im3[:, 3] *= 3
    v3 = oracle.correlate(synth.pack(re3, im3, bits=8, layout=2), N, C, T, bits=8, layout=2)
    rho3, _ = oracle.normalise(v3, N)
    assert np.allclose(rho3, rho, rtol=1e-14, atol=1e-15)
