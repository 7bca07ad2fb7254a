"""Parity of the CUDA X-engine with the oracle, element by element, through
the C ABI.  Integer results must be bit-exact; FP64 correlation
coefficients within 1e-12 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1904_07778_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def xe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300 import xengine
    return xengine


def _run(xe, blocks, N, C, T, layout, lo_is_real=False, device_input=True):
    with xe.Correlator(N, C, T, bits=4, layout=layout, lo_is_real=lo_is_real) as cor:
        for b in blocks:
            if device_input:
                cor.push(torch.from_numpy(b).cuda())
            else:
                cor.push(b)
        return cor.dump()


def _oracle(blocks, N, C, T, layout, lo_is_real=False, chans=None):
    out = None
    for b in blocks:
        out = oracle.correlate(b, N, C, T, bits=4, layout=layout, hi_is_real=not lo_is_real,
                               chans=chans, out=out)
    return out


SHAPES = [
    # (N, C, T): stacked small arrays, one / several 128-row blocks, ragged tails
    (1, 3, 1), (1, 5, 130), (2, 7, 17), (3, 4, 257), (16, 9, 128), (31, 5, 200),
    (32, 6, 1024), (33, 3, 300), (48, 2, 129), (64, 3, 384), (65, 2, 100),
    (100, 2, 513), (192, 2, 256), (257, 1, 160),
]


@pytest.mark.parametrize("N,C,T", SHAPES)
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_random_codes_bit_exact(xe, N, C, T, layout):
    """Uniform random bytes (every 4-bit code incl. -8), every layout."""
    blk = synth.random_bytes(N * 1000 + C * 10 + T + layout, N * C * T)
    got = _run(xe, [blk], N, C, T, layout)
    assert np.array_equal(got, _oracle([blk], N, C, T, layout))


PAYLOAD_SHAPES = [
    # (N, C, T): [t][c][i] blocks read in payload order (16, 32 inputs stacked;
    # 64 or more in 64-row boxes), ragged spectrum counts, odd channel counts
    (16, 7, 77), (16, 9, 256), (32, 5, 200), (32, 3, 1), (64, 3, 130), (128, 2, 129),
    (192, 2, 300), (256, 1, 513), (80, 3, 160),
]


@pytest.mark.parametrize("N,C,T", PAYLOAD_SHAPES)
@pytest.mark.parametrize("lo", [False, True])
def test_payload_order_read_directly(xe, N, C, T, lo):
    """[t][c][i] blocks whose rows suit TMA are cross-multiplied without a
    corner turn: the kernel gathers each input's bytes across time itself."""
    blk = synth.random_bytes(3000 + N * 10 + C + T, N * C * T)
    got = _run(xe, [blk, blk[::-1].copy()], N, C, T, 0, lo_is_real=lo, device_input=not lo)
    assert np.array_equal(got, _oracle([blk, blk[::-1].copy()], N, C, T, 0, lo_is_real=lo))


@pytest.mark.parametrize("lo", [False, True])
def test_nibble_order(xe, lo):
    N, C, T = 8, 4, 64
    blk = synth.random_bytes(77, N * C * T)
    got = _run(xe, [blk], N, C, T, 0, lo_is_real=lo)
    assert np.array_equal(got, _oracle([blk], N, C, T, 0, lo_is_real=lo))


def test_extreme_codes(xe):
    """All -8 (the largest products) and all +7, several blocks integrated."""
    N, C, T = 40, 3, 1024
    a = np.full(N * C * T, 0x88, np.uint8)
    b = np.full(N * C * T, 0x77, np.uint8)
    c = np.full(N * C * T, 0x78, np.uint8)
    got = _run(xe, [a, b, c], N, C, T, 2)
    assert np.array_equal(got, _oracle([a, b, c], N, C, T, 2))


def test_host_and_device_pointers(xe):
    N, C, T = 24, 8, 256
    blks = [synth.block("gauss", s, N, C, T, layout=0) for s in range(3)]
    want = _oracle(blks, N, C, T, 0)
    assert np.array_equal(_run(xe, blks, N, C, T, 0, device_input=False), want)
    pinned = [torch.from_numpy(b).pin_memory() for b in blks]
    with xe.Correlator(N, C, T, layout=0) as cor:
        for p in pinned:
            cor.push(p)
        vis = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda")
        cor.dump_into(vis)
        assert np.array_equal(vis.cpu().numpy(), want)


def test_dump_reset_and_sequence(xe):
    N, C, T = 12, 5, 96
    blks = [synth.random_bytes(s, N * C * T) for s in range(4)]
    with xe.Correlator(N, C, T, layout=2) as cor:
        cor.push(blks[0], seq=10)
        cor.push(blks[1], seq=11)
        assert cor.push(blks[3], seq=13, check=False) == xe.CORR_ESEQ   # gap: not integrated
        assert cor.push(blks[1], seq=11, check=False) == xe.CORR_ESEQ   # duplicate
        v = cor.dump(reset=False)
        assert np.array_equal(v, _oracle(blks[:2], N, C, T, 2))
        cor.push(blks[2], seq=12)
        v = cor.dump(reset=True)
        assert np.array_equal(v, _oracle(blks[:3], N, C, T, 2))
        assert not cor.dump(reset=True).any()          # nothing pushed since the reset
        cor.push(blks[3], seq=99)                        # any seq after a reset
        assert np.array_equal(cor.dump(), _oracle(blks[3:], N, C, T, 2))
        with pytest.raises(xe.CorrError):
            cor.push(blks[0][:-1])                       # wrong size


def test_long_block_chunked(xe):
    """T above the per-accumulation limit (65536 spectra) is split exactly."""
    N, C, T = 4, 2, 70000
    blk = np.full(N * C * T, 0x88, np.uint8)  # worst-case magnitudes
    blk[::7] = 0x7F
    got = _run(xe, [blk], N, C, T, 2)
    assert np.array_equal(got, _oracle([blk], N, C, T, 2))


def test_normalise(xe):
    N, C, T = 20, 4, 512
    blk = synth.block("sky", 3, N, C, T, layout=0)
    blk[:N] = 0  # input bytes of t=0, c=0: keep autos positive but exercise small values
    with xe.Correlator(N, C, T, layout=0) as cor:
        cor.push(blk)
        rho = cor.normalise()
        vis = cor.dump()
    want, _ = oracle.normalise(vis, N)
    assert np.array_equal(vis, _oracle([blk], N, C, T, 0))
    assert np.allclose(rho, want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("device_out", [False, True])
def test_normalise_zero_denominator_flags(xe, device_out):
    """An input silent over the whole integration makes V_ii = 0: rho is 0
    and the flag is set on its row and column (auto included), nowhere
    else; every value and flag equals the oracle's."""
    N, C, T = 24, 5, 300
    silent = 7
    blks = [synth.block("sky", 40 + k, N, C, T, layout=1) for k in range(2)]
    for b in blks:
        b.reshape(T, N, C)[:, silent, :] = 0          # [t][i][c]: input 7 silent everywhere
    with xe.Correlator(N, C, T, layout=1) as cor:
        for b in blks:
            cor.push(b)
        if device_out:
            nb = N * (N + 1) // 2
            rho_d = torch.empty((C, nb, 2), dtype=torch.float64, device="cuda")
            flag_d = torch.full((C, nb), 9, dtype=torch.uint8, device="cuda")
            assert xe.corr_normalise_flags(cor._ctx, rho_d.data_ptr(), flag_d.data_ptr()) == xe.CORR_OK
            cor.sync()
            rho, zf = rho_d.cpu().numpy(), flag_d.cpu().numpy()
        else:
            rho, zf = cor.normalise(flags=True)
        vis = cor.dump()
    assert np.array_equal(vis, _oracle(blks, N, C, T, 1))
    want_rho, want_flag = oracle.normalise(vis, N)
    assert np.array_equal(zf, want_flag)
    assert np.allclose(rho, want_rho, rtol=1e-12, atol=0)
    ii, jj = np.tril_indices(N)
    touched = (ii == silent) | (jj == silent)
    assert (zf[:, touched] == 1).all() and (zf[:, ~touched] == 0).all()
    assert (rho[:, touched] == 0).all()


def test_dish_array_full_size(xe):
    """32 inputs, 256 channels, 1024 spectra, payload order: full parity."""
    N, C, T = 32, 256, 1024
    blk = synth.block("gauss", 0, N, C, T, layout=0)
    got = _run(xe, [blk], N, C, T, 0)
    assert np.array_equal(got, _oracle([blk], N, C, T, 0))


def test_cylinder_array_full_size_sampled(xe):
    """192 inputs, 1024 channels, 8192 spectra, [t][i][c] order (corner turn
    on the GPU): generated on the device; sampled channels against the
    oracle; all channels against invariants that hold at any size."""
    N, C, T = 192, 1024, 8192
    dblk = synth.block_device("sky", 2, N, C, T, layout=1, device="cuda")
    with xe.Correlator(N, C, T, layout=1) as cor:
        cor.push(dblk)
        vis = cor.dump()
    blk = dblk.cpu().numpy()
    chans = np.random.default_rng(5).choice(C, size=12, replace=False)
    chans = np.concatenate([[0, C - 1], chans])
    want = oracle.correlate(blk, N, C, T, layout=1, chans=chans)
    assert np.array_equal(vis[chans], want)
    # total power of every channel: sum_i V_ii = sum_t sum_i |x_i|^2
    x = dblk.view(T, N, C)
    hi = ((x >> 4).to(torch.int32) ^ 8) - 8
    lo = ((x & 15).to(torch.int32) ^ 8) - 8
    p = (hi * hi + lo * lo).sum(dim=(0, 1)).cpu().numpy()
    ii = np.array([i * (i + 1) // 2 + i for i in range(N)])
    assert np.array_equal(vis[:, ii, 0].sum(axis=1), p)
    assert (vis[:, ii, 1] == 0).all() and (vis[:, ii, 0] >= 0).all()


@pytest.mark.parametrize("N,C,T,layout", [(192, 256, 8192, 1), (32, 512, 4096, 0)])
def test_repeatable_and_full_coverage(xe, N, C, T, layout):
    """Races show up as run-to-run differences: five runs on the same bytes
    must agree exactly; every channel is then checked against the oracle
    through the Hermitian quadratic form w^H V w = sum_t |w^H x(t)|^2 for
    random Gaussian-integer weights w (a wrong entry changes the form)."""
    dblk = synth.block_device("sky", 7, N, C, T, layout=layout, device="cuda")
    runs = []
    for _ in range(5):
        with xe.Correlator(N, C, T, layout=layout) as cor:
            cor.push(dblk)
            runs.append(cor.dump())
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    vis = runs[0]
    rng = np.random.default_rng(9)
    w = rng.integers(-2, 3, size=(2, N)) + 1j * rng.integers(-2, 3, size=(2, N))
    want = oracle.projected_power(dblk.cpu().numpy(), N, C, T, w, layout=layout)
    # w^H V w from the lower triangle: sum_i |w_i|^2 V_ii + 2 Re sum_{i>j} conj(w_i) V_ij w_j
    ii, jj = np.tril_indices(N)
    b = ii * (ii + 1) // 2 + jj
    v = vis[:, b, 0] + 1j * vis[:, b, 1]
    coef = np.conj(w[:, ii]) * w[:, jj]                     # [nvec][B]
    diag = ii == jj
    q = (v[:, None, :] * coef[None]).real                   # [C][nvec][B]
    got = q[:, :, diag].sum(axis=2) + 2 * q[:, :, ~diag].sum(axis=2)
    assert np.array_equal(np.rint(got).astype(np.int64), want)


# ----------------------------------------------------------------------- 8-bit
def _sym8(seed, n):
    """Uniform int8 codes in the symmetric quantiser's range [-127, 127]."""
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, size=n, dtype=np.int16).astype(np.int8).view(np.uint8)


def _run8(xe, blocks, N, C, T, layout, device_input=True):
    with xe.Correlator(N, C, T, bits=8, layout=layout) as cor:
        for b in blocks:
            cor.push(torch.from_numpy(b).cuda() if device_input else b)
        return cor.dump()


SHAPES8 = [
    # (N, C, T): stacked (2N <= 64), one block, several blocks, even and odd block counts,
    # ragged 64-spectrum stages (8, 16, 32, 64, 96, 192 inputs in [t][c][i] are read in
    # payload order)
    (1, 3, 5), (2, 5, 130), (7, 4, 257), (8, 5, 99), (16, 3, 256), (17, 2, 100), (32, 2, 384),
    (33, 2, 200), (48, 2, 129), (64, 2, 256), (96, 3, 65), (100, 1, 300), (192, 1, 160),
    (192, 2, 77),
]


@pytest.mark.parametrize("N,C,T", SHAPES8)
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_eight_bit_bit_exact(xe, N, C, T, layout):
    """8-bit complex samples (re, im int8 in [-127, 127]), every layout."""
    blk = _sym8(7000 + N * 100 + C * 10 + T + layout, 2 * N * C * T)
    got = _run8(xe, [blk], N, C, T, layout)
    want = oracle.correlate(blk, N, C, T, bits=8, layout=layout)
    assert np.array_equal(got, want)


LONG8 = [
    # (N, C, T): tasks of several 1024-spectrum accumulations, a ragged last one
    (8, 3, 2100), (16, 2, 1025), (32, 2, 3000), (40, 2, 2049), (64, 2, 1500), (192, 1, 2500),
]


@pytest.mark.parametrize("N,C,T", LONG8)
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_eight_bit_long_tasks(xe, N, C, T, layout):
    """8-bit tasks longer than one 1024-spectrum accumulation: the pieces are
    added as integers in the CTA's scratch before the last goes out."""
    blk = _sym8(8000 + N * 10 + T + layout, 2 * N * C * T)
    got = _run8(xe, [blk], N, C, T, layout)
    assert np.array_equal(got, oracle.correlate(blk, N, C, T, bits=8, layout=layout))


def test_eight_bit_full_scale_accumulations(xe):
    """Full-scale codes at the limit of one FP32 accumulation (127^2 x 1024
    spectra, just below 2^24) and a block that ends one spectrum later, in
    both the payload order and the turned layout."""
    for N, C, T, layout in [(32, 2, 1024, 0), (32, 2, 1025, 0), (64, 1, 1088, 1)]:
        a = np.full(2 * N * C * T, 127, np.int8).view(np.uint8)
        a[1::7] = np.uint8(0x81)  # -127 mixed in
        got = _run8(xe, [a], N, C, T, layout)
        assert np.array_equal(got, oracle.correlate(a, N, C, T, bits=8, layout=layout)), (N, T)


def test_eight_bit_extremes_and_chunking(xe):
    """Full-scale codes over more than one 32768-spectrum accumulation, and
    host-pointer pushes integrated across blocks."""
    N, C, T = 8, 2, 40000
    a = np.full(2 * N * C * T, 127, np.int8).view(np.uint8)
    b = np.full(2 * N * C * T, -127, np.int8).view(np.uint8)
    c = a.copy()
    c[1::3] = np.uint8(0x81)  # -127 mixed in
    got = _run8(xe, [a, b, c], N, C, T, 0, device_input=False)
    want = None
    for blk in (a, b, c):
        want = oracle.correlate(blk, N, C, T, bits=8, layout=0, out=want)
    assert np.array_equal(got, want)


def test_eight_bit_minus_128_reported(xe):
    """-128 is outside the symmetric quantiser: the dump reports CORR_ERANGE,
    and the sums (exact for -128 too) still match the oracle."""
    N, C, T = 40, 3, 256
    blk = _sym8(99, 2 * N * C * T)
    blk[12345] = 0x80
    with xe.Correlator(N, C, T, bits=8, layout=1) as cor:
        cor.push(torch.from_numpy(blk).cuda())
        vis = cor.dump(check=False)
        assert cor.last_status == xe.CORR_ERANGE
        cor.push(torch.from_numpy(_sym8(98, blk.size)).cuda())
        cor.dump()  # the flag was cleared by the previous dump
    want = oracle.correlate(blk, N, C, T, bits=8, layout=1, check_range=False)
    assert np.array_equal(vis, want)


def test_eight_bit_512_inputs(xe):
    """512 inputs (1024 rows of the real Gram, 8 row blocks), full parity."""
    N, C, T = 512, 2, 1024
    blk = _sym8(512, 2 * N * C * T)
    got = _run8(xe, [blk], N, C, T, 0)
    assert np.array_equal(got, oracle.correlate(blk, N, C, T, bits=8, layout=0))


def test_checkpoint_restore_resume(xe):
    """Snapshot (dump without reset) + restore into a fresh context + the
    remaining blocks equals the uninterrupted integration, bit for bit."""
    N, C, T = 48, 6, 512
    blks = [synth.random_bytes(500 + s, N * C * T) for s in range(4)]
    with xe.Correlator(N, C, T, layout=1) as cor:
        for b in blks:
            cor.push(b)
        whole = cor.dump()
    with xe.Correlator(N, C, T, layout=1) as cor:
        cor.push(blks[0], seq=7)
        cor.push(blks[1], seq=8)
        snap = cor.dump(reset=False)
    with xe.Correlator(N, C, T, layout=1) as cor:
        cor.restore(torch.from_numpy(snap).cuda())
        cor.push(blks[2], seq=9)            # the sequence restarts after a restore
        cor.push(blks[3], seq=10)
        resumed = cor.dump()
    assert np.array_equal(resumed, whole)
    assert np.array_equal(whole, _oracle(blks, N, C, T, 1))


def test_dump_leaves_neighbouring_memory_alone(xe):
    """Canaries on both sides of the output: a dump writes exactly the
    visibilities, nothing before or after them."""
    N, C, T = 40, 5, 256
    nb = N * (N + 1) // 2
    guard = 4096
    buf = torch.full((2 * guard + C * nb * 2,), 0x5A5A5A5A5A5A5A5A, dtype=torch.int64, device="cuda")
    blk = synth.random_bytes(77, N * C * T)
    with xe.Correlator(N, C, T, layout=0) as cor:
        cor.push(blk)
        cor.dump_into(buf[guard:guard + C * nb * 2])
    h = buf.cpu().numpy()
    assert (h[:guard] == 0x5A5A5A5A5A5A5A5A).all() and (h[-guard:] == 0x5A5A5A5A5A5A5A5A).all()
    assert np.array_equal(h[guard:-guard].reshape(C, nb, 2), _oracle([blk], N, C, T, 0))


@pytest.mark.parametrize("bits,N,C,T", [(4, 1024, 2, 256), (8, 1024, 1, 128)])
def test_maximum_input_count(xe, bits, N, C, T):
    """1024 inputs, the largest the ABI accepts: 16 row blocks of the real
    Gram at either width, every tile kind of the schedule."""
    if bits == 4:
        blk = synth.random_bytes(1024 + bits, N * C * T)
    else:
        blk = _sym8(1024 + bits, 2 * N * C * T)
    with xe.Correlator(N, C, T, bits=bits, layout=0) as cor:
        cor.push(torch.from_numpy(blk).cuda())
        got = cor.dump()
    assert np.array_equal(got, oracle.correlate(blk, N, C, T, bits=bits, layout=0))


def test_one_full_accumulation_worst_case(xe):
    """Exactly 65536 spectra in one accumulation with the largest offset codes
    (u = 15 everywhere: 225 x 65536 < 2^24, the FP32 bound the path relies on)."""
    N, C, T = 6, 2, 65536
    blk = np.full(N * C * T, 0x77, np.uint8)  # +7 + 7i: offset code 15 in both planes
    blk[::5] = 0x88                           # and -8 - 8i (offset code 0)
    got = _run(xe, [blk], N, C, T, 2)
    assert np.array_equal(got, _oracle([blk], N, C, T, 2))
