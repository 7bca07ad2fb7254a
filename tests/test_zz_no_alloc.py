"""The allocation-free entry point, corr_correlate_noalloc.

It exists for callers that cannot allocate device memory (an allocator owned
by another framework, allocation frozen after start-up, real-time loops).  It
keeps its intermediates in a fixed scratch array inside the library, shared by
every call.  This test calls it through the C ABI several times in a row, with
different shapes, and checks each result against the context path
(corr_create / corr_push / corr_dump) and against the oracle on the same
bytes: the visibilities are integers, so they must agree exactly.  The file
name sorts last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


@pytest.fixture(scope="module")
def xe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_07778_gb300 import build
    build.build()
    from paper_1904_07778_gb300 import xengine
    return xengine


def _reference(xe, blk, N, C, T, layout, bits=4):
    with xe.Correlator(N, C, T, bits=bits, layout=layout) as cor:
        cor.push(blk)
        return cor.dump()


def _noalloc(xe, blk, N, C, T, layout, bits=4, want_status=0):
    nb = N * (N + 1) // 2
    vis = torch.full((C, nb, 2), -1, dtype=torch.int64, device="cuda")  # stale values must vanish
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream or 1  # 1 = the legacy default stream
    if bits == 4:
        rc = xe.corr_correlate_noalloc(blk.data_ptr(), N, C, T, layout, 0, vis.data_ptr(),
                                       status.data_ptr(), stream)
    else:
        rc = xe.corr_correlate_noalloc_bits(blk.data_ptr(), N, C, T, bits, layout, 0, vis.data_ptr(),
                                            status.data_ptr(), stream)
    assert rc == xe.CORR_OK, xe.corr_strerror(rc)
    torch.cuda.synchronize()
    assert int(status.item()) == want_status
    return vis.cpu().numpy()


def _sym8(seed, n):
    """Uniform int8 codes in the symmetric quantiser's range [-127, 127]."""
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, size=n, dtype=np.int16).astype(np.int8).view(np.uint8)


def test_noalloc_matches_context_path_on_consecutive_calls(xe):
    rng = np.random.default_rng(2024)
    cases = [
        (64, 16, 1024, xe.CORR_L_TIC),   # corner turn through the scratch
        (32, 64, 512, xe.CORR_L_TCI),    # stacked small array
        (100, 5, 300, xe.CORR_L_CIT),    # ragged tail, no corner turn
        (130, 4, 1024, xe.CORR_L_TIC),   # three row blocks: paired tasks on the TMA ring kernel
        (4, 1, 70000, xe.CORR_L_CIT),    # longer than one accumulation, unaligned rows
        (64, 16, 1024, xe.CORR_L_TIC),   # first shape again, new data
    ]
    for N, C, T, layout in cases:
        host = rng.integers(0, 256, N * C * T, dtype=np.uint8)
        blk = torch.from_numpy(host).cuda()
        got = _noalloc(xe, blk, N, C, T, layout)
        assert np.array_equal(got, _reference(xe, blk, N, C, T, layout)), (N, C, T, layout)
        assert np.array_equal(got, oracle.correlate(host, N, C, T, layout=layout)), (N, C, T, layout)


def test_noalloc_eight_bit_matches_oracle(xe):
    """8-bit blocks (corr_correlate_noalloc_bits) in every layout: payload
    order read in place (its partial sums in the scratch), payload order and
    [t][i][c] turned through the scratch, [c][i][t] split into planes, and a
    block longer than one 32768-spectrum accumulation."""
    cases = [
        (32, 8, 2100, xe.CORR_L_TCI),    # 64 byte rows, read in place; 1024-spectrum pieces
        (24, 6, 300, xe.CORR_L_TCI),     # 48 byte rows: turned
        (16, 8, 300, xe.CORR_L_TIC),
        (40, 4, 1024, xe.CORR_L_CIT),
        (8, 2, 33000, xe.CORR_L_TCI),    # two accumulations
        (192, 2, 160, xe.CORR_L_TCI),    # 384 byte rows, read in place
    ]
    for k, (N, C, T, layout) in enumerate(cases):
        host = _sym8(8800 + k, 2 * N * C * T)
        blk = torch.from_numpy(host).cuda()
        got = _noalloc(xe, blk, N, C, T, layout, bits=8)
        assert np.array_equal(got, oracle.correlate(host, N, C, T, bits=8, layout=layout)), (N, C, T, layout)
        assert np.array_equal(got, _reference(xe, blk, N, C, T, layout, bits=8)), (N, C, T, layout)


def test_noalloc_eight_bit_reports_minus_128(xe):
    """A -128 byte is integrated exactly and reported in the status word."""
    N, C, T = 16, 4, 256
    host = _sym8(8900, 2 * N * C * T)
    host[37] = 0x80
    blk = torch.from_numpy(host).cuda()
    got = _noalloc(xe, blk, N, C, T, xe.CORR_L_TCI, bits=8, want_status=2)
    assert np.array_equal(got, oracle.correlate(host, N, C, T, bits=8, layout=xe.CORR_L_TCI,
                                                check_range=False))


def test_noalloc_rejects_requests_beyond_the_scratch(xe):
    N, C, T = 192, 16, 8192  # corner-turned copy of 24 MiB > 16 MiB scratch
    assert N * C * T > xe.CORR_NOALLOC_SCRATCH_BYTES
    blk = torch.zeros(N * C * T, dtype=torch.uint8, device="cuda")
    vis = torch.zeros((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda")
    rc = xe.corr_correlate_noalloc(blk.data_ptr(), N, C, T, xe.CORR_L_TIC, 0, vis.data_ptr())
    assert rc == xe.CORR_EINVAL
    host = np.zeros(16, dtype=np.uint8)
    rc = xe.corr_correlate_noalloc(host.ctypes.data, 4, 1, 4, xe.CORR_L_CIT, 0, vis.data_ptr())
    assert rc == xe.CORR_EINVAL  # host memory is not accepted
