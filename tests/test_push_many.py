"""corr_push_many: several blocks of one array integrated by one persistent
cross-multiply launch, against the oracle's sum over the blocks (the
integration over time of Sec. 2.2), through the C ABI.

The single-launch form runs every block's tasks together and adds each
block's partial sums with reductions at L2 into an accumulator that a new
integration zeroes; the tests check it on every layout and bit width that
the cross-multiply reads in place, with ragged time, stacked and unstacked
tiles, 8-bit blocks longer than one FP32 accumulation, many small blocks,
and integrations that mix it with corr_push.  Blocks that need a corner
turn, host blocks and the pipelined mode push one block at a time: those
fallbacks must give the same sums.  Integer results are bit-exact.
"""
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


def _sym8(seed, n):
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, size=n, dtype=np.int16).astype(np.int8).view(np.uint8)


def _blocks(bits, n_blk, N, C, T, seed):
    if bits == 4:
        return [synth.random_bytes(seed + k, N * C * T) for k in range(n_blk)]
    return [_sym8(seed + k, 2 * N * C * T) for k in range(n_blk)]


def _want(blocks, N, C, T, bits, layout):
    out = None
    for b in blocks:
        out = oracle.correlate(b, N, C, T, bits=bits, layout=layout, out=out)
    return out


def _many(xe, blocks, N, C, T, bits, layout, device=True):
    with xe.Correlator(N, C, T, bits=bits, layout=layout) as cor:
        s0 = cor.stats()
        cor.push_many([torch.from_numpy(b).cuda() if device else b for b in blocks])
        got = cor.dump()
        s1 = cor.stats()
    return got, s1["herk_launches"] - s0["herk_launches"], s1["blocks"] - s0["blocks"]


ONE_LAUNCH = [
    # (bits, layout, N, C, T, blocks): payload order read in place (stacked 16/32-input
    # tiles, whole 64-row boxes), the 4-bit turned layout, ragged stages
    (4, 0, 32, 64, 1024, 5), (4, 0, 16, 40, 300, 3), (4, 0, 64, 16, 1000, 4),
    (4, 0, 192, 4, 256, 3), (4, 2, 48, 8, 512, 3), (4, 2, 192, 6, 272, 2),
    (8, 0, 32, 16, 2100, 3), (8, 0, 8, 20, 640, 4), (8, 0, 192, 2, 1100, 2), (8, 0, 64, 6, 1500, 2),
    # large arrays: paired and single column-block tasks of many row blocks in one launch
    (4, 0, 384, 3, 512, 2), (8, 0, 512, 2, 300, 2),
]


@pytest.mark.parametrize("bits,layout,N,C,T,nblk", ONE_LAUNCH)
def test_one_launch_bit_exact(xe, bits, layout, N, C, T, nblk):
    blks = _blocks(bits, nblk, N, C, T, 100 * N + C + T + bits + layout)
    got, launches, blocks = _many(xe, blks, N, C, T, bits, layout)
    assert launches == 1 and blocks == nblk
    assert np.array_equal(got, _want(blks, N, C, T, bits, layout))


@pytest.mark.parametrize("bits,N,C,T", [(4, 16, 2, 70000), (8, 8, 2, 33000)])
def test_blocks_longer_than_one_accumulation(xe, bits, N, C, T):
    """Blocks longer than one exact FP32 accumulation (65536 spectra at 4
    bits, 32768 at 8): each block is two instances with their own time
    ranges, all in one launch."""
    blks = _blocks(bits, 2, N, C, T, 950 + bits)
    got, launches, blocks = _many(xe, blks, N, C, T, bits, 0)
    assert launches == 1 and blocks == 2
    assert np.array_equal(got, _want(blks, N, C, T, bits, 0))


def test_many_small_blocks(xe):
    """Forty 32-input blocks: one launch of 1280 tasks over the SMs (the
    context's task list grows to forty blocks)."""
    N, C, T, nblk = 32, 64, 128, 40
    blks = _blocks(4, nblk, N, C, T, 900)
    got, launches, _ = _many(xe, blks, N, C, T, 4, 0)
    assert launches == 1
    assert np.array_equal(got, _want(blks, N, C, T, 4, 0))


@pytest.mark.parametrize("bits,layout,N,C,T", [(4, 1, 32, 16, 256), (4, 0, 24, 8, 128),
                                               (8, 1, 16, 8, 200), (8, 2, 96, 4, 1040)])
def test_turned_blocks_push_one_by_one(xe, bits, layout, N, C, T):
    """Blocks that need a corner turn ([t][i][c], a payload order whose rows
    do not suit TMA, or 8-bit [c][i][t], whose (re, im) byte pairs are split
    into rows) are pushed one by one: one launch per block."""
    blks = _blocks(bits, 3, N, C, T, 300 + N + bits)
    got, launches, blocks = _many(xe, blks, N, C, T, bits, layout)
    assert launches == 3 and blocks == 3
    assert np.array_equal(got, _want(blks, N, C, T, bits, layout))


def test_host_blocks_push_one_by_one(xe):
    N, C, T = 32, 16, 512
    blks = _blocks(4, 3, N, C, T, 410)
    got, launches, _ = _many(xe, blks, N, C, T, 4, 0, device=False)
    assert launches == 3
    assert np.array_equal(got, _want(blks, N, C, T, 4, 0))


def test_pipelined_context_pushes_one_by_one(xe):
    N, C, T = 32, 64, 512
    blks = _blocks(4, 3, N, C, T, 420)
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        cor.set_pipeline(16)
        cor.push_many([torch.from_numpy(b).cuda() for b in blks])
        got = cor.dump()
    assert np.array_equal(got, _want(blks, N, C, T, 4, 0))


def test_mixed_with_push_and_reset(xe):
    """push, push_many, push in one integration; then, after a reset, a
    push_many that starts the next integration from zero (the old sums are
    gone); then the same blocks again, so that the table is reused."""
    N, C, T = 32, 32, 256
    a, b, c, d, e = _blocks(4, 5, N, C, T, 500)
    dev = [torch.from_numpy(x).cuda() for x in (a, b, c, d, e)]
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        cor.push(dev[0])
        cor.push_many([dev[1], dev[2]])
        cor.push(dev[3])
        first = cor.dump(reset=True)
        cor.push_many([dev[4], dev[1]])
        second = cor.dump(reset=True)
        s0 = cor.stats()
        cor.push_many([dev[4], dev[1]])
        third = cor.dump(reset=True)
        s1 = cor.stats()
    assert np.array_equal(first, _want([a, b, c, d], N, C, T, 4, 0))
    assert np.array_equal(second, _want([e, b], N, C, T, 4, 0))
    assert np.array_equal(third, second)
    assert s1["herk_launches"] - s0["herk_launches"] == 1


def test_tables_alternate(xe):
    """Three different block lists in turn (two tables, refilled in turn)
    inside one integration."""
    N, C, T = 16, 48, 200
    blks = _blocks(4, 6, N, C, T, 600)
    dev = [torch.from_numpy(x).cuda() for x in blks]
    lists = [[0, 1], [2, 3, 4], [5, 0], [2, 3, 4], [1, 5]]
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        for li in lists:
            cor.push_many([dev[i] for i in li])
        got = cor.dump()
    assert np.array_equal(got, _want([blks[i] for li in lists for i in li], N, C, T, 4, 0))


def test_bound_buffers_alternate(xe):
    """Integrations bound to two device buffers in turn with overlapped dumps
    (the streaming benchmark's form)."""
    N, C, T = 32, 64, 512
    nb = N * (N + 1) // 2
    blks = _blocks(4, 4, N, C, T, 700)
    dev = [torch.from_numpy(x).cuda() for x in blks]
    outs = [torch.empty((C, nb, 2), dtype=torch.int64, device="cuda") for _ in range(2)]
    got = []
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        for k in range(4):
            cor.bind(outs[k % 2])
            cor.push_many([dev[(k + p) % 4] for p in range(3)])
            cor.dump_async(outs[k % 2], reset=True)
            assert cor.dump_wait() == xe.CORR_OK
            got.append(outs[k % 2].cpu().numpy())
    for k in range(4):
        assert np.array_equal(got[k], _want([blks[(k + p) % 4] for p in range(3)], N, C, T, 4, 0)), k


def test_sequence_numbers(xe):
    N, C, T = 16, 16, 128
    blks = _blocks(4, 5, N, C, T, 800)
    dev = [torch.from_numpy(x).cuda() for x in blks]
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        assert cor.push_many(dev[:3], seq=10) == xe.CORR_OK
        assert cor.push_many(dev[3:5], seq=14, check=False) == xe.CORR_ESEQ  # gap: nothing integrated
        assert cor.push(dev[3], seq=13) == xe.CORR_OK
        assert cor.push_many([dev[4]], seq=14) == xe.CORR_OK
        got = cor.dump()
    assert np.array_equal(got, _want(blks, N, C, T, 4, 0))


def test_bad_arguments(xe):
    N, C, T = 16, 8, 64
    blk = torch.from_numpy(_blocks(4, 1, N, C, T, 1)[0]).cuda()
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        with pytest.raises(ValueError):
            cor.push_many([])
        with pytest.raises(ValueError):
            cor.push_many([blk, blk[:-1]])
        import ctypes
        arr = (ctypes.c_void_p * 1)(blk.data_ptr())
        assert xe._lib.corr_push_many(cor._ctx, arr, 1, blk.numel() - 1, xe.CORR_SEQ_ANY) == xe.CORR_EINVAL
        assert xe._lib.corr_push_many(cor._ctx, arr, 0, blk.numel(), xe.CORR_SEQ_ANY) == xe.CORR_EINVAL
        assert xe._lib.corr_push_many(cor._ctx, arr, xe.CORR_MAX_PUSH_MANY + 1, blk.numel(),
                                      xe.CORR_SEQ_ANY) == xe.CORR_EINVAL


def test_dish_stream_full_size(xe):
    """The streaming dish workload as the benchmark runs it: 32 blocks of
    32 inputs x 1024 channels x 4096 spectra per dump in one push_many,
    bound to a device buffer, overlapped dump; every channel against the
    oracle."""
    N, C, T, nblk = 32, 1024, 4096, 32
    nb = N * (N + 1) // 2
    dev = torch.device("cuda")
    blocks = [synth.block_device("sky", 200 + k, N, C, T, 0, dev) for k in range(4)]
    out = torch.empty((C, nb, 2), dtype=torch.int64, device=dev)
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        s0 = cor.stats()
        cor.bind(out)
        cor.push_many([blocks[p % 4] for p in range(nblk)])
        cor.dump_async(out, reset=True)
        assert cor.dump_wait() == xe.CORR_OK
        s1 = cor.stats()
    assert s1["herk_launches"] - s0["herk_launches"] == 1
    want = None
    for k in range(4):
        want = oracle.correlate(blocks[k].cpu().numpy(), N, C, T, layout=0, out=want)
    assert np.array_equal(out.cpu().numpy(), want * (nblk // 4))
