"""Pipelined corner turn (corr_set_pipeline): the turn of block k+1 on a few
SMs overlaps the cross-multiply of block k on the others.  Visibilities
must stay bit-exact with the oracle whatever the stream interleaving, and
the caller's stream must be free to overwrite a pushed block once its turn
is done."""
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


def _blk(seed, N, C, T, bits):
    if bits == 4:
        return synth.random_bytes(seed, N * C * T)
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, 2 * N * C * T, dtype=np.int16).astype(np.int8).view(np.uint8)


def _want(blocks, N, C, T, bits, layout, chans=None):
    out = None
    for b in blocks:
        out = oracle.correlate(b, N, C, T, bits=bits, layout=layout, chans=chans, out=out)
    return out


@pytest.mark.parametrize("N,C,T,bits,layout,sms", [
    # byte-path tiles (rows not 32-byte multiples)
    (48, 20, 512, 4, 1, 24), (100, 6, 384, 4, 0, 40), (16, 40, 256, 4, 1, 8),
    (48, 10, 256, 8, 1, 32), (30, 12, 320, 8, 0, 16), (192, 4, 256, 4, 1, 100),
    # full tiles through the prefetching path, with edge tiles beside them
    (64, 128, 768, 4, 1, 40), (32, 16, 512, 4, 0, 48), (32, 64, 512, 8, 1, 32),
    (24, 200, 1280, 4, 1, 20)])
def test_pipelined_pushes_exact(xe, N, C, T, bits, layout, sms):
    blocks = [_blk(700 + k + N, N, C, T, bits) for k in range(5)]
    with xe.Correlator(N, C, T, bits=bits, layout=layout) as cor:
        cor.set_pipeline(sms)
        for k, b in enumerate(blocks):
            cor.push(torch.from_numpy(b).cuda() if k % 2 else b)   # device and host blocks
        got = cor.dump()
    assert np.array_equal(got, _want(blocks, N, C, T, bits, layout))


@pytest.mark.parametrize("bits", [4, 8])
def test_pipelined_blocks_longer_than_one_accumulation(xe, bits):
    """T above the FP32-exact accumulation length: each push issues several
    cross-multiply launches on the pipelined stream, all into one integration."""
    N, C = 12, 3
    T = 70000 if bits == 4 else 40000
    blocks = [_blk(950 + k + bits, N, C, T, bits) for k in range(2)]
    with xe.Correlator(N, C, T, bits=bits, layout=1) as cor:
        cor.set_pipeline(20)
        for b in blocks:
            cor.push(b)
        got = cor.dump()
    assert np.array_equal(got, _want(blocks, N, C, T, bits, 1))


def test_caller_stream_may_overwrite_after_push(xe):
    """One device buffer reused for every block: the next block is written
    into it on the context's stream right after corr_push returns."""
    N, C, T = 64, 16, 1024
    blocks = [_blk(800 + k, N, C, T, 4) for k in range(6)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        buf = torch.empty(N * C * T, dtype=torch.uint8, device="cuda")
        staged = [torch.from_numpy(b).cuda() for b in blocks]
    s.synchronize()
    with xe.Correlator(N, C, T, bits=4, layout=1, stream=s.cuda_stream) as cor:
        cor.set_pipeline(48)
        with torch.cuda.stream(s):
            for b in staged:
                buf.copy_(b, non_blocking=True)   # ordered after the previous block's turn
                cor.push(buf)
        got = cor.dump()
    assert np.array_equal(got, _want(blocks, N, C, T, 4, 1))


def test_overlapped_dumps_and_toggling(xe):
    N, C, T = 40, 24, 512
    blocks = [_blk(900 + k, N, C, T, 4) for k in range(6)]
    outs = [torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, pin_memory=True) for _ in range(3)]
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        cor.set_pipeline(32)
        cor.push(blocks[0])
        cor.push(blocks[1])
        cor.dump_async(outs[0])
        cor.push(blocks[2])
        cor.set_pipeline(0)                   # back to one stream mid-integration
        cor.push(blocks[3])
        cor.dump_async(outs[1])
        cor.set_pipeline(64)
        cor.push(blocks[4])
        cor.push(blocks[5])
        cor.dump_async(outs[2])
        for _ in outs:
            assert cor.dump_wait() == xe.CORR_OK
    assert np.array_equal(outs[0].numpy(), _want(blocks[:2], N, C, T, 4, 0))
    assert np.array_equal(outs[1].numpy(), _want(blocks[2:4], N, C, T, 4, 0))
    assert np.array_equal(outs[2].numpy(), _want(blocks[4:], N, C, T, 4, 0))


def test_rejected_configurations(xe):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    with xe.Correlator(16, 4, 64, bits=4, layout=2) as cor:     # no corner turn to overlap
        with pytest.raises(xe.CorrError):
            cor.set_pipeline(8)
    with xe.Correlator(16, 4, 64, bits=4, layout=1) as cor:
        for bad in (nsm, -1):
            with pytest.raises(xe.CorrError):
                cor.set_pipeline(bad)
        cor.set_pipeline(0)


def test_cylinder_slice_pipelined(xe):
    """192 inputs x 128 channels x 8192 spectra, three blocks in the
    bench's configuration (48 turn SMs), 12 sampled channels."""
    N, C, T = 192, 128, 8192
    dev = torch.device("cuda")
    blocks = [synth.block_device("sky", 40 + k, N, C, T, 1, dev) for k in range(3)]
    with xe.Correlator(N, C, T, bits=4, layout=1) as cor:
        cor.set_pipeline(48)
        for b in blocks:
            cor.push(b)
        got = cor.dump()
    chans = list(range(0, C, 11))
    want = _want([b.cpu().numpy() for b in blocks], N, C, T, 4, 1, chans=chans)
    assert np.array_equal(got[chans], want)


def test_cylinder_full_size_bench_configuration(xe):
    """192 inputs x 1024 channels x 8192 spectra in the launch configuration
    the benchmark times: corner turn on 42 SMs beside the cross-multiply, two
    device blocks cycled, each integration bound to its own device buffer and
    dumped asynchronously.  Every channel of every integration against the
    oracle, element by element, and against the total-power invariant."""
    N, C, T = 192, 1024, 8192
    nb = N * (N + 1) // 2
    blocks = [synth.block_device("sky", 60 + k, N, C, T, 1, torch.device("cuda")) for k in range(2)]
    outs = [torch.empty((C, nb, 2), dtype=torch.int64, device="cuda") for _ in range(2)]
    order = [0, 1, 0]                        # integration k holds block order[k]
    kept = []
    with xe.Correlator(N, C, T, bits=4, layout=1) as cor:
        cor.set_pipeline(42)
        for k, b in enumerate(order):
            out = outs[k % 2]
            if k >= 2:
                assert cor.dump_wait() == xe.CORR_OK
                kept.append(outs[(k - 2) % 2].cpu().numpy())   # read before rebinding
            cor.bind(out)
            cor.push(blocks[b])
            cor.dump_async(out, reset=True)
        while len(kept) < len(order):
            assert cor.dump_wait() == xe.CORR_OK
            kept.append(outs[len(kept) % 2].cpu().numpy())
    ii = np.array([i * (i + 1) // 2 + i for i in range(N)])
    want = {}
    for k, b in enumerate(order):
        if b not in want:
            want[b] = oracle.correlate(blocks[b].cpu().numpy(), N, C, T, layout=1)
        assert np.array_equal(kept[k], want[b]), k
        x = blocks[b].view(T, N, C)
        hi = ((x >> 4).to(torch.int32) ^ 8) - 8
        lo = ((x & 15).to(torch.int32) ^ 8) - 8
        p = (hi * hi + lo * lo).sum(dim=(0, 1)).cpu().numpy()
        assert np.array_equal(kept[k][:, ii, 0].sum(axis=1), p)
