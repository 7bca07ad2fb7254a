"""In-place integration (corr_bind): an integration bound to a caller's
device buffer must leave there exactly the oracle's sums of its blocks, a
dump into that buffer copies nothing, and integrations in the context's own
accumulators before and after it stay exact."""
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


def _want(blocks, N, C, T, layout, bits=4):
    out = None
    for b in blocks:
        out = oracle.correlate(b, N, C, T, bits=bits, layout=layout, out=out)
    return out


def _dev(N, C, fill=None):
    v = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda")
    if fill is not None:
        v.fill_(fill)   # stale contents the first push must overwrite
    return v


@pytest.mark.parametrize("N,C,T,layout,pipe", [(32, 8, 512, 1, 0), (100, 3, 300, 0, 0),
                                                (64, 16, 768, 1, 24), (192, 4, 256, 2, 0)])
def test_bound_integrations_alternate_exact(xe, N, C, T, layout, pipe):
    """Five integrations of two blocks, alternately bound to two device
    buffers holding stale values, dumped asynchronously into themselves."""
    ints = [[synth.random_bytes(300 * k + j + N, N * C * T) for j in range(2)] for k in range(5)]
    bufs = [_dev(N, C, fill=-7), _dev(N, C, fill=123)]
    with xe.Correlator(N, C, T, bits=4, layout=layout) as cor:
        if pipe:
            cor.set_pipeline(pipe)
        for k, blocks in enumerate(ints):
            buf = bufs[k % 2]
            if k >= 2:
                assert cor.dump_wait() == xe.CORR_OK  # the caller reads buf before rebinding
                assert np.array_equal(buf.cpu().numpy(), _want(ints[k - 2], N, C, T, layout))
            cor.bind(buf)
            for j, b in enumerate(blocks):
                cor.push(torch.from_numpy(b).cuda() if j else b)
            cor.dump_async(buf, reset=True)
        for _ in range(2):
            assert cor.dump_wait() == xe.CORR_OK
        cor.sync()
    for k in (3, 4):
        assert np.array_equal(bufs[k % 2].cpu().numpy(), _want(ints[k], N, C, T, layout))


def test_bound_and_own_accumulators_interleave(xe):
    """Own accumulator (overlapped copy out), bound buffer, own accumulator
    again, bound with a synchronous dump: each result exact, and the bound
    dumps copy nothing."""
    N, C, T, L = 48, 6, 512, 1
    ints = [[synth.random_bytes(500 + 10 * k + j, N * C * T) for j in range(2)] for k in range(4)]
    own0 = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, pin_memory=True)
    own2 = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, pin_memory=True)
    b1, b3 = _dev(N, C, fill=5), _dev(N, C, fill=-1)
    with xe.Correlator(N, C, T, bits=4, layout=L) as cor:
        cor.set_timing(True)
        for b in ints[0]:
            cor.push(b)
        cor.dump_async(own0, reset=True)
        cor.bind(b1)
        for b in ints[1]:
            cor.push(b)
        cor.dump_async(b1, reset=True)
        for b in ints[2]:
            cor.push(b)
        cor.dump_async(own2, reset=True)
        for _ in range(3):
            assert cor.dump_wait() == xe.CORR_OK
        copies = cor.stats()["dump_ms"]
        cor.bind(b3)
        for b in ints[3]:
            cor.push(b)
        cor.dump_into(b3, reset=True)
        assert cor.stats()["dump_ms"] == copies   # no copy was timed for the bound dump
    for got, blocks in ((own0, ints[0]), (b1, ints[1]), (own2, ints[2]), (b3, ints[3])):
        assert np.array_equal(got.cpu().numpy(), _want(blocks, N, C, T, L))


def test_bound_copy_out_without_reset_then_continue(xe):
    """A snapshot of a bound integration into another buffer (reset = 0)
    holds the first block; the bound buffer goes on to hold both."""
    N, C, T, L = 40, 5, 384, 0
    b = [synth.random_bytes(900 + j, N * C * T) for j in range(2)]
    bound, snap = _dev(N, C, fill=9), _dev(N, C)
    with xe.Correlator(N, C, T, bits=4, layout=L) as cor:
        cor.bind(bound)
        cor.push(b[0])
        cor.dump_async(snap, reset=False)
        cor.push(b[1])
        assert cor.dump_wait() == xe.CORR_OK
        cor.dump_into(bound, reset=True)
        # the next integration is back in the context's own accumulator
        cor.push(b[0])
        own = cor.dump()
    assert np.array_equal(snap.cpu().numpy(), _want(b[:1], N, C, T, L))
    assert np.array_equal(bound.cpu().numpy(), _want(b, N, C, T, L))
    assert np.array_equal(own, _want(b[:1], N, C, T, L))


def test_bound_empty_and_restore(xe):
    """A bound integration with no block dumps zeros; corr_restore while
    bound writes the bound buffer, and pushes add to it."""
    N, C, T, L = 24, 4, 256, 1
    b = synth.random_bytes(77, N * C * T)
    base = _want([synth.random_bytes(78, N * C * T)], N, C, T, L)
    z, r = _dev(N, C, fill=3), _dev(N, C, fill=4)
    with xe.Correlator(N, C, T, bits=4, layout=L) as cor:
        cor.bind(z)
        cor.dump_into(z, reset=True)
        cor.bind(r)
        cor.restore(base)
        cor.push(b)
        cor.dump_into(r, reset=True)
    assert not z.cpu().numpy().any()
    assert np.array_equal(r.cpu().numpy(), base + _want([b], N, C, T, L))


def test_bind_rejections(xe):
    N, C, T = 16, 4, 64
    with xe.Correlator(N, C, T, bits=4, layout=2) as cor:
        with pytest.raises(xe.CorrError) as e:
            cor.bind(np.zeros((C, N * (N + 1) // 2, 2), dtype=np.int64))   # host memory
        assert e.value.status == xe.CORR_EINVAL
        with pytest.raises(ValueError):
            cor.bind(torch.zeros(5, dtype=torch.int64, device="cuda"))
        cor.push(synth.random_bytes(1, N * C * T))
        with pytest.raises(xe.CorrError) as e:
            cor.bind(_dev(N, C))                        # a block is already in
        assert e.value.status == xe.CORR_ESTATE
        cor.dump(reset=True)
        again = cor.bind(_dev(N, C))
        cor.push(synth.random_bytes(2, N * C * T))
        cor.dump_into(again, reset=True)


def _blk8(seed, N, C, T):
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, 2 * N * C * T, dtype=np.int16).astype(np.int8).view(np.uint8)


@pytest.mark.parametrize("bits,N,C,T,layout", [(8, 48, 6, 512, 1), (8, 30, 4, 256, 0),
                                                (4, 12, 3, 70000, 1), (8, 12, 3, 40000, 1)])
def test_bound_eight_bit_and_multi_launch(xe, bits, N, C, T, layout):
    """8-bit samples (the byte split) and pushes longer than one exact FP32
    accumulation (several cross-multiply launches per push, the first storing
    into the bound buffer and the rest adding)."""
    gen = _blk8 if bits == 8 else (lambda s, n, c, t: synth.random_bytes(s, n * c * t))
    blocks = [gen(40 + k, N, C, T) for k in range(2)]
    buf = _dev(N, C, fill=77)
    with xe.Correlator(N, C, T, bits=bits, layout=layout) as cor:
        cor.bind(buf)
        for b in blocks:
            cor.push(b)
        cor.dump_into(buf, reset=True)
    assert np.array_equal(buf.cpu().numpy(), _want(blocks, N, C, T, layout, bits=bits))
