"""Overlapped dumps (corr_dump_async / corr_dump_wait): every queued dump
must equal the oracle's sums of exactly the blocks pushed before it, while
later pushes integrate into the other accumulator; deferred device status
belongs to the dump whose blocks raised it."""
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


def _want(blocks, N, C, T, layout, bits=4, check_range=True):
    out = None
    for b in blocks:
        out = oracle.correlate(b, N, C, T, bits=bits, layout=layout, out=out, check_range=check_range)
    return out


def _vis(N, C, pinned):
    v = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, pin_memory=pinned)
    return v


@pytest.mark.parametrize("N,C,T,layout", [(32, 8, 512, 1), (100, 3, 300, 0), (192, 4, 256, 2)])
def test_overlapped_integrations_exact(xe, N, C, T, layout):
    """Four integrations of two host blocks each, dumped asynchronously into
    pinned, pageable and device buffers, waited for only at the end."""
    ints = [[synth.random_bytes(1000 * k + j + N, N * C * T) for j in range(2)] for k in range(4)]
    outs = [_vis(N, C, True), torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64),
            torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda"),
            _vis(N, C, True)]
    with xe.Correlator(N, C, T, bits=4, layout=layout) as cor:
        for blocks, out in zip(ints, outs):
            for b in blocks:
                cor.push(b)
            cor.dump_async(out, reset=True)
        for _ in ints:
            assert cor.dump_wait() == xe.CORR_OK
        cor.sync()
    for blocks, out in zip(ints, outs):
        assert np.array_equal(out.cpu().numpy(), _want(blocks, N, C, T, layout))


def test_dump_without_reset_keeps_adding(xe):
    N, C, T = 48, 5, 384
    b = [synth.random_bytes(70 + j, N * C * T) for j in range(3)]
    v1, v2 = _vis(N, C, True), _vis(N, C, True)
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        cor.push(b[0])
        cor.push(b[1])
        cor.dump_async(v1, reset=False)
        cor.push(b[2])                     # waits for the copy, then adds
        cor.dump_async(v2, reset=True)
        cor.dump_wait()
        cor.dump_wait()
        v3 = cor.dump()                    # a fresh, empty integration
    assert np.array_equal(v1.numpy(), _want(b[:2], N, C, T, 0))
    assert np.array_equal(v2.numpy(), _want(b, N, C, T, 0))
    assert not v3.any()


def test_mixed_with_synchronous_dump_and_restore(xe):
    N, C, T = 64, 4, 256
    b = [synth.random_bytes(90 + j, N * C * T) for j in range(4)]
    v1 = _vis(N, C, True)
    with xe.Correlator(N, C, T, bits=4, layout=1) as cor:
        cor.push(b[0])
        cor.dump_async(v1, reset=True)     # integration 1 -> v1; 2 in the other buffer
        cor.push(b[1])
        ck = cor.dump(reset=False)         # synchronous copy of integration 2
        cor.push(b[2])
        cor.restore(ck)                    # back to integration 2's state
        cor.push(b[3])
        final = cor.dump()
        assert cor.dump_wait() == xe.CORR_OK
    assert np.array_equal(v1.numpy(), _want(b[:1], N, C, T, 1))
    assert np.array_equal(ck, _want(b[1:2], N, C, T, 1))
    assert np.array_equal(final, _want([b[1], b[3]], N, C, T, 1))


def test_empty_integration_and_limits(xe):
    N, C, T = 16, 3, 128
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        with pytest.raises(xe.CorrError) as e:
            cor.dump_wait()                # nothing queued
        assert e.value.status == xe.CORR_ESTATE
        outs = [_vis(N, C, True) for _ in range(xe.CORR_MAX_ASYNC_DUMPS + 1)]
        for o in outs[:-1]:
            o.fill_(7)
            cor.dump_async(o)              # nothing pushed: all zero
        with pytest.raises(xe.CorrError) as e:
            cor.dump_async(outs[-1])
        assert e.value.status == xe.CORR_EBUSY
        for o in outs[:-1]:
            cor.dump_wait()
            assert not o.any()
        blk = synth.random_bytes(5, N * C * T)
        cor.push(blk)
        cor.dump_async(outs[-1])           # a slot is free again
        cor.dump_wait()
    assert np.array_equal(outs[-1].numpy(), _want([blk], N, C, T, 0))


def _sym8(seed, n):
    rng = np.random.default_rng(seed)
    return rng.integers(-127, 128, n, dtype=np.int16).astype(np.int8).view(np.uint8)


def test_status_belongs_to_its_dump(xe):
    """-128 in integration 2 of 3: only that dump's wait reports CORR_ERANGE."""
    N, C, T = 40, 3, 256
    blks = [_sym8(200 + k, 2 * N * C * T) for k in range(3)]
    blks[1][4321] = 0x80
    outs = [_vis(N, C, True) for _ in range(3)]
    with xe.Correlator(N, C, T, bits=8, layout=1) as cor:
        for blk, out in zip(blks, outs):
            cor.push(torch.from_numpy(blk).cuda())
            cor.dump_async(out)
        got = [cor.dump_wait(check=False) for _ in blks]
        cor.sync()
    assert got == [xe.CORR_OK, xe.CORR_ERANGE, xe.CORR_OK]
    for blk, out in zip(blks, outs):
        assert np.array_equal(out.numpy(), _want([blk], N, C, T, 1, bits=8, check_range=False))
