"""Host logic of the streaming service (corr_svc_*) in dry-run mode: the same
admission, queueing, slot, push and tick bookkeeping as on the GPU, with no
device memory and no kernels.  No GPU is needed."""
import numpy as np
import pytest

from paper_1904_07778_gb300 import build

build.build()
from paper_1904_07778_gb300 import xengine as xe  # noqa: E402

R4 = dict(n_inputs=32, n_chans=64, bits=4, layout=0, block_spectra=1024)


def _bytes(n, c, bits, layout, t):
    """Device state of one request: int64 accumulator, two ingest buffers, the
    corner-turn buffer (rows padded to 32 bytes), each rounded to 256 bytes.
    No turn buffer for [c][i][t] 4-bit blocks, nor for [t][c][i] blocks read in
    payload order (byte rows per channel 16, 32 or a multiple of 16 from 64 at 4 bits; 16, 32, 64
    or a multiple of 16 from 128 at 8 bits)."""
    r = lambda x: (x + 255) // 256 * 256
    rows = n * bits // 4
    acc = n * (n + 1) // 2 * c * 16
    blk = rows * c * t
    box = 128 if bits == 8 else 64                                     # byte rows of a 128-row block
    stacked = (16, 32, 64) if bits == 8 else (16, 32)
    direct = layout == 0 and rows % 16 == 0 and (rows in stacked or rows >= box)
    turn = 0 if (layout == 2 and bits == 4) or direct else rows * c * ((t + 31) // 32 * 32)
    return r(acc) + 2 * r(blk) + r(turn)


def _blk(n, c, bits, t):
    return np.zeros(n * c * t * bits // 4, dtype=np.uint8)


def test_fifo_admission_by_budget():
    size = _bytes(32, 64, 4, 0, 1024)
    with xe.Service(int(2.5 * size), dry_run=True) as s:
        ids = [s.submit(**R4, n_blocks=2) for _ in range(3)]
        assert [s.state(i) for i in ids] == [xe.CORR_REQ_ACTIVE, xe.CORR_REQ_ACTIVE, xe.CORR_REQ_QUEUED]
        st = s.stats()
        assert st["active"] == 2 and st["queued"] == 1 and st["in_use"] == 2 * size
        assert s.push(ids[2], _blk(32, 64, 4, 1024), check=False) == xe.CORR_ESTATE
        for _ in range(2):
            s.push(ids[0], _blk(32, 64, 4, 1024))
            assert s.tick() == 1
        assert s.state(ids[0]) == xe.CORR_REQ_DONE
        assert s.state(ids[2]) == xe.CORR_REQ_QUEUED   # admitted only when memory is released
        s.fetch(ids[0])
        assert s.state(ids[0]) == xe.CORR_REQ_FETCHED
        assert s.state(ids[2]) == xe.CORR_REQ_ACTIVE


def test_push_rules_and_tick_composition():
    with xe.Service(1 << 30, dry_run=True) as s:
        a = s.submit(**R4, n_blocks=3)
        b = s.submit(**R4, n_blocks=1)
        blk = _blk(32, 64, 4, 1024)
        assert s.push(a, blk[:-1], check=False) == xe.CORR_EINVAL      # wrong size
        s.push(a, blk)
        s.push(a, blk)
        assert s.push(a, blk, check=False) == xe.CORR_EBUSY            # two blocks already waiting
        assert s.tick() == 1                                            # b has nothing pushed yet
        s.push(b, blk)
        assert s.tick() == 2
        assert s.state(b) == xe.CORR_REQ_DONE
        assert s.fetch(a, check=False) == xe.CORR_ESTATE                # not done yet
        s.push(a, blk)
        assert s.push(a, blk, check=False) == xe.CORR_ESTATE            # all its blocks pushed
        assert s.tick() == 1 and s.tick() == 0
        assert s.state(a) == xe.CORR_REQ_DONE
        st = s.stats()
        assert st["blocks"] == 4 and st["ticks"] == 3 and st["completed"] == 2
        assert st["ops"] == 4 * 8 * 528 * 64 * 1024
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_rejects():
    with xe.Service(1 << 20, dry_run=True) as s:
        assert s.submit(**R4, n_blocks=1, check=False) == xe.CORR_EBUSY    # never fits 1 MiB
        bad = dict(R4, bits=5)
        assert s.submit(**bad, n_blocks=1, check=False) == xe.CORR_EINVAL
        bad = dict(R4, block_spectra=70000)
        assert s.submit(**bad, n_blocks=1, check=False) == xe.CORR_EINVAL
        bad = dict(R4, layout=2, block_spectra=1000)                       # unaligned rows in place
        assert s.submit(**bad, n_blocks=1, check=False) == xe.CORR_EINVAL
        with pytest.raises(xe.CorrError):
            s.state(12345)


def test_arena_churn_returns_to_empty():
    """Random sizes submitted and fetched in random order: every request is
    admitted eventually (FIFO), memory never exceeds the budget and returns
    to zero with free ranges coalesced (a full-budget request fits at the end)."""
    rng = np.random.default_rng(5)
    shapes = [(int(rng.choice([4, 16, 48, 100])), int(rng.choice([8, 32, 64])), int(rng.choice([4, 8])),
               int(rng.integers(0, 3)), 256) for _ in range(60)]
    sizes = [_bytes(n, c, b, l, t) for n, c, b, l, t in shapes]
    budget = 3 * max(sizes)
    with xe.Service(budget, dry_run=True) as s:
        ids = [s.submit(n, c, b, l, t, 1) for n, c, b, l, t in shapes]
        pending = list(ids)
        while pending:
            active = [i for i in pending if s.state(i) == xe.CORR_REQ_ACTIVE]
            assert active, "FIFO admission stalled"
            for i in rng.permutation(active):
                n, c, b, l, t = shapes[ids.index(i)]
                s.push(int(i), _blk(n, c, b, t))
            s.tick()
            for i in rng.permutation(active):
                s.fetch(int(i))
                pending.remove(int(i))
            assert s.stats()["in_use"] <= budget
        st = s.stats()
        assert st["in_use"] == 0 and st["peak_in_use"] <= budget and st["fetched"] == 60
        # coalesced: a request larger than two of the largest ones fits again
        big = next((n, c, b, l, t) for t in (256, 512, 1024, 2048) for n in range(8, 200, 4)
                   for c in (8, 16, 32, 64) for b in (4, 8) for l in (0,)
                   if 2 * max(sizes) < _bytes(n, c, b, l, t) <= budget)
        rid = s.submit(*big, 1)
        assert s.state(rid) == xe.CORR_REQ_ACTIVE
