"""Batched arrays (corr_batch_*): one persistent cross-multiply over several
arrays of different shapes, replayed from a CUDA graph.  Every array's
visibilities must equal the oracle's exactly, on every replay, in the plain
one-launch-per-array form and under every autotuned schedule."""
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


SHAPES4 = [  # (N, C, T, bits, layout): stacked, one block, two blocks, three blocks
    (32, 64, 1024, 4, 0),
    (64, 48, 512, 4, 1),
    (20, 40, 320, 4, 2),
    (192, 6, 256, 4, 1),
    (100, 3, 384, 4, 0),
]
SHAPES8 = [(16, 8, 128, 8, 0), (48, 4, 256, 8, 1), (100, 2, 160, 8, 2)]


def _blocks(shapes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n, c, t, bits, _ in shapes:
        if bits == 4:
            out.append(rng.integers(0, 256, n * c * t, dtype=np.uint8))
        else:
            out.append(rng.integers(-127, 128, 2 * n * c * t, dtype=np.int16).astype(np.int8).view(np.uint8))
    return out


def _check(b, shapes, blocks):
    for k, ((n, c, t, bits, layout), blk) in enumerate(zip(shapes, blocks)):
        want = oracle.correlate(blk, n, c, t, bits=bits, layout=layout)
        assert np.array_equal(b.output(k), want), (k, shapes[k])


@pytest.mark.parametrize("shapes", [SHAPES4, SHAPES8], ids=["4bit", "8bit"])
def test_batch_graph_replays_and_plain_form(xe, shapes):
    with xe.Batch(shapes) as b:
        for rep in range(2):                      # the graph replays with new data
            blocks = _blocks(shapes, 100 + rep)
            for k, blk in enumerate(blocks):
                b.set_input(k, torch.from_numpy(blk).cuda() if k % 2 else blk)
            b.run()
            assert b.sync() == xe.CORR_OK
            _check(b, shapes, blocks)
        blocks = _blocks(shapes, 200)
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run_plain()
        assert b.sync() == xe.CORR_OK
        _check(b, shapes, blocks)
        info = b.info()
        assert info["launches_per_run"] == 1 + sum(1 for s in shapes if s[4] != 2 or s[3] == 8)


PAYLOAD4 = [(32, 64, 1024, 4, 0), (64, 48, 512, 4, 0), (192, 6, 256, 4, 0), (16, 20, 300, 4, 0)]
PAYLOAD8 = [(16, 8, 128, 8, 0), (32, 6, 1100, 8, 0), (64, 4, 256, 8, 0), (192, 2, 96, 8, 0)]


@pytest.mark.parametrize("shapes", [PAYLOAD4, PAYLOAD8], ids=["4bit", "8bit"])
def test_batch_read_in_payload_order(xe, shapes):
    """Every array in [t][c][i] with rows that suit TMA: no corner turns, the
    batched kernel transposes as it unpacks -- one launch per run."""
    with xe.Batch(shapes) as b:
        assert b.info()["launches_per_run"] == 1
        for rep in range(2):
            blocks = _blocks(shapes, 700 + rep)
            for k, blk in enumerate(blocks):
                b.set_input(k, blk)
            if rep == 0:
                b.run()
            else:
                b.run_plain()
            assert b.sync() == xe.CORR_OK
            _check(b, shapes, blocks)


def test_batch_autotune_every_schedule_exact(xe):
    blocks = _blocks(SHAPES4, 300)
    with xe.Batch(SHAPES4, tune=True) as b:
        info = b.info()
        assert info["schedule"] in (0, 1, 2) and all(ms > 0 for ms in info["tuned_ms"])
        assert info["tuned_ms"][info["schedule"]] == min(info["tuned_ms"])
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        assert b.sync() == xe.CORR_OK
        _check(b, SHAPES4, blocks)


def test_batch_tune_cache_reuses_schedule(xe, tmp_path, monkeypatch):
    """With XE_TUNE_CACHE set, the first tuned batch times and records its
    schedule; a later batch of the same shapes takes it from the file (the
    last matching line wins) and still correlates exactly."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("XE_TUNE_CACHE", str(cache))
    with xe.Batch(SHAPES4, tune=True) as b:
        first = b.info()
    assert first["tune_source"] == 1
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"schedule": %d' % first["schedule"] in lines[0]
    with xe.Batch(SHAPES4, tune=True) as b:
        again = b.info()
    assert again["tune_source"] == 2 and again["schedule"] == first["schedule"]
    assert np.allclose(again["tuned_ms"], first["tuned_ms"], atol=1e-6)
    forced = (first["schedule"] + 1) % 3             # a later line overrides
    cache.write_text(cache.read_text() + lines[0].replace(
        '"schedule": %d' % first["schedule"], '"schedule": %d' % forced) + "\n")
    blocks = _blocks(SHAPES4, 310)
    with xe.Batch(SHAPES4, tune=True) as b:
        assert b.info()["tune_source"] == 2 and b.info()["schedule"] == forced
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        assert b.sync() == xe.CORR_OK
        _check(b, SHAPES4, blocks)
    with xe.Batch(SHAPES4[:2], tune=True) as b:      # other shapes: timed anew
        assert b.info()["tune_source"] == 1
    assert len(cache.read_text().splitlines()) == 3
    with xe.Batch(SHAPES4) as b:                     # untuned: the default
        assert b.info()["tune_source"] == 0 and b.info()["schedule"] == 0


def test_batch_matches_single_array_contexts(xe):
    """Each array alone through corr_create/corr_push/corr_dump gives the same."""
    blocks = _blocks(SHAPES4, 400)
    with xe.Batch(SHAPES4) as b:
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        b.sync()
        for k, ((n, c, t, bits, layout), blk) in enumerate(zip(SHAPES4, blocks)):
            with xe.Correlator(n, c, t, bits=bits, layout=layout) as cor:
                cor.push(blk)
                assert np.array_equal(cor.dump(), b.output(k))


def test_batch_rejects_bad_shapes(xe):
    for shapes in ([(32, 4, 64, 4, 0), (32, 4, 64, 8, 0)],      # mixed bits
                   [(32, 4, 70000, 4, 0)],                        # longer than one accumulation
                   [(32, 4, 40, 4, 2)]):                          # unaligned rows in place
        with pytest.raises(xe.CorrError):
            xe.Batch(shapes)


def test_batch_of_many_small_arrays(xe):
    """Sixteen arrays of assorted shapes and layouts in one launch."""
    rng = np.random.default_rng(77)
    shapes = []
    for _ in range(16):
        n = int(rng.choice([3, 8, 16, 24, 40, 64, 72]))
        layout = int(rng.integers(0, 3))
        t = int(rng.choice([96, 128, 256, 320]))
        if layout == 2:
            t = t // 16 * 16
        shapes.append((n, int(rng.integers(1, 9)), t, 4, layout))
    blocks = _blocks(shapes, 900)
    with xe.Batch(shapes) as b:
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        assert b.sync() == xe.CORR_OK
        _check(b, shapes, blocks)


PIPE_CASES = [
    # split array [t][i][c] at whole 128-channel ranges, beside stacked and pre-turned arrays
    ([(192, 256, 256, 4, 1), (32, 64, 1024, 4, 0), (20, 40, 320, 4, 2)], 16, 4),
    # [t][i][c] with a ragged last range (300 channels: the byte path), alone
    ([(160, 300, 256, 4, 1)], 24, 3),
    # [t][c][i]: ranges on even channels at 64 inputs, beside a [t][i][c] array
    ([(64, 300, 256, 4, 0), (48, 8, 512, 4, 1), (100, 3, 384, 4, 0)], 32, 3),
]


@pytest.mark.parametrize("shapes,turn_sms,chunks", PIPE_CASES)
def test_batch_pipelined_exact(xe, shapes, turn_sms, chunks):
    """corr_batch_set_pipeline: the largest splittable array turned in channel
    ranges on a second stream beside the cross-multiply; every replay exact,
    and the single-launch graph restored afterwards."""
    with xe.Batch(shapes) as b:
        b.set_pipeline(turn_sms, chunks)
        assert b.info()["launches_per_run"] > 2
        for rep in range(2):
            blocks = _blocks(shapes, 300 + rep)
            for k, blk in enumerate(blocks):
                b.set_input(k, blk)
            b.run()
            assert b.sync() == xe.CORR_OK
            _check(b, shapes, blocks)
        b.set_pipeline(0)
        blocks = _blocks(shapes, 310)
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        assert b.sync() == xe.CORR_OK
        _check(b, shapes, blocks)


def test_batch_pipeline_rejections(xe):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    with xe.Batch([(32, 64, 1024, 4, 0), (20, 40, 320, 4, 2)]) as b:   # nothing to split
        with pytest.raises(xe.CorrError):
            b.set_pipeline(16, 4)
    with xe.Batch([(64, 16, 256, 4, 1)]) as b:
        for sms, ch in ((nsm, 4), (-1, 4), (8, 0)):
            with pytest.raises(xe.CorrError):
                b.set_pipeline(sms, ch)
