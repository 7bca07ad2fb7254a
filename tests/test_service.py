"""Streaming service on the GPU (corr_svc_*): requests of different arrays,
sample widths and lengths integrated by shared ticks must give exactly the
oracle's visibilities, and the same result alone as in the mix."""
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


REQS = [  # (N, C, bits, layout, block_spectra, n_blocks)
    (32, 64, 4, 0, 512, 3),
    (64, 16, 4, 1, 256, 2),
    (20, 24, 4, 2, 320, 4),
    (48, 8, 8, 0, 256, 3),
    (100, 4, 8, 1, 128, 2),
    (192, 2, 4, 1, 384, 1),
]


def _blocks(req, seed):
    n, c, bits, _, t, nb = req
    rng = np.random.default_rng(seed)
    if bits == 4:
        return [rng.integers(0, 256, n * c * t, dtype=np.uint8) for _ in range(nb)]
    return [rng.integers(-127, 128, 2 * n * c * t, dtype=np.int16).astype(np.int8).view(np.uint8)
            for _ in range(nb)]


def _want(req, blocks):
    n, c, bits, layout, t, _ = req
    out = None
    for b in blocks:
        out = oracle.correlate(b, n, c, t, bits=bits, layout=layout, out=out)
    return out


def _drive(xe, svc, reqs, data):
    """Submit everything, then push and tick until every request is done."""
    ids = [svc.submit(n, c, bits, layout, t, nb) for n, c, bits, layout, t, nb in reqs]
    nxt = [0] * len(reqs)
    results = {}
    for _ in range(1000):
        for k, rid in enumerate(ids):
            if svc.state(rid) == xe.CORR_REQ_ACTIVE and nxt[k] < len(data[k]):
                blk = data[k][nxt[k]]
                if svc.push(rid, torch.from_numpy(blk).cuda() if k % 2 else blk, check=False) == xe.CORR_OK:
                    nxt[k] += 1
        svc.tick()
        assert svc.wait() == xe.CORR_OK
        for k, rid in enumerate(ids):
            if k not in results and svc.state(rid) == xe.CORR_REQ_DONE:
                results[k] = svc.fetch(rid)
        if len(results) == len(reqs):
            return results
    raise AssertionError("service did not finish")


def test_mixed_requests_exact_and_same_alone(xe):
    data = [_blocks(r, 50 + k) for k, r in enumerate(REQS)]
    with xe.Service(8 << 30) as svc:
        mix = _drive(xe, svc, REQS, data)
        st = svc.stats()
    assert st["completed"] == len(REQS) and st["in_use"] == 0
    assert st["launches"] > st["ticks"]      # 4-bit and 8-bit requests shared ticks
    for k, r in enumerate(REQS):
        assert np.array_equal(mix[k], _want(r, data[k])), r
        with xe.Service(1 << 30) as alone:
            one = _drive(xe, alone, [r], [data[k]])
        assert np.array_equal(one[0], mix[k]), r


def test_small_budget_queues_and_still_exact(xe):
    """A budget that holds about two requests at a time: the rest wait in the
    queue and are admitted as results are fetched."""
    reqs = [(64, 32, 4, 0, 256, 2)] * 5
    data = [_blocks(r, 90 + k) for k, r in enumerate(reqs)]
    rows = 64
    per = (64 * 65 // 2 * 32 * 16) + 2 * rows * 32 * 256 + rows * 32 * 256
    with xe.Service(int(2.5 * per) + 4096) as svc:
        res = _drive(xe, svc, reqs, data)
        st = svc.stats()
    assert st["peak_in_use"] <= int(2.5 * per) + 4096
    for k, r in enumerate(reqs):
        assert np.array_equal(res[k], _want(r, data[k]))
