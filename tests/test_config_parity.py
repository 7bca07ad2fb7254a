"""Parity at the workload sizes the benchmark runs, through the C ABI.

Each test correlates one of the five synthetic Tianlai-shaped workloads at its
full size on the GPU and compares the int64 visibilities with the oracle:

* dish streaming integration: 32 inputs x 1024 channels, 32 blocks of 4096
  spectra integrated into int64 per dump (pipelined corner turn, integration
  bound to a device buffer, overlapped dump), every channel in full;
* batched mixed arrays: 32 x 256 x 1024, 64 x 1024 x 4096 and
  192 x 4096 x 16384 in one batch run: the first two in full, the third on
  64 seeded channels in full plus the Hermitian quadratic form of every
  channel;
* streaming service: 8-bit requests of 512, 192 and 32 inputs x 2048
  channels (4096 spectra each) admitted and ticked together: 16 seeded
  channels per request in full plus the quadratic form of every channel.

The cylinder workload (192 x 1024 x 8192, [t][i][c]) is checked in full in
tests/test_pipeline.py in the benchmark's launch configuration.

The quadratic form w^H V w = sum_t |w^H x(t)|^2 (w: small Gaussian-integer
vectors) covers every entry of a channel's matrix: a wrong visibility
changes it for all but a vanishing set of w.  Both sides are exact integers.
The definition being checked is the CMAC of Sec. 2 integrated over blocks
(Sec. 2, Sec. 2.2).
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


def _weights(seed, n_vec, n_inputs):
    rng = np.random.default_rng(seed)
    return rng.integers(-1, 2, size=(n_vec, n_inputs)) + 1j * rng.integers(-1, 2, size=(n_vec, n_inputs))


def _quadratic_form(vis, w):
    """w^H V w per channel from the stored lower triangle, exactly:
    sum_i |w_i|^2 V_ii + 2 Re sum_{i>j} conj(w_i) V_ij w_j, int64 [C][nvec]."""
    n = w.shape[1]
    ii, jj = np.tril_indices(n)
    coef = np.conj(w[:, ii]) * w[:, jj] * np.where(ii == jj, 1, 2)[None, :]   # [nvec][B]
    b = ii * (ii + 1) // 2 + jj
    vre = vis[:, b, 0].astype(np.float64)
    vim = vis[:, b, 1].astype(np.float64)
    # every product and partial sum is an integer below 2^53: exact in float64
    q = vre @ coef.real.T - vim @ coef.imag.T
    return np.rint(q).astype(np.int64)


def test_dish_streaming_integration_full(xe):
    """32 inputs x 1024 channels, 32 blocks of 4096 spectra per dump, one push
    per block with the corner turn pipelined (turn of block k+1 on 48 SMs
    beside the cross-multiply of block k), integration bound to its device
    buffer, the dump overlapped; every channel against the oracle.  (The
    benchmark reads these blocks in place, all 32 in one corr_push_many:
    tests/test_push_many.py checks that form at this size.)"""
    N, C, T, nblk = 32, 1024, 4096, 32
    nb = N * (N + 1) // 2
    dev = torch.device("cuda")
    out = torch.empty((C, nb, 2), dtype=torch.int64, device=dev)
    want = np.zeros((C, nb, 2), dtype=np.int64)
    with xe.Correlator(N, C, T, bits=4, layout=0) as cor:
        cor.set_pipeline(48)
        cor.bind(out)
        for k in range(nblk):
            blk = synth.block_device("sky", 100 + k, N, C, T, 0, dev)
            cor.push(blk)
            cor.sync()                      # the block may be freed after its turn
            oracle.correlate(blk.cpu().numpy(), N, C, T, layout=0, out=want)
        cor.dump_async(out, reset=True)
        assert cor.dump_wait() == xe.CORR_OK
    assert np.array_equal(out.cpu().numpy(), want)


def test_dish_plain_as_batch_of_instances(xe):
    """The plain dish block (32 x 256 x 1024) as twelve independent arrays of
    one batch, the form in which the benchmark measures its throughput (one
    persistent launch per run): every instance in full."""
    N, C, T, n = 32, 256, 1024, 12
    dev = torch.device("cuda")
    blocks = [synth.block_device("gauss", 60 + k, N, C, T, 0, dev) for k in range(n)]
    with xe.Batch([(N, C, T, 4, 0)] * n) as b:
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        b.run()                                          # outputs are overwritten, not added
        assert b.sync() == xe.CORR_OK
        outs = [b.output(k) for k in range(n)]
    for k in range(n):
        assert np.array_equal(outs[k], oracle.correlate(blocks[k].cpu().numpy(), N, C, T, layout=0)), k


def test_batched_mixed_arrays_full_size(xe):
    """The three arrays of the batched workload in one batch run (one
    persistent cross-multiply over all their tasks), Gaussian samples in the
    payload order."""
    shapes = [(32, 256, 1024, 4, 0), (64, 1024, 4096, 4, 0), (192, 4096, 16384, 4, 0)]
    dev = torch.device("cuda")
    blocks = [synth.block_device("gauss", 30 + k, n, c, t, lay, dev)
              for k, (n, c, t, _, lay) in enumerate(shapes)]
    with xe.Batch(shapes) as b:
        for k, blk in enumerate(blocks):
            b.set_input(k, blk)
        b.run()
        assert b.sync() == xe.CORR_OK
        outs = [b.output(k) for k in range(len(shapes))]
    for k in range(2):                                   # 32 and 64 inputs: every entry
        n, c, t, _, lay = shapes[k]
        want = oracle.correlate(blocks[k].cpu().numpy(), n, c, t, layout=lay)
        assert np.array_equal(outs[k], want), shapes[k]
    n, c, t, _, lay = shapes[2]
    host = blocks[2].cpu().numpy()
    del blocks
    chans = np.sort(np.random.default_rng(32).choice(c, size=64, replace=False))
    chans[0], chans[-1] = 0, c - 1
    assert np.array_equal(outs[2][chans], oracle.correlate(host, n, c, t, layout=lay, chans=chans))
    w = _weights(33, 2, n)
    assert np.array_equal(_quadratic_form(outs[2], w),
                          oracle.projected_power(host, n, c, t, w, layout=lay))


def test_service_scale_up_arrays(xe):
    """8-bit requests of 512, 192 and 32 inputs x 2048 channels, 4096 spectra
    each (the 512- and 32-input requests in two blocks), admitted by the HBM
    budget and correlated by shared ticks; 16 seeded channels of every
    request in full and every channel through the quadratic form."""
    C, bits, lay = 2048, 8, 0
    reqs = [(512, 2048, 2), (192, 4096, 1), (32, 2048, 2)]   # inputs, block spectra, blocks
    dev = torch.device("cuda")
    data = {k: [synth.block_device("gauss", 400 + 10 * k + s, n, C, t, lay, dev, bits=bits)
                for s in range(nblk)] for k, (n, t, nblk) in enumerate(reqs)}
    torch.cuda.synchronize()   # a pushed block must be complete: the service copies it on its own stream
    results = {}
    with xe.Service(48 << 30) as svc:
        ids = [svc.submit(n, C, bits, lay, t, nblk) for n, t, nblk in reqs]
        nxt = [0] * len(reqs)
        for _ in range(64):
            for k, rid in enumerate(ids):
                if svc.state(rid) == xe.CORR_REQ_ACTIVE and nxt[k] < len(data[k]):
                    if svc.push(rid, data[k][nxt[k]], check=False) == xe.CORR_OK:
                        nxt[k] += 1
            svc.tick()
            assert svc.wait() == xe.CORR_OK
            for k, rid in enumerate(ids):
                if k not in results and svc.state(rid) == xe.CORR_REQ_DONE:
                    results[k] = svc.fetch(rid)
            if len(results) == len(reqs):
                break
    assert len(results) == len(reqs)
    for k, (n, t, nblk) in enumerate(reqs):
        hosts = [blk.cpu().numpy() for blk in data[k]]
        chans = np.sort(np.random.default_rng(500 + k).choice(C, size=16, replace=False))
        want = None
        for h in hosts:
            want = oracle.correlate(h, n, C, t, bits=bits, layout=lay, chans=chans, out=want)
        assert np.array_equal(results[k][chans], want), (n, t)
        w = _weights(600 + k, 2, n)
        p = sum(oracle.projected_power(h, n, C, t, w, bits=bits, layout=lay) for h in hosts)
        assert np.array_equal(_quadratic_form(results[k], w), p), (n, t)
