"""Failure detection of the bounded device-side waits.

Every wait inside the cross-multiply kernel gives up after a cycle budget,
records CORR_ETIMEDOUT in the context's status word and lets the CTA unwind
(no copy or MMA left in flight, tensor memory freed), so the kernel returns
and the CUDA context stays usable.  The test makes one wait run out on
purpose -- the first CTA's loader withholds one stage, a load that nothing
will ever deliver -- with a short budget, and checks that the dump reports
the timeout, that the kernel came back promptly, and that the same context
then integrates a new block exactly (against the oracle).
"""
import time

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


# stages count per CTA over its tasks: 128 spectra a stage for a two-block
# task, 256 for a one-block (A = B) task; the withheld stage must exist
@pytest.mark.parametrize("N,C,T,stage", [(192, 4, 1024, 2), (64, 8, 2048, 0), (32, 16, 1024, 3)])
def test_withheld_stage_times_out_and_context_recovers(xe, N, C, T, stage):
    blocks = [synth.random_bytes(900 + k, N * C * T) for k in range(2)]
    with xe.Correlator(N, C, T, bits=4, layout=xe.CORR_L_CIT) as cor:
        cor.set_fault_injection(stage, wait_log2=24)            # about 8 ms per wait
        t0 = time.perf_counter()
        cor.push(torch.from_numpy(blocks[0]).cuda())
        cor.dump(check=False)
        elapsed = time.perf_counter() - t0
        assert cor.last_status == xe.CORR_ETIMEDOUT
        assert elapsed < 5.0                                    # returned, not hung
        cor.set_fault_injection(-1, 0)
        cor.push(torch.from_numpy(blocks[1]).cuda())
        vis = cor.dump()                                        # raises on a non-OK status
    assert np.array_equal(vis, oracle.correlate(blocks[1], N, C, T, layout=oracle.L_CIT))
    # the device is still usable by other work afterwards
    x = torch.arange(1024, device="cuda", dtype=torch.int64)
    assert int(x.sum().item()) == 1023 * 1024 // 2
