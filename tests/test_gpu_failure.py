"""Failure detection on the device without a fault: the column pass's wait on
its tile barrier is bounded.  A self-test tile whose barrier expects more bytes
than its copy delivers must end in OZFFT_ERR_TIMEOUT (no invalid address, no
unbounded spin), and the context must stay usable afterwards."""
import time

import numpy as np
import pytest

import oracle
from paper_2603_29129_gb300 import build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oz():
    build.build()
    from paper_2603_29129_gb300 import ozfft
    ozfft.load()
    return ozfft


def test_bounded_wait_times_out_and_context_survives(oz):
    t0 = time.perf_counter()
    assert oz.selftest_wait_timeout() == oz.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    n = 1 << 16                                  # a size whose column pass uses the same TMA kernel
    x = synth.complex_signal("uniform", n, 91, batch=2)
    plan = oz.Plan(n, 2)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    assert np.array_equal(y[1].view(np.uint64), oracle.ozfft(x[1])[0].view(np.uint64))
