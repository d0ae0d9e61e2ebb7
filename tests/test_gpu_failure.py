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


def _plan_bit_exact(oz, n=4096, seed=92):
    x = synth.complex_signal("uniform", n, seed, batch=2)
    plan = oz.Plan(n, 2)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    for b in range(2):
        assert np.array_equal(y[b].view(np.uint64), oracle.ozfft(x[b])[0].view(np.uint64)), b


@pytest.mark.parametrize("spec", ["alloc", "alloc:1", "alloc:4", "alloc:9", "alloc:15"])
def test_injected_allocation_failure_in_plan_creation(oz, monkeypatch, spec):
    """OZFFT_FAULT=alloc[:N] fails a device allocation while the plan is built
    (the first, middle ones, the last of the 15 a plain plan makes); creation
    reports it and frees what it had allocated, and the next plan on the same
    context is bit-exact."""
    monkeypatch.setenv("OZFFT_FAULT", spec)
    with pytest.raises(oz.OzfftError, match="OZFFT_FAULT"):
        oz.Plan(4096, 2)
    monkeypatch.delenv("OZFFT_FAULT")
    _plan_bit_exact(oz)


def test_injected_allocation_failure_in_host_execution(oz, monkeypatch):
    """The staging buffers of a first host-buffer execution fail to allocate:
    the call returns OZFFT_ERR_ALLOC, and after the hook is cleared the same
    plan runs from host buffers bit-exactly."""
    n = 4096
    x = synth.complex_signal("uniform", n, 93, batch=2)
    plan = oz.Plan(n, 2)
    xin = torch.from_numpy(x).pin_memory()
    out = torch.empty_like(xin).pin_memory()
    for spec in ("alloc", "alloc:2"):
        monkeypatch.setenv("OZFFT_FAULT", spec)
        with pytest.raises(oz.OzfftError) as ei:
            plan.execute_host(xin, out)
        assert ei.value.code == oz.ERR_ALLOC
    monkeypatch.delenv("OZFFT_FAULT")
    plan.execute_host(xin, out)
    for b in range(2):
        assert np.array_equal(out[b].numpy().view(np.uint64), oracle.ozfft(x[b])[0].view(np.uint64)), b


@pytest.mark.parametrize("code", ["ERR_NONFINITE", "ERR_RANGE", "ERR_TIMEOUT", "ERR_LEVELS"])
def test_injected_device_status(oz, monkeypatch, code):
    """OZFFT_FAULT=status:C makes an execution record status C as its kernels
    would; ozfft_get_status reports it once, and the next execution without the
    hook is clean and bit-exact."""
    c = getattr(oz, code)
    n = 4096
    x = synth.complex_signal("uniform", n, 94, batch=2)
    plan = oz.Plan(n, 2)
    xt = torch.from_numpy(x).cuda()
    monkeypatch.setenv("OZFFT_FAULT", f"status:{c}")
    plan.execute(xt)
    assert plan.status() == c
    assert plan.status() == oz.OK
    monkeypatch.delenv("OZFFT_FAULT")
    y = plan.execute(xt).cpu().numpy()
    assert plan.status() == oz.OK
    assert np.array_equal(y[0].view(np.uint64), oracle.ozfft(x[0])[0].view(np.uint64))
