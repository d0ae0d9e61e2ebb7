"""ozfft_execute_noalloc, the entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc (code inside an application that
owns the device memory pool, or latency-critical paths that must not enter the
allocator): its whole workspace is a static device array.  Through the C ABI,
its output must equal, bit for bit, what ozfft_execute gives on a plan for the
same length and direction, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that everything which must start at
zero is cleared).  This file is collected last so that a run that stops at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2603_29129_gb300 import build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oz():
    build.build()
    from paper_2603_29129_gb300 import ozfft
    ozfft.load()
    return ozfft


@pytest.mark.parametrize("n,direction", [(1000, -1), (4096, 1), (8192, -1), (777, -1)])
def test_noalloc_equals_planned_execution(oz, n, direction):
    plan = oz.Plan(n, 1, direction)
    for seed in (1, 2):          # two calls in a row on the shared static array
        x = torch.from_numpy(synth.complex_signal("phi", n, seed, phi=1.0)[0]).to("cuda:0")
        ref = plan.execute(x)
        out = torch.full_like(x, float("nan"))
        oz.execute_noalloc(x, out, direction)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.cpu().numpy().view(np.uint64)), (n, seed)


def test_noalloc_rejects_lengths_beyond_its_array(oz):
    x = torch.zeros(4097, dtype=torch.complex128, device="cuda:0")   # N = 16384 > 8192
    with pytest.raises(oz.OzfftError) as e:
        oz.execute_noalloc(x, torch.empty_like(x))
    assert e.value.code == oz.ERR_LENGTH
