"""Large transforms: the benchmark length n = 2^18 and the accumulation-stress
lengths n = 2^20 and 2^22 (uniform parts with 1% spikes of magnitude 1e12,
which force the maximum split count K = 3 on every vector).

At n = 2^18 and 2^20 one signal is compared bit for bit with the oracle's
whole transform.  At n = 2^22, where the oracle takes minutes, sampled bins
are checked against the binary128 DFT, and the transform counts of the
accumulated (L = 3) and plain (L = 1) forms against §4.5's formulas.
"""
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


@pytest.mark.parametrize("n,kind,L", [(1 << 18, "uniform", 1), (1 << 20, "spikes", 3)])
def test_full_size_bit_exact(oz, n, kind, L):
    x = synth.complex_signal(kind, n, 2, batch=2)
    plan = oz.Plan(n, 2, oz.FORWARD, L=L)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    yo, _ = oracle.ozfft(x[1], K=3, L=L)
    assert np.array_equal(y[1].view(np.uint64), yo.view(np.uint64))


@pytest.mark.parametrize("n", [1 << 20, 1 << 22])
def test_stress_sampled_bins_and_counts(oz, n):
    B = 2
    x = synth.complex_signal("spikes", n, 4, batch=B)
    xt = torch.from_numpy(x).cuda()
    bins = np.array([0, 1, 2, n // 3, n // 2, n - 1])
    hi, lo = oracle.dft_q(x[0], bins=bins)
    scale = np.linalg.norm(x[0])                         # rms of the exact spectrum (Parseval)
    for L in (1, 3):
        plan = oz.Plan(n, B, oz.FORWARD, L=L)
        y = plan.execute(xt).cpu().numpy()
        assert plan.status() == oz.OK
        st = plan.stats()
        # spikes of 1e12 over U[-1,1) parts: every vector of x~' needs all K = 3 levels
        assert st["ntt_forward_runtime"] == B * 2 * 3 * 2
        inv_per = st["ntt_inverse"] // (B * 2)          # inverse NTTs per transform and prime
        # L = 1: one group per (s, t) pair (96 NTTs with the 12 of w~*); L = 3: the
        # equal-scale anti-diagonals of 1, 2, 3, 2, 1 pairs become 5 groups (64 NTTs)
        assert inv_per == 4 * (9 if L == 1 else 5)
        assert 12 + 2 * inv_per + 12 == (96 if L == 1 else 64)
        err = np.abs(y[0][bins] - (hi + lo))
        assert np.max(err) <= 1e-14 * scale, (L, err / scale)
