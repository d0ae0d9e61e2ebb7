"""The TS (triple-single) variant through the C ABI against the oracle's TS
variant: slice residues, spectra, flush schedules, inverse-NTT residues and the
final binary64 output bit-exact; the output within 1e-15 of the binary128 DFT."""
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


CASES = [(1024, 3, 1, "uniform"), (1000, 3, 1, "phi"), (777, 4, 2, "gaussian"), (4096, 3, 3, "spikes"),
         (64, 1, 1, "uniform"), (1 << 14, 3, 1, "loguniform")]


@pytest.mark.parametrize("case", CASES)
def test_ts_every_stage_bit_exact(oz, case):
    n, K, L, kind = case
    x = synth.complex_signal(kind, n, 81, batch=2, phi=4.0)
    plan = oz.Plan(n, 2, K=K, L=L, ts=True, debug=True)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    for b in range(2):
        yo, info = oracle.ozfft_ts(x[b], N=plan.N, K=K, L=L, trace={"q", "spec", "groups", "zres"})
        assert plan.alpha == info["alpha"] == oracle.alpha_ts(n, L)
        res, spec = plan.dump(oz.DUMP_XRES, b), plan.dump(oz.DUMP_XSPEC, b)
        for v in range(2):
            for k in range(info["kcount"][v]):
                for i in range(2):
                    p = oracle.prime(i)
                    assert np.array_equal(res[v, k, i], (info["q"][v, k] % p).astype(np.uint32)), (b, v, k, i)
                    assert np.array_equal(spec[v, k, i], info["spec"][v, k, i]), (b, v, k, i)
        sched, zres = plan.dump(oz.DUMP_SCHED, b), plan.dump(oz.DUMP_ZRES, b)
        for c in range(4):
            ng = info["ngroups"][c]
            ref = [(int(info["gS"][c, g]), [tuple(int(t) for t in info["gpairs"][c, g, m])
                                            for m in range(info["gsize"][c, g])]) for g in range(ng)]
            assert sched[c] == ref, (b, c)
            for g in range(ng):
                assert np.array_equal(zres[c, g], info["zres"][c, g]), (b, c, g)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


@pytest.mark.parametrize("n", [1 << 16, 3000])
def test_ts_larger_and_accuracy(oz, n):
    x = synth.complex_signal("uniform", n, 82, batch=2)
    plan = oz.Plan(n, 2, ts=True)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(2):
        yo, _ = oracle.ozfft_ts(x[b], N=plan.N)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b
    hi, lo = oracle.fft_q(x[0]) if n & (n - 1) == 0 else oracle.dft_q(x[0])
    assert oracle.rel_l2_error(y[0], hi, lo) <= 1e-15


def test_ts_directions_and_errors(oz):
    n = 1000
    x = synth.complex_signal("gaussian", n, 83, batch=1)
    xt = torch.from_numpy(x).cuda()
    for d in (oz.INVERSE, oz.ADJOINT, oz.INVERSE_ADJOINT):
        y = oz.Plan(n, 1, d, ts=True).execute(xt).cpu().numpy()
        assert np.array_equal(y[0].view(np.uint64), oracle.ozfft_ts(x[0], direction=d)[0].view(np.uint64)), d
    big = np.full((1, 64), 1e39 + 0j)          # outside the binary32 range of TS words
    p = oz.Plan(64, 1, ts=True)
    p.execute(torch.from_numpy(big).cuda())
    assert p.status() == oz.ERR_RANGE
    nan = synth.complex_signal("uniform", 64, 84, batch=1)
    nan[0, 3] = np.nan
    p.execute(torch.from_numpy(nan).cuda())
    assert p.status() == oz.ERR_NONFINITE
    with pytest.raises(oz.OzfftError):
        oz.Plan(64, 1, ts=True, nprimes=3)
    with pytest.raises(oz.OzfftError):
        oz.Plan(64, 1, ts=True, L=2, merge=True)
