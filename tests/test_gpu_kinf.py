"""K = infinity on the GPU (§4.4: Alg. 3 runs until the residual is zero).

The plan option K = K_INF splits every real vector into as many levels as it
needs, up to a cap of 8 levels.  On inputs of the §5.1 generator with phi = 0,
1 and 4 the level counts, the Alg. 8 flush schedules, the transform counts and
the output must equal the oracle's K = infinity (K = 0) transform bit for bit;
the counts grow with phi as in §5.2 and §5.4.  A vector that needs more than
the cap sets OZFFT_ERR_LEVELS, and its result is then that of K = 8.
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


def run(oz, x, **kw):
    B, n = x.shape
    plan = oz.Plan(n, B, K=oz.K_INF, **kw)
    y = plan.execute(torch.from_numpy(x).to("cuda:0"))
    torch.cuda.synchronize()
    return y.cpu().numpy(), plan


@pytest.mark.parametrize("n", [1024, 4096, 1 << 14, 3000])
@pytest.mark.parametrize("L", [1, 3])
def test_kinf_matches_oracle(oz, n, L):
    phis = (0.0, 1.0, 4.0)
    x = np.stack([synth.complex_signal("phi", n, 31 + i, batch=1, phi=phi)[0] for i, phi in enumerate(phis)])
    y, plan = run(oz, x, L=L)
    assert plan.status() == oz.OK
    st = plan.stats()
    assert st["K"] == oz.K_INF
    inv = fwd = 0
    per_phi = []
    for b in range(len(phis)):
        yo, info = oracle.ozfft(x[b], N=plan.N, K=0, L=L, trace={"groups"})
        assert plan.alpha == info["alpha"]
        mu = plan.dump(oz.DUMP_MU, b)
        for v in range(2):
            assert np.count_nonzero(mu[v][:oz.K_INF_CAP]) == info["kcount"][v], (b, v)
        sched = plan.dump(oz.DUMP_SCHED, b)
        for c in range(4):
            ref = [(int(info["gS"][c, g]),
                    [tuple(int(t) for t in info["gpairs"][c, g, m]) for m in range(info["gsize"][c, g])])
                   for g in range(info["ngroups"][c])]
            assert sched[c] == ref, (b, c)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b
        inv += info["n_inv"]
        fwd += info["n_fwd_runtime"]
        per_phi.append(info["kcount"][0] + info["kcount"][1])
    assert st["ntt_inverse"] == inv
    assert st["ntt_forward_runtime"] == fwd
    # a wider spread of magnitudes (larger phi) needs at least as many split levels (§5.2, §5.4)
    assert per_phi[0] <= per_phi[1] <= per_phi[2], per_phi


def test_kinf_two_pass_size(oz):
    """A two-pass NTT length (column and row passes) with K = infinity."""
    n = 1 << 16
    x = synth.complex_signal("phi", n, 41, batch=2, phi=4.0)
    y, plan = run(oz, x)
    assert plan.status() == oz.OK
    for b in range(2):
        yo, info = oracle.ozfft(x[b], K=0, L=1)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


def test_kinf_level_cap_reported(oz):
    """One sample of 1e200 and one of 1e-200 among U[-1,1] samples: Alg. 3 takes
    three levels for each of the three magnitudes (nine in all), one more than
    the cap, so the status says so and the result is the K = 8 transform."""
    n = 1024
    x = synth.complex_signal("uniform", n, 43, batch=2)
    x[0, 5] = 1e200
    x[0, 9] = 1e-200 + 3e-201j
    y, plan = run(oz, x)
    assert plan.status() == oz.ERR_LEVELS
    assert plan.status() == oz.OK          # the status word was cleared by the first read
    for b in range(2):
        yo, _ = oracle.ozfft(x[b], N=plan.N, K=oz.K_INF_CAP, L=1)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b
