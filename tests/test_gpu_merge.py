"""Merged schedules: NTT-domain accumulation across the two real convolutions of
one output part (RR with -II, IR with RI).

y' is the exactly rounded sum of the same rescaled products however they are
grouped, so a merged plan must give the same bits as an unmerged plan with the
same L (and as the oracle); the number of inverse NTTs must be the brute-force
count of equal-scale groups of at most L products per output part.
"""
import math
from collections import Counter

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


def merged_groups(info, L):
    """Groups per output part: products (s, t) of both of its convolutions with
    scale sx[s] + sy[t], counted per distinct scale in chunks of L."""
    sexp = info["sexp"]                          # vectors: Re x', Im x', Re w*, Im w*
    total = 0
    for convs in (((0, 2), (1, 3)), ((1, 2), (0, 3))):
        scales = Counter()
        for vx, vw in convs:
            for a in sexp[vx]:
                for b in sexp[vw]:
                    scales[a + b] += 1
        total += sum(math.ceil(c / L) for c in scales.values())
    return total


@pytest.mark.parametrize("n,L,P,kind", [(1024, 2, 2, "uniform"), (1000, 3, 2, "phi"), (4096, 4, 2, "gaussian"),
                                        (777, 2, 3, "loguniform"), (1 << 14, 6, 2, "spikes")])
def test_merged_equals_unmerged_and_oracle(oz, n, L, P, kind):
    B = 3
    x = synth.complex_signal(kind, n, 71, batch=B, phi=4.0)
    xt = torch.from_numpy(x).cuda()
    pm = oz.Plan(n, B, L=L, nprimes=P, merge=True)
    pu = oz.Plan(n, B, L=L, nprimes=P)
    ym = pm.execute(xt).cpu().numpy()
    yu = pu.execute(xt).cpu().numpy()
    assert np.array_equal(ym.view(np.uint64), yu.view(np.uint64))
    groups = 0
    for b in range(B):
        yo, info = oracle.ozfft(x[b], L=L, nprimes=P)
        assert np.array_equal(ym[b].view(np.uint64), yo.view(np.uint64)), b
        groups += merged_groups(info, L)
    assert pm.stats()["ntt_inverse"] == groups * P
    assert pm.stats()["ntt_inverse"] <= pu.stats()["ntt_inverse"]


def test_merged_counts_without_gaps(oz):
    """Without gaps every part has scales S0 + k alpha with 2, 4, 6, 4, 2 products
    (K = 3): 9 groups per part at L = 2 (36 inverse NTTs with two primes instead
    of 48 unmerged), 5 at L = 6 (20 instead of 40 at L = 3 unmerged)."""
    x = synth.complex_signal("uniform", 4096, 72, batch=1)   # Re and Im share their split scales
    xt = torch.from_numpy(x).cuda()
    for L, expect in ((2, 36), (3, 32), (6, 20)):
        info = oracle.ozfft(x[0], L=L)[1]
        assert info["sexp"][0] == info["sexp"][1] and info["sexp"][2] == info["sexp"][3]
        assert merged_groups(info, L) * 2 == expect
        p = oz.Plan(4096, 1, L=L, merge=True)
        p.execute(xt)
        assert p.stats()["ntt_inverse"] == expect, L


def test_merged_wide_spans_and_uneven(oz):
    n = 4096
    xs = synth.complex_signal("uniform", n, 73, batch=2)
    xs[0, 1:] *= 1e-120
    xs[0, 0] = 1.0
    y = oz.Plan(n, 2, L=3, merge=True).execute(torch.from_numpy(xs).cuda()).cpu().numpy()
    for b in range(2):
        assert np.array_equal(y[b].view(np.uint64), oracle.ozfft(xs[b], L=3)[0].view(np.uint64))
    lens = [1000, 5000, 64, 3333, 20000]
    x = synth.complex_signal("loguniform", sum(lens), 74)[0]
    pl = oz.PlanMany(lens, L=2, merge=True)
    y = pl.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    for xi, yi in zip(pl.split(x), pl.split(y)):
        assert np.array_equal(yi.view(np.uint64), oracle.ozfft(xi, L=2)[0].view(np.uint64))
