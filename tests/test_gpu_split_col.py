"""The Ozaki split (Alg. 3) fused with the forward NTT's column pass.

The fused kernel transforms the slice residues of every level on chip before
they reach device memory, so the stage dumps (which need the untransformed
residues) turn it off: these tests compare plans with the fusion forced on and
off, bit for bit, and both against the oracle.  They cover every column-stage
count the kernel takes (5..8), K P up to 9 tiles, the 64-bit digits of alpha > 30,
the vectors whose guessed level exponents are redone untransformed (and then
transformed by the column pass alone), and plans over uneven lengths.
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


def _both(oz, x, **kw):
    """Outputs of the plan with the split fused and apart; asserts the stats say which."""
    B, n = x.shape
    xt = torch.from_numpy(x).cuda()
    ys = []
    for f in (1, 2):
        p = oz.Plan(n, B, split_fuse=f, **kw)
        ys.append(p.execute(xt).cpu().numpy())
        assert p.status() == oz.OK
        st = p.stats()
        m1 = int(p.N).bit_length() - 1 - st["row_log_fwd"]
        assert st["split_fused_classes"] == (1 if f == 1 and 5 <= m1 <= 8 else 0), (f, m1, st)
    return ys[0], ys[1], p


def _oracle_bits(x, plan):
    return oracle.ozfft(x, N=plan.N, K=plan.K, L=plan.L, nprimes=plan.nprimes, direction=plan.direction)[0]


@pytest.mark.parametrize("n,row_log", [(10000, 10), (1 << 15, 10), (1 << 16, 10), (40000, 12)])
def test_fused_split_column_stage_counts(oz, n, row_log):
    """5, 6 and 7 column stages (N = 2^15 .. 2^17), fused against apart, both against
    the oracle."""
    x = synth.complex_signal("phi", n, 80, batch=2, phi=2.0)
    yf, ya, plan = _both(oz, x, row_log=row_log)
    assert np.array_equal(yf.view(np.uint64), ya.view(np.uint64))
    for b in range(2):
        assert np.array_equal(yf[b].view(np.uint64), _oracle_bits(x[b], plan).view(np.uint64)), b


def test_fused_split_eight_column_stages(oz):
    """N = 2^18 with a row pass of 10 stages (8 column stages, 8-column tiles), and the
    default split (6 column stages): fused, apart and the stage-dump plan agree."""
    n, B = 1 << 17, 2
    x = synth.complex_signal("gaussian", n, 81, batch=B)
    xt = torch.from_numpy(x).cuda()
    ref = oz.Plan(n, B, debug=True).execute(xt).cpu().numpy()
    for kw in (dict(row_log=10), {}):
        yf, ya, _ = _both(oz, x, **kw)
        assert np.array_equal(yf.view(np.uint64), ref.view(np.uint64)), kw
        assert np.array_equal(ya.view(np.uint64), ref.view(np.uint64)), kw


@pytest.mark.parametrize("kw", [dict(K=4), dict(K=1), dict(K=3, nprimes=3), dict(K=2, nprimes=3),
                                dict(K=4, L=3, merge=True)])
def test_fused_split_levels_and_primes(oz, kw):
    """K P from 2 to 9 tiles; K = 2 with three primes has alpha > 30 (64-bit digits)."""
    n = 5000
    x = synth.complex_signal("uniform", n, 82, batch=2)
    yf, ya, plan = _both(oz, x, row_log=9, **kw)
    if kw == dict(K=2, nprimes=3):
        assert plan.alpha > 30
    assert np.array_equal(yf.view(np.uint64), ya.view(np.uint64))
    for b in range(2):
        assert np.array_equal(yf[b].view(np.uint64), _oracle_bits(x[b], plan).view(np.uint64)), b


def test_fused_split_guess_redone(oz):
    """Vectors whose guessed level exponents fail (a short second slice, or none)
    next to vectors where the guess holds: the redone ones are rewritten
    untransformed and transformed by the column pass alone, the others are left
    as the fused kernel wrote them; the output matches the oracle."""
    n = 10000
    xs = synth.complex_signal("uniform", n, 83, batch=6)
    xs[1] = 0.0
    xs[1, 0] = (1.0 + 2.0 ** -40) + (3.0 - 2.0 ** -45) * 1j
    xs[2] = 0.0
    xs[2, 0] = 1.0 - 0.5j
    xs[3, 1:] *= 2.0 ** -30
    xs[3, 0] = 1.0 + 2.0 ** -20
    xs[4] = synth.complex_signal("spikes", n, 84)[0]
    xs[5] = 0.0                                       # all levels empty
    yf, ya, plan = _both(oz, xs, row_log=10)
    assert np.array_equal(yf.view(np.uint64), ya.view(np.uint64))
    for b in range(xs.shape[0]):
        assert np.array_equal(yf[b].view(np.uint64), _oracle_bits(xs[b], plan).view(np.uint64)), b


def test_fused_split_repeated_executions(oz):
    """The redo flags are rewritten every execution: a batch whose guess fails,
    then one where it holds, then the first again, on one plan."""
    n, B = 10000, 2
    good = synth.complex_signal("uniform", n, 85, batch=B)
    bad = good.copy()
    bad[:, 1:] = 0.0
    bad[:, 0] = 1.0 + 2.0 ** -40
    p = oz.Plan(n, B, row_log=10, split_fuse=1)
    assert p.stats()["split_fused_classes"] == 1
    for x in (bad, good, bad):
        y = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
        for b in range(B):
            assert np.array_equal(y[b].view(np.uint64), _oracle_bits(x[b], p).view(np.uint64)), b


def test_fused_split_autotuned(oz):
    """With the autotuner the split fusion is timed like the NTT split: any choice
    gives the same bits as the plan with the split apart."""
    n, B = 1 << 16, 3
    x = torch.from_numpy(synth.complex_signal("phi", n, 86, batch=B, phi=1.0)).cuda()
    ya = oz.Plan(n, B, split_fuse=2).execute(x).cpu().numpy()
    p = oz.Plan(n, B, autotune=True)
    y = p.execute(x).cpu().numpy()
    assert np.array_equal(y.view(np.uint64), ya.view(np.uint64))
    assert p.stats()["split_fused_classes"] in (0, 1)


def test_fused_split_uneven_lengths(oz):
    """A plan over uneven lengths with the fusion forced (the classes with N = 2^17
    .. 2^18 fuse, the smaller ones have too few column stages) and with it off:
    the same bits, and each signal bit-exact against the oracle."""
    lens = [70000, 100000, 3000, 131072, 65537, 5000]
    xh = synth.complex_signal("phi", int(np.sum(lens)), 87, phi=4.0)[0]
    x = torch.from_numpy(xh).cuda()
    outs = []
    for f in (1, 2):
        p = oz.PlanMany(lens, split_fuse=f)
        outs.append(p.execute(x).cpu().numpy())
        assert p.status() == oz.OK
        st = p.stats()
        assert (st["split_fused_classes"] >= 1) if f == 1 else (st["split_fused_classes"] == 0), st
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    xs, ys = p.split(xh), p.split(outs[0])
    for i in range(len(lens)):
        yo, _ = oracle.ozfft(xs[i])
        assert np.array_equal(ys[i].view(np.uint64), yo.view(np.uint64)), (i, lens[i])
