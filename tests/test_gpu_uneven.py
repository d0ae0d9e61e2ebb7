"""Plans over signals of uneven lengths (ozfft_plan_many), through the C ABI.

Each signal of the packed batch must equal, bit for bit, the oracle's
transform of that signal alone (its own N, chirp, w~* and alpha), whatever
the grouping into length classes, the inverse-stage chunking, the NTT split
chosen by the autotuner, and whether the classes run from the captured CUDA
graph or on plain streams.
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


MIXED = [1, 2, 3, 7, 16, 100, 1000, 1024, 1500, 2048, 4097, 5000, 777, 64, 8192, 3, 1000, 12000, 20000, 65536]


def packed(lengths, kind, seed):
    total = int(np.sum(lengths))
    return synth.complex_signal(kind, total, seed, phi=4.0)[0]


def check_against_oracle(plan, x, y, idx=None, **kw):
    xs, ys = plan.split(x), plan.split(y)
    for i in (range(plan.batch) if idx is None else idx):
        yo, _ = oracle.ozfft(xs[i], K=plan.K, L=plan.L, nprimes=plan.nprimes, direction=plan.direction, **kw)
        assert np.array_equal(ys[i].view(np.uint64), yo.view(np.uint64)), (i, len(xs[i]))


@pytest.mark.parametrize("kind", ["loguniform", "phi", "spikes"])
def test_mixed_lengths_bit_exact(oz, kind):
    plan = oz.PlanMany(MIXED)
    x = packed(MIXED, kind, 61)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    check_against_oracle(plan, x, y)


@pytest.mark.parametrize("opts", [dict(L=3), dict(nprimes=3), dict(direction=1), dict(direction=2, L=2)])
def test_mixed_lengths_options(oz, opts):
    lens = [5, 1000, 1024, 3000, 333, 4096, 17, 9000]
    plan = oz.PlanMany(lens, **opts)
    x = packed(lens, "uniform", 62)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    check_against_oracle(plan, x, y)


def test_graph_chunking_autotune_agree(oz):
    """No graph, one signal per chunk, and autotuned NTT splits give the same bits
    as the default plan; two executions in a row with other inputs (the graph
    reads the current pointers), in place."""
    lens = [3000, 70000, 5000, 1024, 40000, 131072, 2500, 100000]
    x1 = torch.from_numpy(packed(lens, "loguniform", 63)).cuda()
    x2 = torch.from_numpy(packed(lens, "gaussian", 64)).cuda()
    ref = oz.PlanMany(lens)
    r1, r2 = ref.execute(x1).cpu().numpy(), ref.execute(x2).cpu().numpy()
    check_against_oracle(ref, x1.cpu().numpy(), r1, idx=[0, 3, 6])
    for kw in (dict(graph=False), dict(chunk=1), dict(autotune=True), dict(autotune=True, chunk=3)):
        p = oz.PlanMany(lens, **kw)
        for x, r in ((x1, r1), (x2, r2), (x1, r1)):
            y = p.execute(x).cpu().numpy()
            assert np.array_equal(y.view(np.uint64), r.view(np.uint64)), kw
        xi = x2.clone()
        p.execute(xi, out=xi)
        assert np.array_equal(xi.cpu().numpy().view(np.uint64), r2.view(np.uint64)), kw


def test_autotuned_and_forced_splits(oz):
    """The autotuner's choice and every forced row/column split give the same bits."""
    n, B = 1 << 16, 4
    x = torch.from_numpy(synth.complex_signal("uniform", n, 65, batch=B)).cuda()
    a = oz.Plan(n, B).execute(x).cpu().numpy()
    b = oz.Plan(n, B, autotune=True).execute(x).cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    for m2 in (10, 11, 13, 14):       # column passes of 2^6 (TMA) down to 2^2 (per-thread loads) rows
        p = oz.Plan(n, B, row_log=m2)
        assert p.stats()["row_log_inv"] == m2
        c = p.execute(x).cpu().numpy()
        assert np.array_equal(a.view(np.uint64), c.view(np.uint64)), m2
    with pytest.raises(oz.OzfftError):
        oz.Plan(n, B, row_log=3)


def test_status_stats_and_errors(oz):
    lens = [100, 5000, 300]
    plan = oz.PlanMany(lens)
    x = packed(lens, "uniform", 66)
    bad = x.copy()
    bad[150] = np.inf                                   # inside the second signal
    plan.execute(torch.from_numpy(bad).cuda())
    assert plan.status() == oz.ERR_NONFINITE
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    check_against_oracle(plan, x, y)
    st = plan.stats()
    assert st["batch"] == 3 and st["n"] == 5400 and st["N"] == 16384
    assert st["alpha"] == min(oracle.alpha(n, 1, 2) for n in lens)
    # uniform U[-1,1) parts: every x~' vector needs all three levels (as the oracle counts)
    infos = [oracle.ozfft(s)[1] for s in plan.split(x)]
    assert st["ntt_forward_runtime"] == sum(i["n_fwd_runtime"] for i in infos)
    assert st["ntt_inverse"] == sum(i["n_inv"] for i in infos)
    assert st["ntt_forward_plan"] == sum(i["n_fwd_plan"] for i in infos)
    hin = np.ascontiguousarray(x)
    hout = np.empty_like(hin)
    plan.execute_host(hin, hout)
    assert np.array_equal(hout.view(np.uint64), y.view(np.uint64))
    with pytest.raises(oz.OzfftError):
        oz.PlanMany([])
    with pytest.raises(oz.OzfftError):
        oz.PlanMany([10, 0, 5])
    with pytest.raises(oz.OzfftError):
        plan.set_profiling(True)


def test_log_uniform_batch_sampled(oz):
    """512 lengths of the log-uniform [1000, 300000] draw (powers of two
    redrawn), parts +-10^U[-8,8]; the smallest, median and largest signals
    against the oracle, the rest against the binary128 DFT at sampled bins."""
    lens = synth.uneven_lengths(512, 3)
    x = packed(lens, "loguniform", 67)
    plan = oz.PlanMany(lens)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    order = np.argsort(lens)
    check_against_oracle(plan, x, y, idx=[int(order[0]), int(order[len(order) // 2]), int(order[-1])])
    xs, ys = plan.split(x), plan.split(y)
    for i in range(0, 512, 64):
        bins = np.array([0, 1, len(xs[i]) // 2, len(xs[i]) - 1])
        hi, lo = oracle.dft_q(xs[i], bins=bins)
        assert np.max(np.abs(ys[i][bins] - (hi + lo))) <= 1e-14 * np.linalg.norm(xs[i]), i


@pytest.mark.parametrize("opts", [dict(crt_fuse=1), dict(crt_fuse=2), dict(inv_vecs=1), dict(inv_vecs=2),
                                  dict(row_log=11), dict(crt_fuse=1, inv_vecs=1, L=3),
                                  dict(crt_fuse=1, L=3, merge=True), dict(autotune=True)])
def test_each_tuned_choice_forced(oz, opts):
    """Every choice the autotuner makes per length class, forced in turn: the
    inverse column pass fused with the CRT or not, one or two vectors per CTA
    in the inverse row pass, a forced NTT split; each plan is bit-exact against
    the oracle's transform of every signal alone, and stats report the choice."""
    lens = [3000, 70000, 5000, 1024, 40000, 131072, 2500, 100000, 777, 16]
    x = packed(lens, "phi", 68)
    plan = oz.PlanMany(lens, **opts)
    y = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    check_against_oracle(plan, x, y)
    st = plan.stats()
    assert st["classes"] == len({1 << (2 * n - 2).bit_length() if n & (n - 1) else n for n in lens})
    if opts.get("crt_fuse") == 2:
        assert st["crt_fused_classes"] == 0
    if opts.get("crt_fuse") == 1:
        assert st["crt_fused_classes"] >= 1
    if "inv_vecs" in opts and not opts.get("L", 1) > 1:
        assert st["inv_vecs"] == opts["inv_vecs"]


@pytest.mark.parametrize("n,kw", [(4096, {}), (1 << 14, {}), (1 << 16, {}), (3000, {}), (1 << 14, dict(L=3, merge=True)),
                                  (4096, dict(K=-1)), (1 << 16, dict(nprimes=3, K=2))])
def test_inverse_row_vectors_per_cta_agree(oz, n, kw):
    """The inverse row pass with one and with two vectors of a prime per CTA
    (twiddle loads shared): bit-identical, and bit-exact against the oracle."""
    B = 3
    x = synth.complex_signal("phi", n, 69, batch=B, phi=1.0)
    xt = torch.from_numpy(x).cuda()
    ys = []
    for v in (1, 2):
        p = oz.Plan(n, B, inv_vecs=v, **kw)
        ys.append(p.execute(xt).cpu().numpy())
        assert p.status() == oz.OK
    assert np.array_equal(ys[0].view(np.uint64), ys[1].view(np.uint64))
    K = kw.get("K", 3)
    for b in range(B):
        yo, _ = oracle.ozfft(x[b], K=0 if K == -1 else K, L=kw.get("L", 1), nprimes=kw.get("nprimes", 2))
        assert np.array_equal(ys[1][b].view(np.uint64), yo.view(np.uint64)), b


def test_plain_plan_crt_fusion_forced(oz):
    """A plain plan with the inverse column pass fused with the CRT and without
    it, and the autotuned choice: the same bits."""
    n, B = 1 << 16, 4
    x = torch.from_numpy(synth.complex_signal("uniform", n, 70, batch=B)).cuda()
    outs = []
    for kw in (dict(crt_fuse=1), dict(crt_fuse=2), dict(autotune=True)):
        p = oz.Plan(n, B, **kw)
        outs.append(p.execute(x).cpu().numpy())
        st = p.stats()
        if kw.get("crt_fuse") == 1:
            assert st["crt_fused_classes"] == 1
        if kw.get("crt_fuse") == 2:
            assert st["crt_fused_classes"] == 0
    for o in outs[1:]:
        assert np.array_equal(outs[0].view(np.uint64), o.view(np.uint64))
