"""GPU path (through the C ABI) against the CPU oracle, element by element.

Integer stages (slice residues, spectra, flush schedules, inverse-NTT residues)
must be bit-exact.  The binary64 stages (chirp table, x~', per-level maxima and
the final output) must also be bit-exact: both sides evaluate the same IEEE-754
operations in the same order (correctly rounded chirp, fma-form complex
products, Alg. 3's exact split) or the same exactly defined quantity (the exact
sum of the rescaled CRT integers, rounded once to nearest).  The final output is additionally held to the method's accuracy
target, relative l2 error <= 1e-15 against the binary128 DFT.
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


def run_gpu(oz, x, **kw):
    """x: [B, n] complex128 numpy.  Returns (y numpy, plan)."""
    B, n = x.shape
    plan = oz.Plan(n, B, **kw)
    xt = torch.from_numpy(x).to("cuda:0")
    y = plan.execute(xt)
    torch.cuda.synchronize()
    return y.cpu().numpy(), plan


def oracle_vs(x1, plan, **kw):
    return oracle.ozfft(x1, N=plan.N, K=plan.K, L=plan.L, nprimes=plan.nprimes,
                        direction=plan.direction, **kw)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 100, 1000, 1024, 4097, 1 << 16])
def test_chirp_table_bit_exact(oz, n):
    plan = oz.Plan(n, 1)
    w = plan.dump(oz.DUMP_CHIRP)
    assert np.array_equal(w.view(np.uint64), oracle.chirp(n).view(np.uint64))


STAGE_CASES = [  # n, N (0 = default), K, L, nprimes
    (1024, 2048, 3, 1, 2),
    (1024, 0, 3, 1, 2),
    (1024, 2048, 3, 1, 3),
    (1024, 0, 3, 3, 2),
    (1000, 0, 3, 1, 2),
    (777, 0, 4, 2, 3),
    (64, 0, 1, 1, 2),
    (4096, 0, 2, 3, 2),
    (4096, 0, 2, 1, 3),     # three primes, K = 2 (alpha 39 at this n): the three-prime Horner path
    (1000, 0, 2, 2, 3),
]


@pytest.mark.parametrize("case", STAGE_CASES)
def test_every_stage_bit_exact(oz, case):
    n, N, K, L, P = case
    x = synth.complex_signal("phi", n, 11, batch=2, phi=1.0)
    y, plan = run_gpu(oz, x, K=K, L=L, nprimes=P, conv_len=N, debug=True)
    assert plan.status() == oz.OK
    for b in range(2):
        yo, info = oracle_vs(x[b], plan, trace={"xprime", "q", "spec", "groups", "zres", "yprime"})
        kc = info["kcount"]
        assert plan.alpha == info["alpha"]
        assert np.array_equal(plan.dump(oz.DUMP_XPRIME, b), info["xprime"])
        mu = plan.dump(oz.DUMP_MU, b)
        res = plan.dump(oz.DUMP_XRES, b)
        spec = plan.dump(oz.DUMP_XSPEC, b)
        for v in range(2):
            assert np.count_nonzero(mu[v][:K]) == kc[v]
            for k in range(kc[v]):
                q = info["q"][v, k]
                for i in range(P):
                    p = oracle.prime(i)
                    assert np.array_equal(res[v, k, i], (q % p).astype(np.uint32)), (b, v, k, i)
                    assert np.array_equal(spec[v, k, i], info["spec"][v, k, i]), (b, v, k, i)
        ysp = plan.dump(oz.DUMP_YSPEC)
        for v in range(2):
            for k in range(info["kcount"][2 + v]):
                for i in range(P):
                    p = oracle.prime(i)
                    f = pow(plan.N, p - 2, p) * (1 << 32) % p
                    expect = (info["spec"][2 + v, k, i].astype(np.uint64) * np.uint64(f)) % np.uint64(p)
                    assert np.array_equal(ysp[v, k, i].astype(np.uint64), expect)
        sched = plan.dump(oz.DUMP_SCHED, b)
        zres = plan.dump(oz.DUMP_ZRES, b)
        for c in range(4):
            ng = info["ngroups"][c]
            ref = [(int(info["gS"][c, g]),
                    [tuple(int(t) for t in info["gpairs"][c, g, m]) for m in range(info["gsize"][c, g])])
                   for g in range(ng)]
            assert sched[c] == ref, (b, c)
            for g in range(ng):
                assert np.array_equal(zres[c, g], info["zres"][c, g]), (b, c, g)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


@pytest.mark.parametrize("n,kind", [(1 << 14, "uniform"), (1 << 15, "phi"), (1 << 16, "gaussian"),
                                    (3 * 1024 + 5, "loguniform"), (20000, "spikes")])
def test_multi_pass_sizes_bit_exact(oz, n, kind):
    """Sizes that take the two-pass NTT and span many CTA tiles."""
    x = synth.complex_signal(kind, n, 5, batch=2, phi=4.0)
    y, plan = run_gpu(oz, x)
    for b in range(2):
        yo, _ = oracle_vs(x[b], plan)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


def test_wide_scale_spans(oz):
    """A dominant sample over a sea of tiny ones leaves split levels with gaps,
    so the flush groups' scales span more than the register accumulator holds;
    such signals take the shared-memory accumulation path, still bit-exact."""
    n = 4096
    xs = synth.complex_signal("uniform", n, 12, batch=3)
    for b, tiny in enumerate((1e-50, 1e-100, 1e-200)):
        xs[b, 1:] *= tiny
        xs[b, 0] = 1.0
    for P in (2, 3):
        y, plan = run_gpu(oz, xs, nprimes=P)
        assert plan.status() == oz.OK
        for b in range(3):
            yo, _ = oracle_vs(xs[b], plan)
            assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), (P, b)


@pytest.mark.parametrize("tiny", [1e-9, 1e-12, 1e-20, 1e-30])
def test_split_gaps_moderate_spans(oz, tiny):
    """A dominant sample over samples 1e-9 .. 1e-30 smaller: the split levels
    have gaps, so flush-group scales are not monotone in schedule order, with
    scale spans that still fit the register accumulator."""
    n = 2048
    xs = synth.complex_signal("uniform", n, 15, batch=2)
    xs[:, 1:] *= tiny
    xs[:, 0] = 1.0 - 0.5j
    for L in (1, 3):
        y, plan = run_gpu(oz, xs, L=L)
        for b in range(2):
            yo, _ = oracle_vs(xs[b], plan)
            assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), (tiny, L, b)


def test_split_exponent_guess_redone(oz):
    """The one-pass split guesses e_k = e_0 - k alpha for the later levels and
    redoes, level by level, every vector whose residual maxima say otherwise.
    Impulses whose value has a short second slice (1 + 2^-40: the level-1
    residual is far below its bound) or none at all (1.0) sit in one batch with
    vectors where the guess holds; every level's residues and the output must
    match the oracle."""
    n = 10000                         # N = 2^15: several CTAs per vector in the one-pass kernel
    xs = synth.complex_signal("uniform", n, 16, batch=5)
    xs[1] = 0.0
    xs[1, 0] = (1.0 + 2.0 ** -40) + (3.0 - 2.0 ** -45) * 1j
    xs[2] = 0.0
    xs[2, 0] = 1.0 - 0.5j
    xs[3, 1:] *= 2.0 ** -30            # level 1 of a dominant first sample over small ones
    xs[3, 0] = 1.0 + 2.0 ** -20
    xs[4] = synth.complex_signal("spikes", n, 17)[0]
    y, plan = run_gpu(oz, xs, debug=True)
    assert plan.status() == oz.OK
    for b in range(xs.shape[0]):
        yo, info = oracle_vs(xs[b], plan, trace={"q"})
        res = plan.dump(oz.DUMP_XRES, b)
        mu = plan.dump(oz.DUMP_MU, b)
        for v in range(2):
            assert np.count_nonzero(mu[v][:plan.K]) == info["kcount"][v], (b, v)
            for k in range(info["kcount"][v]):
                for i in range(plan.nprimes):
                    p = oracle.prime(i)
                    assert np.array_equal(res[v, k, i], (info["q"][v, k] % p).astype(np.uint32)), (b, v, k, i)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


@pytest.mark.parametrize("n,row_log", [(1 << 16, 0), (1 << 16, 11), (1 << 17, 10)])
def test_gap_spans_in_two_pass_sizes(oz, n, row_log):
    """Gap-producing inputs at two-pass lengths (4, 5 and 7 column stages), so that the
    inverse column pass fused with the CRT meets signals off its Horner path (column pass
    only, written back for the limb kernels) next to signals on it."""
    xs = synth.complex_signal("uniform", n, 18, batch=4)
    xs[1, 1:] *= 1e-12
    xs[1, 0] = 1.0 - 0.5j
    xs[2, 1:] *= 1e-100
    xs[2, 0] = 1.0
    y, plan = run_gpu(oz, xs, row_log=row_log) if row_log else run_gpu(oz, xs)
    assert plan.status() == oz.OK
    for b in range(4):
        yo, _ = oracle_vs(xs[b], plan)
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), (row_log, b)


def test_fused_column_stage_counts_agree(oz):
    """The fused column pass + CRT with 6, 7 and 8 column stages (row passes of 12, 11,
    10 stages) and the unfused kernels (stage dumps on) give the same bits."""
    n, B = 1 << 18, 2
    x = torch.from_numpy(synth.complex_signal("phi", n, 19, batch=B, phi=4.0)).cuda()
    ref = oz.Plan(n, B, debug=True).execute(x).cpu().numpy()
    for m2 in (12, 11, 10):
        p = oz.Plan(n, B, row_log=m2)
        assert p.stats()["row_log_inv"] == m2
        y = p.execute(x).cpu().numpy()
        assert np.array_equal(y.view(np.uint64), ref.view(np.uint64)), m2


def test_premultiply_tiny_subnormal_and_signed_zero_parts(oz):
    """x~' = x w (the fma form of the complex product) for parts down to the subnormal
    range, signed zeros and exact zeros, against the oracle bit for bit, and the whole
    transform."""
    n = 1000
    rng = np.random.default_rng(20)
    mag = 10.0 ** rng.uniform(-322, -290, size=(2, n, 2))
    sgn = rng.choice([-1.0, 1.0], size=(2, n, 2))
    parts = mag * sgn
    parts[0, ::7, 0] = 0.0
    parts[0, ::11, 1] = -0.0
    parts[1, :5] = [[1e-300, -3e-310], [5e-324, -5e-324], [2.2250738585072014e-308, 0.0], [-0.0, 1e-320], [0.0, -0.0]]
    xs = np.empty((2, n), dtype=np.complex128)
    xs.real = parts[..., 0]
    xs.imag = parts[..., 1]
    y, plan = run_gpu(oz, xs, debug=True)
    assert plan.status() == oz.OK
    for b in range(2):
        yo, info = oracle_vs(xs[b], plan, trace={"xprime"})
        assert np.array_equal(plan.dump(oz.DUMP_XPRIME, b).view(np.uint64), info["xprime"].view(np.uint64)), b
        assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), b


def test_batch_mixed_distributions(oz):
    n = 2048
    xs = np.concatenate([synth.complex_signal(k, n, 7, phi=4.0) for k in
                         ("uniform", "phi", "gaussian", "spikes", "loguniform")])
    xs = np.concatenate([xs, np.zeros((1, n), complex)])
    d = np.zeros((1, n), complex); d[0, 0] = 1.0
    xs = np.concatenate([xs, d])
    for L in (1, 3):
        y, plan = run_gpu(oz, xs, L=L)
        for b in range(xs.shape[0]):
            yo, _ = oracle_vs(xs[b], plan)
            assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), (L, b)


@pytest.mark.parametrize("n", [1024, 1000])
def test_inverse_direction_and_roundtrip(oz, n):
    x = synth.complex_signal("uniform", n, 9, batch=3)
    yi, plan = run_gpu(oz, x, direction=oz.INVERSE)
    for b in range(3):
        yo, _ = oracle_vs(x[b], plan)
        assert np.array_equal(yi[b].view(np.uint64), yo.view(np.uint64))
    yf, _ = run_gpu(oz, x)
    back, _ = run_gpu(oz, yf, direction=oz.INVERSE)
    assert np.linalg.norm(back - x) / np.linalg.norm(x) <= 1e-15


@pytest.mark.parametrize("n", [1024, 1 << 14])
def test_accuracy_target(oz, n):
    x = synth.complex_signal("uniform", n, 1, batch=2)
    y, _ = run_gpu(oz, x)
    for b in range(2):
        hi, lo = oracle.fft_q(x[b]) if n > 4096 else oracle.dft_q(x[b])
        assert oracle.rel_l2_error(y[b], hi, lo) <= 1e-15


def test_transform_counts(oz):
    x = synth.complex_signal("phi", 4096, 1, batch=4, phi=0.0)
    _, p1 = run_gpu(oz, x, L=1)
    s1 = p1.stats()
    assert s1["ntt_forward_runtime"] == 4 * 12 and s1["ntt_inverse"] == 4 * 72
    assert s1["ntt_forward_plan"] == 12
    _, p3 = run_gpu(oz, x, L=3)
    s3 = p3.stats()
    assert s3["ntt_forward_runtime"] + s3["ntt_inverse"] == 4 * 52
    assert s3["ntt_forward_plan"] + (s3["ntt_forward_runtime"] + s3["ntt_inverse"]) // 4 == 64


def test_edge_cases_and_status(oz):
    # n = 1: y = x
    x = np.array([[1.5 - 2.0j]])
    y, plan = run_gpu(oz, x)
    assert np.array_equal(y, oracle_vs(x[0], plan)[0][None])
    # all-zero signal
    z = np.zeros((2, 64), complex)
    y, plan = run_gpu(oz, z)
    assert np.all(y == 0) and plan.status() == oz.OK
    # non-finite input -> status, plan stays usable
    bad = synth.complex_signal("uniform", 64, 3, batch=2)
    bad[1, 5] = np.nan
    y, plan = run_gpu(oz, bad)
    assert plan.status() == oz.ERR_NONFINITE
    assert plan.status() == oz.OK
    good = synth.complex_signal("uniform", 64, 3, batch=2)
    y = plan.execute(torch.from_numpy(good).cuda()).cpu().numpy()
    assert plan.status() == oz.OK
    assert np.array_equal(y[0].view(np.uint64), oracle_vs(good[0], plan)[0].view(np.uint64))
    # exponent overflow of sigma -> status
    big = np.full((1, 64), 1e307 + 0j)   # 2^(ceil(log2 max) + 53 - alpha) > 2^1023
    y, plan = run_gpu(oz, big)
    assert plan.status() == oz.ERR_RANGE
    # argument errors
    with pytest.raises(oz.OzfftError):
        oz.Plan(0, 1)
    with pytest.raises(oz.OzfftError):
        oz.Plan(8, 1, K=9)
    with pytest.raises(oz.OzfftError):
        oz.Plan(1 << 25, 1)


def test_in_place_and_host_buffers(oz):
    n, B = 4096, 3
    x = synth.complex_signal("gaussian", n, 4, batch=B)
    ref, plan = run_gpu(oz, x)
    xt = torch.from_numpy(x).cuda()
    plan.execute(xt, out=xt)
    assert np.array_equal(xt.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    plan.execute_host(hin, hout)
    assert np.array_equal(hout.numpy().view(np.uint64), ref.view(np.uint64))
    out = np.empty_like(x)
    plan.execute_host(np.ascontiguousarray(x), out)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("B", [8, 13, 28, 45])
def test_host_buffer_pipeline(oz, B):
    """Batches of 8 or more signals run the host-buffer path as a pipeline of parts
    (copies overlapping computation; from 28 signals the first and last parts are
    small): same bits as the device-buffer execution."""
    n = 3000
    x = synth.complex_signal("phi", n, 16, batch=B, phi=1.0)
    ref, plan = run_gpu(oz, x)
    for pinned in (True, False):
        hin = torch.from_numpy(x).pin_memory() if pinned else np.ascontiguousarray(x)
        hout = torch.empty_like(hin).pin_memory() if pinned else np.empty_like(x)
        for _ in range(2):
            plan.execute_host(hin, hout)
            got = hout.numpy() if pinned else hout
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (B, pinned)


def test_async_host_execution_pipelined(oz):
    """ozfft_execute_host_async: several calls in flight with different inputs
    and outputs (each call's copies overlapping its neighbours' computation),
    then ozfft_execute_host_wait; every output equals the synchronous call's,
    bit for bit, and the oracle's.  A synchronous call after asynchronous ones
    (and the reverse) shares the staging buffers safely."""
    n, B = 4096, 9
    xs = [synth.complex_signal(kind, n, 80 + i, batch=B) for i, kind in enumerate(("uniform", "phi", "gaussian"))]
    plan = oz.Plan(n, B)
    ref = []
    for x in xs:
        out = np.empty_like(x)
        plan.execute_host(x, out)
        ref.append(out)
    pins = [torch.from_numpy(x).pin_memory() for x in xs]
    outs = [torch.empty_like(t).pin_memory() for t in pins]
    for rep in range(2):
        for xin, o in zip(pins, outs):
            plan.execute_host_async(xin, o)
        plan.host_wait()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.numpy().view(np.uint64), r.view(np.uint64)), rep
    plan.execute_host_async(pins[0], outs[1])
    out = np.empty_like(xs[2])
    plan.execute_host(xs[2], out)                       # waits for the asynchronous call's copy out
    plan.host_wait()
    assert np.array_equal(out.view(np.uint64), ref[2].view(np.uint64))
    assert np.array_equal(outs[1].numpy().view(np.uint64), ref[0].view(np.uint64))
    for b in (0, B - 1):
        yo, _ = oracle.ozfft(xs[1][b])
        assert np.array_equal(ref[1][b].view(np.uint64), yo.view(np.uint64))
    assert plan.status() == oz.OK
