"""Pins of the oracle's transform layer: the chirp table (Alg. 1), the binary128
DFT reference, and the whole method (Alg. 1 around Alg. 8, §4.5) against DFT
closed forms, Parseval, the error target and the paper's transform counts."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2603_29129_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --- chirp table ---------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 8, 100, 1000, 1024, 4097])
def test_chirp_correctly_rounded(n):
    """w(j) = exp(-i pi j^2 / n) rounded to nearest (reading of §4.2's correctly
    rounded table assumption), checked with 200-bit mpmath."""
    mpmath = pytest.importorskip("mpmath")
    w = oracle.chirp(n)
    mpmath.mp.prec = 200
    idx = range(n) if n <= 1100 else list(range(0, n, 7)) + [n - 1]
    for j in idx:
        t = mpmath.mpf((j * j) % (2 * n)) / n
        assert w[j].real == float(mpmath.cospi(t))
        assert w[j].imag == float(-mpmath.sinpi(t))


def test_chirp_exact_angles():
    # r/n in {0, 1/2, 1, 3/2} give exact 0 / +-1 components
    w = oracle.chirp(8)  # j^2 mod 16: 0 1 4 9 0 9 4 1
    assert w[0] == 1 and w[4] == 1
    assert w[2] == -1j and w[6] == -1j  # r = 4: exp(-i pi/2)
    s = oracle.sincospi_q(1, 1)  # sin(pi), cos(pi)
    assert s[0] == 0 and s[2] == -1


# --- binary128 reference ---------------------------------------------------------
def test_dft_q_closed_forms():
    n = 256
    d = np.zeros(n, complex); d[0] = 1
    hi, lo = oracle.dft_q(d)
    assert np.all(hi == 1) and np.all(lo == 0)
    c = np.full(n, 0.75 - 0.5j)
    hi, lo = oracle.dft_q(c)
    assert hi[0] == n * (0.75 - 0.5j)
    assert np.max(np.abs(hi[1:])) < 1e-30
    m = 37
    tone = np.exp(2j * np.pi * m * np.arange(n) / n)
    hi, lo = oracle.dft_q(tone)
    expect = np.zeros(n, complex); expect[m] = n
    assert np.max(np.abs(hi - expect)) < 1e-12  # tone itself is only binary64-accurate


@pytest.mark.parametrize("n", [16, 1024])
def test_dft_q_against_numpy_and_fft_q(n):
    x = synth.complex_signal("uniform", n, 9)[0]
    hi, lo = oracle.dft_q(x)
    ref = np.fft.fft(x)
    assert np.max(np.abs(hi - ref)) / np.max(np.abs(hi)) < 1e-14
    fhi, flo = oracle.fft_q(x)
    assert np.max(np.abs((fhi - hi) + (flo - lo))) / np.max(np.abs(hi)) < 1e-30
    ihi, ilo = oracle.dft_q(hi, direction=oracle.INVERSE)
    assert np.max(np.abs(ihi - x)) < 1e-15
    # Parseval
    assert abs(np.sum(np.abs(hi) ** 2) - n * np.sum(np.abs(x) ** 2)) / (n * np.sum(np.abs(x) ** 2)) < 1e-15


def test_dft_q_bins_subset():
    n = 3000
    x = synth.complex_signal("gaussian", n, 2)[0]
    bins = np.array([0, 1, 17, 2999], dtype=np.int64)
    hi, lo = oracle.dft_q(x, bins=bins)
    ref = np.fft.fft(x)[bins]
    assert np.max(np.abs(hi - ref)) / np.max(np.abs(ref)) < 1e-13


# --- the whole method -------------------------------------------------------------
def err_vs_q(y, x, direction=oracle.FORWARD):
    hi, lo = oracle.dft_q(x, direction=direction)
    return oracle.rel_l2_error(y, hi, lo)


CASES = [  # (n, N, K, L, nprimes)
    (1024, 2048, 3, 1, 2), (1024, 1024, 3, 1, 2), (1024, 2048, 3, 1, 3),
    (1024, 1024, 0, 1, 2), (1024, 1024, 3, 3, 2), (1000, 2048, 3, 1, 2), (777, 2048, 3, 3, 3),
]


@pytest.mark.parametrize("case", CASES)
def test_method_error_target(case):
    n, N, K, L, P = case
    x = synth.complex_signal("uniform", n, 1)[0]
    y, info = oracle.ozfft(x, N=N, K=K, L=L, nprimes=P)
    assert err_vs_q(y, x) <= 1e-15


@pytest.mark.parametrize("kind", ["phi", "loguniform", "spikes", "gaussian"])
def test_method_error_distributions(kind):
    n = 512
    x = synth.complex_signal(kind, n, 4, phi=4.0)[0]
    y, _ = oracle.ozfft(x, K=3, L=1)
    assert err_vs_q(y, x) <= 1e-15


def test_method_closed_forms():
    n = 256
    d = np.zeros(n, complex); d[0] = 1.0
    y, _ = oracle.ozfft(d)
    assert np.max(np.abs(y - 1)) <= 1e-15
    c = 0.3 - 0.7j
    y, _ = oracle.ozfft(np.full(n, c))
    assert abs(y[0] - n * c) <= 1e-15 * n and np.max(np.abs(y[1:])) <= 1e-15 * n
    m = 5
    tone = np.exp(2j * np.pi * m * np.arange(n) / n)
    y, _ = oracle.ozfft(tone)
    e = np.zeros(n, complex); e[m] = n
    assert np.linalg.norm(y - e) / n <= 1e-14
    x = synth.complex_signal("gaussian", n, 6)[0]
    y, _ = oracle.ozfft(x)
    assert abs(np.vdot(y, y).real - n * np.vdot(x, x).real) <= 1e-14 * n * np.vdot(x, x).real
    # shift theorem: DFT(x(j-1)) = w_n^k DFT(x)
    ys, _ = oracle.ozfft(np.roll(x, 1))
    ramp = np.exp(-2j * np.pi * np.arange(n) / n)
    assert np.linalg.norm(ys - ramp * y) / np.linalg.norm(y) <= 1e-14
    # linearity
    x2 = synth.complex_signal("uniform", n, 7)[0]
    y2, _ = oracle.ozfft(x2)
    y12, _ = oracle.ozfft(x + 2 * x2)
    assert np.linalg.norm(y12 - (y + 2 * y2)) / np.linalg.norm(y12) <= 1e-14


def test_method_inverse_and_roundtrip():
    n = 1024
    x = synth.complex_signal("uniform", n, 3)[0]
    y, _ = oracle.ozfft(x)
    xi, _ = oracle.ozfft(y, direction=oracle.INVERSE)
    assert np.linalg.norm(xi - x) / np.linalg.norm(x) <= 1e-15
    yi, _ = oracle.ozfft(x, direction=oracle.INVERSE)
    assert err_vs_q(yi, x, oracle.INVERSE) <= 1e-15


def test_dft_q_adjoint_directions():
    """The adjoint directions of the binary128 DFT: F^H x (sign +, no division)
    and (1/n) F x, against closed forms on a delta and against numpy's FFT."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    n, j0 = 12, 5
    d = np.zeros(n, complex); d[j0] = 1.0
    ang = [mpmath.mpf(2 * (j0 * k % n)) / n for k in range(n)]       # exp(+-i pi ang)
    up = np.array([complex(float(mpmath.cospi(a)), float(mpmath.sinpi(a))) for a in ang])
    hi, _ = oracle.dft_q(d, direction=oracle.ADJOINT)
    assert np.max(np.abs(hi - up)) <= 2 ** -53
    hi, _ = oracle.dft_q(d, direction=oracle.INVERSE_ADJOINT)
    down = np.array([complex(float(mpmath.cospi(a) / n), float(-mpmath.sinpi(a) / n)) for a in ang])
    assert np.max(np.abs(hi - down)) <= 2 ** -53 / n
    x = synth.complex_signal("gaussian", 64, 8)[0]
    assert np.allclose(oracle.dft_q(x, oracle.ADJOINT)[0], 64 * np.fft.ifft(x), rtol=0, atol=1e-13)
    assert np.allclose(oracle.fft_q(x, oracle.ADJOINT)[0], 64 * np.fft.ifft(x), rtol=0, atol=1e-13)
    assert np.allclose(oracle.dft_q(x, oracle.INVERSE_ADJOINT)[0], np.fft.fft(x) / 64, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [256, 1000])
def test_method_adjoints(n):
    """<F x, g> = <x, F^H g> and <F^-1 x, g> = <x, (1/n) F g> for the method's
    transforms; each adjoint also meets the 1e-15 target against binary128."""
    x = synth.complex_signal("uniform", n, 21)[0]
    g = synth.complex_signal("gaussian", n, 22)[0]
    fx, _ = oracle.ozfft(x)
    ahg, _ = oracle.ozfft(g, direction=oracle.ADJOINT)
    lhs, rhs = np.vdot(g, fx), np.vdot(ahg, x)
    assert abs(lhs - rhs) <= 1e-14 * np.linalg.norm(fx) * np.linalg.norm(g)
    ix, _ = oracle.ozfft(x, direction=oracle.INVERSE)
    aig, _ = oracle.ozfft(g, direction=oracle.INVERSE_ADJOINT)
    assert abs(np.vdot(g, ix) - np.vdot(aig, x)) <= 1e-14 * np.linalg.norm(ix) * np.linalg.norm(g)
    assert err_vs_q(ahg, g, oracle.ADJOINT) <= 1e-15
    assert err_vs_q(aig, g, oracle.INVERSE_ADJOINT) <= 1e-15
    # the adjoint is the conjugated forward transform of the conjugate, exactly
    cf, _ = oracle.ozfft(np.conj(g))
    assert np.array_equal(np.conj(cf), ahg)


def test_padding_invariance_power_of_two():
    """Reading D3: for power-of-two n the cyclic length N = n and the padded
    N = 2n give bit-identical results."""
    for n in (8, 1024):
        x = synth.complex_signal("phi", n, 5, phi=1.0)[0]
        a, ia = oracle.ozfft(x, N=n, trace={"yprime"})
        b, ib = oracle.ozfft(x, N=2 * n, trace={"yprime"})
        assert np.array_equal(a, b) and np.array_equal(ia["yprime"], ib["yprime"])


def test_transform_counts_paper():
    """§5.3-5.5: K = 3 gives 96 transforms (84 at run time) with L = 1 and 64
    (52 at run time) with L = 3 when the splits have no gaps."""
    g = GOLD
    x = synth.complex_signal("phi", 1024, 1, phi=0.0)[0]
    _, i1 = oracle.ozfft(x, K=3, L=1)
    _, i3 = oracle.ozfft(x, K=3, L=3)
    assert i1["ntt_total"] == g["ntt_total_K3_L1"]["value"] and i1["ntt_runtime"] == 84
    assert i3["ntt_total"] == g["ntt_total_K3_L3_narrow"]["value"]
    assert i3["ntt_runtime"] == g["ntt_runtime_K3_L3"]["value"]


def test_transform_count_trends():
    """§5.2/§5.4 trends: K = inf counts grow with phi; (3,3) counts stay within
    [64, 96].  (The paper's 268/196/80 maxima are for TS precision and are not
    expected here: binary64 carries 53 bits, TS 72.)"""
    counts = {}
    for phi in (0.0, 4.0):
        x = synth.complex_signal("phi", 2048, 2, phi=phi)[0]
        _, inf = oracle.ozfft(x, K=0, L=1)
        _, k33 = oracle.ozfft(x, K=3, L=3)
        counts[phi] = inf["ntt_total"]
        assert 64 <= k33["ntt_total"] <= 96
    assert counts[4.0] > counts[0.0]


def test_accumulation_is_the_rounded_exact_sum():
    """Reading R7: y' is the exact sum of the rescaled CRT integers of every
    flush group (RR - II, IR + RI), rounded once to nearest; recomputed here with
    rational arithmetic from the oracle's CRT integers and group scales."""
    n = 128
    x = synth.complex_signal("phi", n, 8, phi=1.0)[0]
    y, info = oracle.ozfft(x, K=3, L=1, trace={"zcrt", "groups", "yprime"})
    z = info["zcrt"]
    gS = info["gS"]
    exact = [[Fraction(0)] * n, [Fraction(0)] * n]
    sign = [1, -1, 1, 1]
    part = [0, 0, 1, 1]
    for c in range(4):
        for g in range(info["ngroups"][c]):
            scale = Fraction(1, 2 ** int(gS[c, g])) if gS[c, g] >= 0 else Fraction(2 ** int(-gS[c, g]))
            for j in range(n):
                v = int(np.uint64(z[c, g, j, 0])) + (int(z[c, g, j, 1]) << 64)
                exact[part[c]][j] += sign[c] * v * scale
    yp = info["yprime"]
    for j in range(n):
        assert yp[j].real == float(exact[0][j]) and yp[j].imag == float(exact[1][j])


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def test_double_double_accumulation_within_one_ulp():
    """The paper accumulates the rescaled CRT integers with a compensated (TSAdd) sum
    in flush order; reading R7 rounds their exact sum once.  A fixed-order double-double
    accumulation of the same terms (z' split exactly into hi + lo, TwoSum per term in
    the order RR, II, IR, RI) lands within 1 ulp of the exact rounding everywhere and
    on it for nearly every element."""
    n = 512
    x = synth.complex_signal("phi", n, 21, phi=1.0)[0]
    _, info = oracle.ozfft(x, K=3, L=1, trace={"zcrt", "groups", "yprime"})
    z, gS, yp = info["zcrt"], info["gS"], info["yprime"]
    sign = [1, -1, 1, 1]
    part = [0, 0, 1, 1]
    acc = [[(0.0, 0.0)] * n, [(0.0, 0.0)] * n]
    for c in range(4):
        for g in range(info["ngroups"][c]):
            S = int(gS[c, g])
            for j in range(n):
                v = sign[c] * (int(np.uint64(z[c, g, j, 0])) + (int(z[c, g, j, 1]) << 64))
                hi = float(v)
                lo = float(v - int(hi))                      # exact: |v - hi| < 2^10
                s_, e_ = acc[part[c]][j]
                for t in (math.ldexp(hi, -S), math.ldexp(lo, -S)):
                    s_, err = _two_sum(s_, t)
                    e_ += err
                acc[part[c]][j] = (s_, e_)
    equal = 0
    for j in range(n):
        for p, ref in ((0, yp[j].real), (1, yp[j].imag)):
            got = acc[p][j][0] + acc[p][j][1]
            assert got == ref or got in (np.nextafter(ref, np.inf), np.nextafter(ref, -np.inf)), (j, p, got, ref)
            equal += got == ref
    assert equal >= 0.99 * 2 * n, equal


def test_method_argument_errors():
    x = np.ones(8, complex)
    with pytest.raises(oracle.OracleError):
        oracle.ozfft(x, N=12)  # not a power of two
    with pytest.raises(oracle.OracleError):
        oracle.ozfft(np.ones(6, complex), N=8)  # N < 2n-1 and N != n
    with pytest.raises(oracle.OracleError):
        oracle.ozfft(np.array([np.inf, 0], complex))
