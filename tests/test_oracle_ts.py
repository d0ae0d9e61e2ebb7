"""Pins of the oracle's TS (triple-single) variant: TS conversion, TSAdd, TSSub
and TSMul against exact rational arithmetic, the error-free TS split of Alg. 6,
and the whole TS method (Alg. 4 around Alg. 8) against the binary128 DFT,
closed forms and the transform counts of §4.5."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2603_29129_gb300 import synth

rng = np.random.default_rng(11)


def rand_ts(N, spread):
    """Random TS numbers: x0 any binary32, |x1| <= ulp(x0)/2, |x2| <= ulp(x1)/2."""
    x0 = (rng.uniform(-1, 1, N) * np.exp2(rng.integers(-spread, spread + 1, N))).astype(np.float32)
    x1 = (rng.uniform(-0.5, 0.5, N) * np.spacing(np.abs(x0))).astype(np.float32)
    x2 = (rng.uniform(-0.5, 0.5, N) * np.spacing(np.abs(x1))).astype(np.float32)
    return np.stack([x0, x1, x2], axis=1)


def val(t):
    return sum(Fraction(float(w)) for w in t)


def test_ts_conversion_exact_and_nonoverlapping():
    # TS keeps the binary32 exponent range: exact while the third word stays normal
    x = rng.uniform(-1, 1, 5000) * np.exp2(rng.integers(-70, 100, 5000))
    x = np.concatenate([x, [0.0, 1.0, -3.0, np.pi, 2.0 ** -126, 1e30]])
    t = oracle.ts_from_double(x)
    for xi, ti in zip(x, t):
        assert val(ti) == Fraction(float(xi))
        for a, b in ((ti[0], ti[1]), (ti[1], ti[2])):
            assert b == 0 or abs(float(b)) <= np.spacing(np.float32(abs(a))) / 2
    assert np.array_equal(oracle.ts_to_double(t), x)


@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_ts_arithmetic_error_bound(op):
    """TS words carry 72 bits: every operation is within 2^-69 of the exact
    result (relative to the larger operand for add/sub, to the product for mul)."""
    worst = 0.0
    for spread in (0, 3, 30):
        a, b = rand_ts(1500, spread), rand_ts(1500, spread)
        r = oracle.ts_op(op, a, b)
        for i in range(len(a)):
            A, B = val(a[i]), val(b[i])
            ex = A + B if op == "add" else A - B if op == "sub" else A * B
            scale = abs(ex) if op == "mul" else max(abs(A), abs(B))
            if scale:
                worst = max(worst, float(abs(val(r[i]) - ex) / scale))
    assert worst <= 2.0 ** -69, worst


def test_ts_arithmetic_exact_cases():
    a = oracle.ts_from_double(np.array([3.0, 1.5, -7.25, 1e-3]))
    b = oracle.ts_from_double(np.array([5.0, 2.0, 7.25, 1e-3]))
    assert np.array_equal(oracle.ts_to_double(oracle.ts_op("add", a, b)), [8.0, 3.5, 0.0, 2e-3])
    assert np.array_equal(oracle.ts_to_double(oracle.ts_op("mul", a, b)), [15.0, 3.0, -52.5625, 1e-3 * 1e-3])
    z = oracle.ts_op("sub", a, a)
    assert np.all(z == 0)
    # a binary64 product is exact in 72 bits: TSMul of two converted doubles has it to 2^-69
    x = rng.uniform(-1, 1, 200)
    y = rng.uniform(-1, 1, 200)
    p = oracle.ts_op("mul", oracle.ts_from_double(x), oracle.ts_from_double(y))
    for i in range(200):
        ex = Fraction(float(x[i])) * Fraction(float(y[i]))
        assert abs(val(p[i]) - ex) <= abs(ex) * Fraction(1, 2 ** 69)


@pytest.mark.parametrize("alpha", [10, 20, 23])
def test_ts_split_error_free(alpha):
    """Alg. 6 run to mu = 0: sum_k q^(k) 2^-sexp[k] equals the TS value exactly,
    with |q^(k)| <= 2^alpha; the scales drop by at least alpha - 1 per level (the
    next residual's leading word absorbs the old second word, which may carry
    it one binade above the slice grid)."""
    for spread in (0, 20):
        v = np.ascontiguousarray(rand_ts(300, spread).T)
        q, sexp = oracle.ts_split(v, alpha, 0)
        assert np.abs(q).max() <= 2 ** alpha
        assert all(sexp[k + 1] - sexp[k] >= alpha - 1 for k in range(len(sexp) - 1))
        for j in range(v.shape[1]):
            rec = sum(Fraction(int(q[k, j])) * Fraction(2) ** (-sexp[k]) for k in range(len(sexp)))
            assert rec == val(v[:, j])


def test_ts_alpha_reading():
    for n in (1, 1000, 1 << 10, 1 << 18, 1 << 22):
        for L in (1, 3):
            assert oracle.alpha_ts(n, L) == min(oracle.alpha(n, L, 2), 23)


@pytest.mark.parametrize("n,kind", [(1024, "uniform"), (1000, "phi"), (777, "gaussian"), (2048, "spikes"),
                                    (4096, "loguniform")])
def test_ts_method_error_target(n, kind):
    x = synth.complex_signal(kind, n, 12, phi=4.0)[0]
    y, info = oracle.ozfft_ts(x)
    hi, lo = oracle.dft_q(x)
    assert oracle.rel_l2_error(y, hi, lo) <= 1e-15
    assert info["alpha"] == oracle.alpha_ts(n, 1)


def test_ts_method_closed_forms_and_directions():
    n = 256
    d = np.zeros(n, complex); d[0] = 1.0
    y, _ = oracle.ozfft_ts(d)
    assert np.max(np.abs(y - 1)) <= 1e-15
    tone = np.exp(2j * np.pi * 5 * np.arange(n) / n)
    y, _ = oracle.ozfft_ts(tone)
    e = np.zeros(n, complex); e[5] = n
    assert np.linalg.norm(y - e) / n <= 1e-14
    x = synth.complex_signal("uniform", 1000, 13)[0]
    y, _ = oracle.ozfft_ts(x)
    back, _ = oracle.ozfft_ts(y, direction=oracle.INVERSE)
    assert np.linalg.norm(back - x) / np.linalg.norm(x) <= 1e-15
    hi, lo = oracle.dft_q(x, direction=oracle.ADJOINT)
    assert oracle.rel_l2_error(oracle.ozfft_ts(x, direction=oracle.ADJOINT)[0], hi, lo) <= 1e-15


def test_ts_method_counts_and_accumulation():
    """No gaps (uniform input): 96 transforms (84 at run time) with L = 1 and 64
    (52) with L = 3, as the binary64 variant; L = 3 keeps the 1e-15 target."""
    x = synth.complex_signal("uniform", 1024, 14)[0]
    for L, tot in ((1, 96), (3, 64)):
        y, info = oracle.ozfft_ts(x, L=L)
        assert info["n_fwd_runtime"] + info["n_inv"] + info["n_fwd_plan"] == tot
        hi, lo = oracle.dft_q(x)
        assert oracle.rel_l2_error(y, hi, lo) <= 1e-15
