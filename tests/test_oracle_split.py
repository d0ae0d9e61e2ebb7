"""Pins of the oracle's Ozaki layer: alpha (§4.2, §4.4), the split (Alg. 3), the
Alg. 8 flush schedule, and the double-word accumulation pieces."""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2603_29129_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_alpha_printed_values():
    g = GOLD
    assert oracle.alpha(2 ** 20, 1, 2) == g["alpha_two_prime_n2e20"]["value"]
    assert oracle.alpha(2 ** 17, 1, 2) == g["alpha_two_prime_L1_n2e17"]["value"]
    assert oracle.alpha(2 ** 17, 3, 2) == g["alpha_two_prime_L3_n2e17"]["value"]
    assert oracle.alpha(2 ** 18, 1, 2) == g["alpha_two_prime_L1_n2e18"]["value"]
    assert oracle.alpha(2 ** 18, 3, 2) == g["alpha_two_prime_L3_n2e18"]["value"]
    # §4.2: a single modulus gives only slightly more than the original Ozaki
    # scheme's fp32 alpha floor((24 - log2 n)/2) = 2 at n = 2^20
    orig = (24 - 20) // 2
    assert orig == g["alpha_fp32_original_ozaki_n2e20"]["value"]
    assert orig < oracle.alpha(2 ** 20, 1, 1) < oracle.alpha(2 ** 20, 1, 2)


@pytest.mark.parametrize("nprimes", [1, 2, 3])
@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_alpha_is_largest_exact_bound(nprimes, L):
    """alpha = max a with L n 2^(2a) < P/2, the integer form of
    floor((log2(P/2) - log2(L n))/2) (§4.4)."""
    P = 1
    for i in range(nprimes):
        P *= oracle.prime(i)
    for lg in range(0, 25):
        n = 1 << lg
        a = oracle.alpha(n, L, nprimes)
        if a < 0:
            assert 2 * L * n >= P
            continue
        a_cap = min(a, 52)
        assert 2 * L * n * 4 ** a_cap < P
        if a < 52:
            assert 2 * L * n * 4 ** (a + 1) >= P
        fl = math.floor((math.log2(P / 2) - math.log2(L * n)) / 2)
        assert a == min(fl, 52)


def split_props(v, alpha, K):
    sl, q, se, st = oracle.split(v, alpha, K)
    assert st == 0
    rho = 53 - alpha
    r = [Fraction(float(t)) for t in v]
    for k in range(len(se)):
        mu = max(abs(t) for t in r)
        assert mu > 0
        e = 0  # exact ceil(log2(mu)) on a Fraction
        while Fraction(2) ** e < mu:
            e += 1
        while Fraction(2) ** (e - 1) >= mu:
            e -= 1
        sigma = Fraction(2) ** (e + rho)
        unit = sigma * Fraction(1, 2 ** 53)  # u sigma
        assert se[k] == alpha - e  # c = (u sigma)^-1 = 2^(alpha - e)
        for j, t in enumerate(sl[k]):
            ft = Fraction(float(t))
            assert ft / unit == q[k][j] and abs(q[k][j]) <= 2 ** alpha  # split condition (§3.4)
            r[j] -= ft
    return sl, q, se, r


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("alpha", [21, 25, 40])
def test_split_is_error_free_with_K_inf(seed, alpha):
    v = synth.complex_signal("phi", 64, seed, phi=4.0).real[0]
    sl, q, se, r = split_props(v, alpha, 0)
    assert all(t == 0 for t in r)  # sum of slices == v exactly
    # split count bound (§3.4), u = 2^-53
    nz = np.abs(v[v != 0])
    bound = math.ceil((math.log2(nz.max()) - math.log2(nz.min()) + 53 - 1) / (alpha - 1))
    assert len(se) <= bound


def test_split_truncates_at_K_and_scale_invariance():
    v = synth.uniform(5, 128)
    sl, q, se, r = split_props(v, 21, 3)
    assert len(se) == 3
    # remainder after 3 levels is below u sigma of level 2
    assert max(abs(t) for t in r) <= Fraction(2) ** (-int(se[2]))
    for m in (-7, 1, 30):
        _, q2, se2, _ = oracle.split(np.ldexp(v, m), 21, 3)
        assert np.array_equal(q2, q)
        assert np.array_equal(se2, se - m)


def test_split_special_cases():
    # constant vector: one level, q = 2^alpha (mu = 1 exactly a power of two)
    sl, q, se, st = oracle.split(np.ones(8), 21, 0)
    assert st == 0 and len(se) == 1 and np.all(q[0] == 2 ** 21) and se[0] == 21
    # zero vector: no level
    sl, q, se, st = oracle.split(np.zeros(8), 21, 0)
    assert st == 0 and len(se) == 0
    # non-finite input is rejected
    assert oracle.split(np.array([1.0, np.nan]), 21, 3)[3] == oracle.ERR_NONFINITE
    # huge magnitude overflows sigma = 2^(e + rho)
    assert oracle.split(np.array([1e300, 1.0]), 21, 3)[3] == oracle.ERR_RANGE


def no_gap(k0, k, alpha):
    return np.array([k0 + alpha * i for i in range(k)], dtype=np.int32)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_schedule_counts_match_paper_formulas(K):
    """§4.5: with kx = ky = K and no gaps, a real convolution needs K^2 inverse
    NTT pairs at L = 1 and 2K - 1 at L >= K."""
    sx, sy = no_gap(24, K, 21), no_gap(25, K, 21)
    assert len(oracle.schedule(sx, sy, 1)) == K * K
    assert len(oracle.schedule(sx, sy, K)) == 2 * K - 1
    assert len(oracle.schedule(sx, sy, K + 3)) == 2 * K - 1
    # totals of §4.5 with 2 primes and 4 real convolutions
    fwd = 8 * K
    assert fwd + 2 * 4 * K * K == 8 * K + 8 * K * K
    assert fwd + 2 * 4 * (2 * K - 1) == 24 * K - 8


def test_schedule_structure_brute_force():
    rng = random.Random(11)
    for trial in range(300):
        kx, ky = rng.randint(1, 6), rng.randint(1, 6)
        sx = np.array(sorted(rng.sample(range(0, 200), kx)), dtype=np.int32)
        sy = np.array(sorted(rng.sample(range(0, 200), ky)), dtype=np.int32)
        if rng.random() < 0.5:
            sx, sy = no_gap(3, kx, 20), no_gap(5, ky, 20)
        L = rng.randint(1, 5)
        groups = oracle.schedule(sx, sy, L)
        seen = []
        for S, pairs in groups:
            assert 1 <= len(pairs) <= L
            assert all(sx[s] + sy[t] == S for s, t in pairs)
            seen += pairs
        # every pair once, in Alg. 8's order: k = s + t descending, s ascending
        order = [(s, k - s) for k in range(kx + ky - 2, -1, -1)
                 for s in range(max(0, k - ky + 1), min(kx - 1, k) + 1)]
        assert seen == order
        # consecutive groups split only on a full group or a scale change
        for (S0, p0), (S1, p1) in zip(groups, groups[1:]):
            assert len(p0) == L or S0 != S1


def test_exact_sum_rounds_the_exact_rational():
    """Reading R7: round-to-nearest-even of the exact sum, checked with Fractions
    (Fraction -> float is correctly rounded), including ties, cancellation,
    huge scale spreads and subnormal results."""
    rng = random.Random(6)
    P3 = oracle.prime(0) * oracle.prime(1) * oracle.prime(2)
    cases = []
    for _ in range(400):
        k = rng.randint(1, 12)
        zs = [rng.randrange(-(P3 // 2), P3 // 2) for _ in range(k)]
        base = rng.randint(-200, 1100)
        Ss = [base + rng.choice([0, 21, 42, 63, 84, rng.randint(-60, 600)]) for _ in range(k)]
        cases.append((zs, Ss, [rng.choice([1, -1]) for _ in range(k)]))
    # exact ties: 2^53 + 1 (a midpoint) rounds to even, and a tiny term breaks the tie
    cases.append(([2 ** 53 + 1], [0], [1]))
    cases.append(([2 ** 53 + 1, 1], [0, 700], [1, 1]))
    cases.append(([2 ** 53 + 3], [0], [1]))
    cases.append(([5, 5], [0, 0], [1, -1]))          # exact cancellation -> +0
    cases.append(([3], [1076], [1]))                   # subnormal with rounding
    cases.append(([1 << 60, -(1 << 60) + 1], [10, 10], [1, 1]))
    for zs, Ss, sg in cases:
        exact = sum(Fraction(s * z) / Fraction(2) ** S for z, S, s in zip(zs, Ss, sg))
        got = oracle.exact_sum(zs, Ss, sg)
        assert got == float(exact), (zs, Ss, sg)
        if exact == 0:
            assert np.copysign(1.0, got) == 1.0
