"""Pins of the oracle's modular layer (§3.3): moduli, roots, NTT, CRT.

Every expected value here comes from the paper's printed constants or from a
brute-force Python computation that shares nothing with the oracle's C code.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
PRIMES = [oracle.prime(i) for i in range(3)]


def is_prime(m):
    if m < 2:
        return False
    d = 2
    while d * d <= m:
        if m % d == 0:
            return False
        d += 1
    return True


def test_paper_primes():
    assert PRIMES[:2] == GOLD["primes"]["value"]
    for p in PRIMES:
        assert is_prime(p)
        assert p < 2 ** 31
    # 2-adic orders bound the NTT lengths: 2^24, 2^25, 2^27
    assert [((p - 1) & -(p - 1)).bit_length() - 1 for p in PRIMES] == [24, 25, 27]


@pytest.mark.parametrize("i", [0, 1, 2])
def test_generator_is_smallest_primitive_root(i):
    p = PRIMES[i]
    g = oracle.generator(p)
    m, fac, d = p - 1, [], 2
    while d * d <= m:
        if m % d == 0:
            fac.append(d)
            while m % d == 0:
                m //= d
        d += 1
    if m > 1:
        fac.append(m)

    def primitive(h):
        return all(pow(h, (p - 1) // f, p) != 1 for f in fac)

    assert primitive(g)
    assert not any(primitive(h) for h in range(2, g))


@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("lg", [1, 2, 5, 10, 18, 24])
def test_root_of_unity_order(i, lg):
    p, N = PRIMES[i], 1 << lg
    w = oracle.root(p, N)
    assert pow(w, N, p) == 1
    assert pow(w, N // 2, p) == p - 1  # order exactly N


def brute_ntt(a, p, w):
    N = len(a)
    return [sum(int(a[j]) * pow(w, j * k, p) for j in range(N)) % p for k in range(N)]


@pytest.mark.parametrize("i", [0, 1, 2])
def test_ntt_definition_brute_force(i):
    p = PRIMES[i]
    rng = random.Random(10 + i)
    for N in (1, 2, 4, 8, 16):
        a = np.array([rng.randrange(p) for _ in range(N)], dtype=np.uint32)
        w = pow(oracle.generator(p), (p - 1) // N, p)
        ref = brute_ntt(a, p, w)
        assert list(oracle.ntt(a, p, naive=True)) == ref
        assert list(oracle.ntt(a, p)) == ref
        winv = pow(w, p - 2, p)
        ninv = pow(N, p - 2, p)
        inv_ref = [x * ninv % p for x in brute_ntt(a, p, winv)]
        assert list(oracle.ntt(a, p, inverse=True)) == inv_ref


@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("N", [32, 256, 1024])
def test_fast_ntt_equals_naive(i, N):
    p = PRIMES[i]
    a = np.random.default_rng(N + i).integers(0, p, N, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(oracle.ntt(a, p), oracle.ntt(a, p, naive=True))
    assert np.array_equal(oracle.ntt(a, p, inverse=True), oracle.ntt(a, p, inverse=True, naive=True))


@pytest.mark.parametrize("i", [0, 1, 2])
def test_ntt_closed_forms(i):
    p = PRIMES[i]
    for N in (2, 64, 4096):
        delta = np.zeros(N, dtype=np.uint32); delta[0] = 1
        assert np.all(oracle.ntt(delta, p) == 1)
        ones = np.ones(N, dtype=np.uint32)
        expect = np.zeros(N, dtype=np.uint32); expect[0] = N % p
        assert np.array_equal(oracle.ntt(ones, p), expect)
        a = np.random.default_rng(N).integers(0, p, N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(oracle.ntt(oracle.ntt(a, p), p, inverse=True), a)


@pytest.mark.parametrize("i", [0, 1])
def test_convolution_theorem(i):
    """§3.3: INTT(NTT(x) . NTT(y)) is the cyclic convolution modulo p."""
    p = PRIMES[i]
    N = 16
    rng = random.Random(7 + i)
    x = [rng.randrange(p) for _ in range(N)]
    y = [rng.randrange(p) for _ in range(N)]
    brute = [sum(x[j] * y[(k - j) % N] for j in range(N)) % p for k in range(N)]
    X = oracle.ntt(np.array(x, dtype=np.uint32), p).astype(object)
    Y = oracle.ntt(np.array(y, dtype=np.uint32), p).astype(object)
    Z = np.array([(a * b) % p for a, b in zip(X, Y)], dtype=np.uint32)
    assert list(oracle.ntt(Z, p, inverse=True)) == brute


def test_exact_integer_convolution_via_two_primes():
    """§4.2: slices with |q| <= 2^alpha convolve exactly through NTT mod p0, p1 + CRT."""
    n = 64
    a = oracle.alpha(n, 1, 2)
    rng = random.Random(3)
    x = [rng.randint(-(2 ** a), 2 ** a) for _ in range(n)]
    y = [rng.randint(-(2 ** a), 2 ** a) for _ in range(n)]
    x[0] = y[0] = 2 ** a  # extreme entries
    exact = [sum(x[j] * y[(k - j) % n] for j in range(n)) for k in range(n)]
    res = []
    for p in PRIMES[:2]:
        X = oracle.ntt(np.array([v % p for v in x], dtype=np.uint32), p).astype(object)
        Y = oracle.ntt(np.array([v % p for v in y], dtype=np.uint32), p).astype(object)
        Z = np.array([(u * v) % p for u, v in zip(X, Y)], dtype=np.uint32)
        res.append(oracle.ntt(Z, p, inverse=True))
    assert oracle.garner(np.stack(res), 2) == exact


@pytest.mark.parametrize("nprimes", [2, 3])
def test_garner_equals_direct_crt(nprimes):
    """Garner (incremental form, §3.3) against the direct formula sum z_j P_j P_j^-1 mod P,
    followed by the symmetric remainder of Eq. (1)."""
    ps = PRIMES[:nprimes]
    P = 1
    for p in ps:
        P *= p
    rng = random.Random(nprimes)
    zs = [rng.randrange(-(P - 1) // 2, (P - 1) // 2 + 1) for _ in range(500)]
    zs += [0, 1, -1, (P - 1) // 2, -(P - 1) // 2]
    res = np.array([[z % p for z in zs] for p in ps], dtype=np.uint32)
    got = oracle.garner(res, nprimes)
    direct = []
    for j in range(len(zs)):
        acc = 0
        for i, p in enumerate(ps):
            Pi = P // p
            acc += int(res[i, j]) * Pi * pow(Pi, -1, p)
        acc %= P
        acc = acc - P * ((2 * acc + P) // (2 * P))  # a - P floor(a/P + 1/2)
        direct.append(acc)
    assert direct == zs
    assert got == zs
