"""Pins of the oracle's prime chain, NTT and ring products.

Each check compares the oracle with something computed independently of it:
an independent primality test, the first primes of each chain, the NTT's
O(N^2) definition and the schoolbook negacyclic product, both written here in
plain Python integers.
"""
import random

import numpy as np
import pytest

from oracle import lib
from oracle.bgv import Oracle
from tests.params import CHAIN36, CHAIN50


def trial_division_is_prime(n):
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def test_miller_rabin_small_range():
    L = lib()
    for n in range(0, 5000):
        assert bool(L.orc_is_prime(n)) == trial_division_is_prime(n), n


def test_miller_rabin_strong_pseudoprimes():
    # strong pseudoprimes to several small bases, and Carmichael numbers
    L = lib()
    for n in [2047, 1373653, 25326001, 3215031751, 2152302898747, 3474749660383,
              341550071728321, 3825123056546413051, 561, 1105, 1729, 2465]:
        assert not L.orc_is_prime(n), n
    for n in [2 ** 61 - 1, 2 ** 31 - 1, 1000000007, 998244353]:
        assert L.orc_is_prime(n), n


def test_chain36_first_primes_by_trial_division():
    o = Oracle(logN=6, p=17, L=4, K=1, **CHAIN36)
    # every listed prime is prime, = 1 mod U, in range, increasing, and no
    # prime of that form was skipped in between
    U, lo = CHAIN36["U"], CHAIN36["lo"]
    k = -(-(lo - 1) // U)
    expect = []
    while len(expect) < 5:
        q = k * U + 1
        if q >= lo and trial_division_is_prime(q):
            expect.append(q)
        k += 1
    assert o.primes == expect
    assert o.primes[0] == 34359771137


def test_chain50_first_primes_independent():
    sympy = pytest.importorskip("sympy")
    o = Oracle(logN=6, p=131, L=10, K=3, **CHAIN50)
    U, lo = CHAIN50["U"], CHAIN50["lo"]
    k = -(-(lo - 1) // U)
    expect = []
    while len(expect) < 13:
        q = k * U + 1
        if sympy.isprime(q):
            expect.append(q)
        k += 1
    assert o.primes == expect
    assert o.primes[0] == 564395044569089


@pytest.mark.parametrize("logN", [3, 5, 12])
def test_psi_is_primitive_2N_root(logN):
    o = Oracle(logN=logN, p=17, L=3, K=1, **CHAIN36)
    N = 1 << logN
    for i, q in enumerate(o.primes):
        psi = o.psi(i)
        assert pow(psi, N, q) == q - 1  # psi^N = -1  =>  order exactly 2N


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.mark.parametrize("logN", [1, 3, 4, 5])
def test_ntt_matches_definition_in_python(logN):
    o = Oracle(logN=logN, p=131, L=2, K=1, **CHAIN50)
    N = 1 << logN
    rnd = random.Random(logN)
    for i, q in enumerate(o.primes):
        psi = o.psi(i)
        a = [rnd.randrange(q) for _ in range(N)]
        want = [sum(a[n] * pow(psi, (2 * brv(k, logN) + 1) * n, q) for n in range(N)) % q for k in range(N)]
        got = o.ntt(i, np.array(a, dtype=np.uint64))
        assert [int(v) for v in got] == want
        assert [int(v) for v in o.ntt_direct(i, np.array(a, dtype=np.uint64))] == want


def schoolbook(a, b, q):
    N = len(a)
    out = [0] * N
    for x in range(N):
        for y in range(N):
            if x + y < N:
                out[x + y] += a[x] * b[y]
            else:
                out[x + y - N] -= a[x] * b[y]
    return [v % q for v in out]


@pytest.mark.parametrize("logN", [3, 4, 5, 6])
def test_polymul_matches_schoolbook(logN):
    o = Oracle(logN=logN, p=131, L=3, K=1, **CHAIN50)
    N = 1 << logN
    rnd = random.Random(100 + logN)
    for i, q in enumerate(o.primes):
        a = [rnd.randrange(q) for _ in range(N)]
        b = [rnd.randrange(q) for _ in range(N)]
        got = o.polymul(i, np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64))
        assert [int(v) for v in got] == schoolbook(a, b, q)


def test_polymul_36bit_chain_schoolbook():
    o = Oracle(logN=5, p=17, L=4, K=1, **CHAIN36)
    rnd = random.Random(7)
    for i, q in enumerate(o.primes):
        a = [rnd.randrange(q) for _ in range(32)]
        b = [rnd.choice([q - 1, 0, 1]) for _ in range(32)]
        got = o.polymul(i, np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64))
        assert [int(v) for v in got] == schoolbook(a, b, q)


@pytest.mark.parametrize("logN", [1, 6, 12, 14])
def test_intt_inverts_ntt(logN):
    o = Oracle(logN=logN, p=131, L=2, K=1, **CHAIN50)
    N = 1 << logN
    g = np.random.default_rng(logN)
    for i, q in enumerate(o.primes):
        a = g.integers(0, q, size=N, dtype=np.uint64)
        assert np.array_equal(o.intt(i, o.ntt(i, a)), a)


def test_polymul_int_and_automorphism_int():
    o = Oracle(logN=4, p=17, L=1, K=1, **CHAIN36)
    rnd = random.Random(3)
    a = [rnd.randint(-1, 1) for _ in range(16)]
    b = [rnd.randint(-1, 1) for _ in range(16)]
    got = o.polymul_int(np.array(a), np.array(b))
    big = 1 << 40
    assert [int(v) for v in got] == [((v + big // 2) % big) - big // 2 for v in schoolbook(a, b, big)]
    # sigma_g(a)(X) = a(X^g): compare with evaluation at a 2N-th root mod q
    q = o.primes[0]
    psi = o.psi(0)
    for g in (3, 5, 31):
        sa = [int(v) for v in o.automorphism_int(np.array(a), g)]
        for k in (1, 3, 7):
            x = pow(psi, k, q)
            lhs = sum(c * pow(x, n, q) for n, c in enumerate(sa)) % q
            rhs = sum(c * pow(x, (n * g), q) for n, c in enumerate(a)) % q
            assert lhs == rhs
