"""Pins of the slot structure: decode(encode) = id, ring products are
slot-wise products, sigma_5 / sigma_{-1} permute slots, and n_s equals
N / ord_{2N}(p) by brute force."""
import random

import numpy as np
import pytest

from oracle.encoding import SlotStructure


def order_mod(p, m):
    o, x = 1, p % m
    while x != 1:
        x = x * p % m
        o += 1
    return o


def negacyclic_mul_mod_p(a, b, p):
    N = len(a)
    out = [0] * N
    for x in range(N):
        if a[x] == 0:
            continue
        for y in range(N):
            if b[y] == 0:
                continue
            if x + y < N:
                out[x + y] += a[x] * b[y]
            else:
                out[x + y - N] -= a[x] * b[y]
    return [v % p for v in out]


@pytest.mark.parametrize("p,logN", [(17, 12), (131, 14), (257, 15), (17, 13), (257, 13), (131, 12), (5, 8)])
def test_slot_count(p, logN):
    N = 1 << logN
    ss = SlotStructure(p, N)
    assert ss.ns == N // order_mod(p, 2 * N)


@pytest.mark.parametrize("p", [5, 17, 131, 257])
def test_roundtrip_and_homomorphism(p):
    N = 512
    ss = SlotStructure(p, N)
    rnd = random.Random(p)
    for _ in range(3):
        v = [rnd.randrange(p) for _ in range(ss.ns)]
        w = [rnd.randrange(p) for _ in range(ss.ns)]
        m, n = ss.encode(v), ss.encode(w)
        assert ss.decode(m) == v
        prod = negacyclic_mul_mod_p([int(x) for x in m], [int(x) for x in n], p)
        assert ss.decode(prod) == [(a * b) % p for a, b in zip(v, w)]
        s = [(int(a) + int(b)) % p for a, b in zip(m, n)]
        assert ss.decode(s) == [(a + b) % p for a, b in zip(v, w)]


def automorph(m, g):
    N = len(m)
    out = [0] * N
    for n, c in enumerate(m):
        e = (n * g) % (2 * N)
        if e < N:
            out[e] += int(c)
        else:
            out[e - N] -= int(c)
    return out


@pytest.mark.parametrize("p", [17, 257])
def test_rotations_linear(p):
    N = 1024
    ss = SlotStructure(p, N)
    cols = ss.M // 2
    v = list(range(1, ss.ns + 1))
    m = ss.encode(v)
    r5 = ss.decode([x % p for x in automorph(m, 5)])
    want = [v[r * cols + (c + 1) % cols] for r in range(2) for c in range(cols)]
    assert r5 == want
    rs = ss.decode([x % p for x in automorph(m, 2 * N - 1)])
    assert rs == v[cols:] + v[:cols]


def test_decode_rejects_non_subring():
    ss = SlotStructure(17, 64)
    m = ss.encode([1] * ss.ns)
    m[1] = 3
    with pytest.raises(ValueError):
        ss.decode(m)
