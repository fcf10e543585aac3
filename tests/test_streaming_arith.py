"""Host check of the streaming kernels' 64-bit scalar products, emulated word
for word: the PS leaves and scalar multiples (sum_t c_t x_t with centred
scalars |c_t| <= p/2, the circuits of Sec. 2.1) are formed as
sum_t (c_t < 0 ? q - x_t : x_t) |c_t| in 64-bit arithmetic when
q_max sum_t |c_t| < 2^64, then reduced by v - floor(v floor(2^64/q) / 2^64) q
and one correction.  Checked against the exact sum mod q, including the
extreme operands (x = 0 and x = q - 1, the largest scalars, eight terms), for
the plaintext primes and prime sizes the library runs."""
import random

import pytest

M64 = (1 << 64) - 1


def reduce64(v, q):
    """The kernels' reduction of any 64-bit v to [0, q)."""
    assert 0 <= v <= M64
    mu = (1 << 64) // q
    r = v - ((v * mu) >> 64) * q
    assert 0 <= r < 2 * q
    return r - q if r >= q else r


def scaled(a, k, q):
    """One term: a k mod q as a 64-bit product of non-negative words."""
    r = (q - a if k < 0 else a) * abs(k)
    assert r <= q * abs(k)
    return r


def small_form_applies(q_max, ks):
    return sum(abs(k) for k in ks) * q_max < (1 << 64)


@pytest.mark.parametrize("p,bits", [(17, 36), (131, 50), (257, 50), (257, 57)])
def test_lincomb_64bit_form_equals_exact(p, bits):
    rnd = random.Random(p * 100 + bits)
    q = (1 << bits) - rnd.randrange(1 << 20) * 2 - 1  # any odd modulus of that size
    half = p // 2
    checked = 0
    for trial in range(2000):
        n = rnd.randint(1, 8)
        ks = [rnd.randint(-half, half) for _ in range(n)]
        if trial % 7 == 0:
            ks = [rnd.choice((-half, half)) for _ in range(8)]
        xs = [rnd.choice((0, q - 1, rnd.randrange(q))) for _ in range(len(ks))]
        want = sum(x * k for x, k in zip(xs, ks)) % q
        if not small_form_applies(q, ks):
            continue  # the kernels take the 128-bit form
        acc = 0
        for x, k in zip(xs, ks):
            acc += scaled(x, k, q)
        assert acc <= M64
        assert reduce64(acc, q) == want
        checked += 1
    assert checked > 100


def test_small_form_covers_the_benchmark_chains():
    """Eight terms with the largest centred scalars of every plaintext prime
    stay in 64 bits for the 50-bit chains; near 2^57 the 128-bit form is
    taken for the largest primes (the host decision)."""
    for p in (17, 131, 257):
        assert small_form_applies((1 << 50) - 1, [p // 2] * 8)
    assert not small_form_applies((1 << 57) - 1, [257 // 2] * 8)
