"""Host check of the lazy arithmetic of the NTT kernels (Harvey's lazy
butterflies, Sec. 2.2's radix-2 negacyclic NTT), emulated word for word:

- the forward butterfly t = Y w - qhat q with the cheaper Shoup quotient
  (qhat = ah wh + floor(ah wl / 2^32) + floor(al wh / 2^32), at most 2 below
  floor(Y ws / 2^64)), X <- X + t, Y <- X - t + 4q, with every intermediate an
  exact non-negative integer below 2^64 (no wrap), so the kernels' arithmetic
  mod 2^64 is exact;
- inputs anywhere in [0, 4q) (the lazy results of the fused conversions:
  Barrett without corrections in [0, 3q), chained Shoup products in [0, 4q))
  stay below (4s + 4) q after s stages and give, after the final reduction,
  the same transform as canonical inputs;
- the transform equals its definition A[k] = sum_i a_i psi^((2 brv(k) + 1) i)
  on a small ring, and the inverse butterflies (values kept in [0, 4q)) undo
  it, for a 50-bit prime of the comparison chain and the largest prime size the
  library accepts (just below 2^57)."""
import random

import pytest

M64 = (1 << 64) - 1


def is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_prime(bits, two_n):
    """Largest prime below 2^bits with q = 1 mod 2N."""
    q = ((1 << bits) - 1) // two_n * two_n + 1
    while not is_prime(q):
        q -= two_n
    return q


def root_2n(q, two_n):
    """A primitive 2N-th root of unity mod q."""
    for g in range(2, 1000):
        psi = pow(g, (q - 1) // two_n, q)
        if pow(psi, two_n // 2, q) == q - 1:
            return psi
    raise AssertionError("no root")


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def lazy_mul(a, w, ws, q):
    """The kernels' lazy Shoup product of any 64-bit a: result in [0, 4q)."""
    assert 0 <= a <= M64
    al, ah = a & 0xFFFFFFFF, a >> 32
    wl, wh = ws & 0xFFFFFFFF, ws >> 32
    qhat = ah * wh + ((ah * wl) >> 32) + ((al * wh) >> 32)
    exact = (a * ws) >> 64
    assert exact - 2 <= qhat <= exact
    r = a * w - qhat * q  # exact integer; the kernels compute it mod 2^64
    assert 0 <= r < 4 * q
    assert r == ((a * w) + qhat * ((1 << 64) - q)) & M64  # the multiply-add chain's form
    return r


def forward(a, q, psi, logn, track):
    """Forward negacyclic NTT, natural in, bit-reversed out, lazy butterflies;
    track[s] = max value after stage s."""
    n = 1 << logn
    x = list(a)
    q4 = 4 * q
    m, t, s = 1, n, 0
    while m < n:
        t //= 2
        for i in range(m):
            w = pow(psi, brv(m + i, logn), q)
            ws = (w << 64) // q
            for j in range(2 * i * t, 2 * i * t + t):
                tt = lazy_mul(x[j + t], w, ws, q)
                X = x[j]
                x[j] = X + tt
                x[j + t] = X - tt + q4
                assert 0 <= x[j + t] and x[j] <= M64 and x[j + t] <= M64
        track.append(max(x))
        m *= 2
        s += 1
    return x


def inverse(a, q, psi, logn):
    """Inverse (Gentleman-Sande) with values kept in [0, 4q), then N^-1."""
    n = 1 << logn
    x = list(a)
    q4 = 4 * q
    ipsi = pow(psi, -1, q)
    t, m = 1, n
    while m > 1:
        h = m // 2
        j1 = 0
        for i in range(h):
            w = pow(ipsi, brv(h + i, logn), q)
            ws = (w << 64) // q
            for j in range(j1, j1 + t):
                X, Y = x[j], x[j + t]
                assert X < q4 and Y < q4
                sm = X + Y
                sm = sm - q4 if sm >= q4 else sm
                x[j] = sm
                x[j + t] = lazy_mul(X - Y + q4, w, ws, q)
            j1 += 2 * t
        t *= 2
        m = h
    ninv = pow(n, -1, q)
    return [v * ninv % q for v in x]


@pytest.mark.parametrize("bits", [50, 57])
def test_lazy_inputs_give_the_canonical_transform(bits):
    logn = 10
    n = 1 << logn
    q = ntt_prime(bits, 2 * n)
    assert q < (1 << 57) and q.bit_length() == bits
    psi = root_2n(q, 2 * n)
    rnd = random.Random(bits)
    canon = [rnd.randrange(q) for _ in range(n)]
    canon[:8] = [q - 1] * 8
    # lazy representatives in [0, 4q): x + k q, including the top of the range
    lazy = [v + rnd.randrange(4) * q for v in canon]
    lazy[:8] = [q - 1 + 3 * q] * 8
    t1, t2 = [], []
    out_c = [v % q for v in forward(canon, q, psi, logn, t1)]
    out_l = [v % q for v in forward(lazy, q, psi, logn, t2)]
    assert out_l == out_c
    for s, mx in enumerate(t2, start=1):
        assert mx < (4 * s + 4) * q  # the bound the kernels rely on
    assert max(t2) < (1 << 63)
    # the inverse undoes it (inputs canonical, as the kernels hand them over)
    assert inverse(out_c, q, psi, logn) == canon


@pytest.mark.parametrize("bits", [50, 57])
def test_transform_matches_definition_small_ring(bits):
    logn = 5
    n = 1 << logn
    q = ntt_prime(bits, 2 * n)
    psi = root_2n(q, 2 * n)
    rnd = random.Random(7 + bits)
    a = [rnd.randrange(4 * q) for _ in range(n)]
    got = [v % q for v in forward(a, q, psi, logn, [])]
    want = [sum(a[i] * pow(psi, (2 * brv(k, logn) + 1) * i, q) for i in range(n)) % q for k in range(n)]
    assert got == want


def test_fifteen_stages_at_the_largest_prime_size():
    """The largest ring (N = 2^15, 15 stages) at the largest prime size the
    library accepts, from inputs at the top of the lazy range (4q - 1 and
    random values in [0, 4q)): every value stays below (4s + 4) q <= 64 q <
    2^63 and the outputs equal the canonical inputs' transform."""
    logn = 15
    n = 1 << logn
    q = ntt_prime(57, 2 * n)
    psi = root_2n(q, 2 * n)
    rnd = random.Random(15)
    lazy = [4 * q - 1 if i % 3 == 0 else rnd.randrange(4 * q) for i in range(n)]
    track = []
    out = [v % q for v in forward(lazy, q, psi, logn, track)]
    assert all(mx < (4 * s + 4) * q for s, mx in enumerate(track, start=1))
    assert max(track) < 64 * q < (1 << 63)
    assert out == [v % q for v in forward([v % q for v in lazy], q, psi, logn, [])]
