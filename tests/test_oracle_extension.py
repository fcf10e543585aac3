"""Pins of the F_{p^d}-slot encoding and of digit extraction (mod extract,
Sec. 2.1) against facts fixed outside the oracle's own code: factorisation of
Y^(M e)+1, irreducibility by brute force, the F_p-slot encoder, ring products
by schoolbook multiplication, the automorphism X -> X^p written out as an index
map, the defining property of the trace-dual basis, and decryption."""
import itertools
import random

import numpy as np
import pytest

from oracle.encoding import SlotStructure
from oracle.extension import ExtSlots, poly_mul
from tests.oracle_setup import OracleSetup
from tests.params import CHAIN50

CASES = [(17, 2 ** 6, 2), (17, 2 ** 7, 4), (131, 2 ** 5, 2), (131, 2 ** 6, 4), (257, 2 ** 9, 2)]


def _negacyclic(a, b, N, p):
    out = [0] * N
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                k = i + j
                if k < N:
                    out[k] = (out[k] + x * y) % p
                else:
                    out[k - N] = (out[k - N] - x * y) % p
    return out


def _sigma(m, g, N, p):
    """X^i -> X^(i g) in Z_p[X]/(X^N+1), written out."""
    out = [0] * N
    for i, v in enumerate(m):
        k = i * g % (2 * N)
        if k < N:
            out[k] = (out[k] + int(v)) % p
        else:
            out[k - N] = (out[k - N] - int(v)) % p
    return out


@pytest.mark.parametrize("p,N,d", CASES)
def test_factors_multiply_to_cyclotomic_and_are_irreducible(p, N, d):
    xs = ExtSlots(p, N, d)
    prod = [1]
    for f in xs.factors:
        assert len(f) == d + 1 and f[-1] == 1
        prod = poly_mul(prod, f, p)
    assert prod == [1] + [0] * (xs.Me - 1) + [1]
    if p ** (d // 2) <= 20000:  # brute force: no monic factor of degree 1 .. d/2
        for f in xs.factors:
            for k in range(1, d // 2 + 1):
                for low in itertools.product(range(p), repeat=k):
                    g = list(low) + [1]
                    # remainder of f by g, by long division written out
                    r = list(f)
                    for i in range(len(r) - len(g), -1, -1):
                        c = r[i + len(g) - 1]
                        for j, gj in enumerate(g):
                            r[i + j] = (r[i + j] - c * gj) % p
                    assert any(r[: len(g) - 1]), (f, g)


@pytest.mark.parametrize("p,N,d", CASES)
def test_encode_decode_products_frobenius(p, N, d):
    xs = ExtSlots(p, N, d)
    rnd = random.Random(p * d)
    a = [[rnd.randrange(p) for _ in range(d)] for _ in range(xs.ns)]
    b = [[rnd.randrange(p) for _ in range(d)] for _ in range(xs.ns)]
    ma, mb = xs.encode(a), xs.encode(b)
    assert xs.decode(ma) == a
    # F_p constants: the F_p-slot encoder's plaintext
    c = [rnd.randrange(p) for _ in range(xs.ns)]
    assert np.array_equal(xs.encode([[v] + [0] * (d - 1) for v in c]), SlotStructure(p, N).encode(c))
    # ring product -> slot-wise field product
    prod = xs.decode(_negacyclic([int(v) for v in ma], [int(v) for v in mb], N, p))
    for s in range(xs.ns):
        want = xs.fmul(s, a[s], b[s])
        assert prod[s] == want + [0] * (d - len(want))
    # sigma_p -> p-th power in every slot; sigma_{p^d} -> identity
    fr = xs.decode(_sigma(ma, p % (2 * N), N, p))
    for s in range(xs.ns):
        want = xs.fpow(s, a[s], p)
        assert fr[s] == want + [0] * (d - len(want))
    assert xs.decode(_sigma(ma, pow(p, d, 2 * N), N, p)) == a


@pytest.mark.parametrize("p,N,d", CASES)
def test_dual_basis(p, N, d):
    xs = ExtSlots(p, N, d)
    for s in range(xs.ns):
        lam = xs.dual_basis(s)
        for k in range(d):
            for j in range(d):
                assert xs.trace(s, xs.fmul(s, lam[k], [0] * j + [1])) == (1 if k == j else 0)


def test_no_extension_slots_where_none_exist():
    for p, N, d in ((131, 2 ** 6, 1), (17, 2 ** 6, 3), (257, 2 ** 8, 4)):
        with pytest.raises(ValueError):
            ExtSlots(p, N, d)


@pytest.mark.parametrize("p,d", [(17, 2), (131, 2), (131, 4)])
def test_extract_digits_decrypts(p, d):
    """Encrypt F_{p^d} slot elements; extraction gives digit k of every slot
    as an F_p constant; the LT/EQ circuit on the extracted digits is the
    integer comparison (values below b^d, b = (p + 1) / 2)."""
    from oracle.circuits import extract_digits

    logN = 8
    xs = ExtSlots(p, 2 ** logN, d)
    st = OracleSetup(logN=logN, p=p, L=6 if p == 17 else 11, K=2, seed=41, galois=xs.galois(), **CHAIN50)
    rnd = random.Random(d)
    b = (p + 1) // 2
    xv = [rnd.randrange(b ** d) for _ in range(xs.ns)]
    yv = [rnd.randrange(b ** d) for _ in range(xs.ns)]
    yv[0] = xv[0]
    dig = lambda v: [(v // b ** k) % b for k in range(d)]  # noqa: E731
    cx = st.encrypt_coeffs([xs.encode([dig(v) for v in xv])], seed=90)[0]
    cy = st.encrypt_coeffs([xs.encode([dig(v) for v in yv])], seed=91)[0]
    ev = st.evaluator()
    dx, dy = extract_digits(ev, cx, d, xs), extract_digits(ev, cy, d, xs)
    for k in range(d):
        assert st.decrypt_slots(dx[k]) == [dig(v)[k] for v in xv]
    lt, eq = ev.compare(dx, dy, True, True)
    assert st.decrypt_slots(lt) == [int(x < y) for x, y in zip(xv, yv)]
    assert st.decrypt_slots(eq) == [int(x == y) for x, y in zip(xv, yv)]
