"""GPU: degenerate and extreme inputs of the comparison path, the largest
supported parameter shapes, and the error codes of malformed calls (each a
host-side check: no kernel runs on a bad argument)."""
import random

import numpy as np
import pytest

from tests.params import CHAIN50

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07308_gb300 import build

    build.build()


def _digits(vals, b, d):
    vals = np.asarray(vals)
    return [(vals // b ** k) % b for k in range(d)]


def test_degenerate_values_bitexact():
    """Equal operands (LT 0, EQ 1, max = min = the value), all-zero operands
    and the extremes 0 / b^d - 1 in both orders, in one batch; the whole batch
    bit-exact with the oracle ciphertext by ciphertext."""
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    p, d = 17, 3
    b = (p + 1) // 2
    top = b ** d - 1
    params = dict(logN=10, p=p, L=9, K=2, **CHAIN50)
    g = GpuSetup(seed=5, **params)
    o = OracleSetup(seed=5, **params)
    try:
        ns = g.ns
        rnd = random.Random(1)
        same = [rnd.randrange(b ** d) for _ in range(ns)]
        xv = np.array([same, [0] * ns, [0] * ns, [top] * ns])
        yv = np.array([same, [0] * ns, [top] * ns, [0] * ns])
        xd, yd = _digits(xv, b, d), _digits(yv, b, d)
        xg = [g.encrypt_slots(xd[k], seed=10 + k) for k in range(d)]
        yg = [g.encrypt_slots(yd[k], seed=20 + k) for k in range(d)]
        lt, eq = fhe.fhe_compare(g.ctx, g.evk, xg, yg)
        g.own(lt)
        g.own(eq)
        mx, mn = fhe.fhe_max_min(g.ctx, g.evk, xg, yg)
        for h in mx + mn:
            g.own(h)
        assert (g.decrypt(lt) == (xv < yv)).all() and (g.decrypt(eq) == (xv == yv)).all()
        got_max = sum(g.decrypt(mx[k]).astype(np.int64) * b ** k for k in range(d))
        got_min = sum(g.decrypt(mn[k]).astype(np.int64) * b ** k for k in range(d))
        assert (got_max == np.maximum(xv, yv)).all() and (got_min == np.minimum(xv, yv)).all()
        xo = [o.encrypt_slots(xd[k].tolist(), seed=10 + k) for k in range(d)]
        yo = [o.encrypt_slots(yd[k].tolist(), seed=20 + k) for k in range(d)]
        for c in range(4):
            ev = o.evaluator()
            lt_o, eq_o = ev.compare([x[c] for x in xo], [y[c] for y in yo], True, True)
            assert np.array_equal(g.export(lt)[c], lt_o.data)
            assert np.array_equal(g.export(eq)[c], eq_o.data)
    finally:
        g.close()


def test_largest_prime_counts():
    """32 primes (the most a context holds: 28 data + 4 special) and 8
    special primes (the most; relinearisation then runs its two ModDowns
    separately): products and a comparison decrypt correctly; 33 primes are
    refused."""
    from paper_2407_07308_gb300 import fhe

    for L, K in ((28, 4), (16, 8)):
        ctx = fhe.fhe_ctx_create(11, 17, L, K, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
        try:
            sk, pk = fhe.fhe_keygen(ctx, L)
            evk = fhe.fhe_evk_create(ctx, sk, [], L + 1)
            ns = fhe.fhe_ctx_info(ctx).slots
            rnd = np.random.default_rng(L)
            xv, yv = rnd.integers(0, 9, size=(2, ns)), rnd.integers(0, 9, size=(2, ns))
            x, y = fhe.fhe_encrypt(ctx, pk, xv, 1), fhe.fhe_encrypt(ctx, pk, yv, 2)
            m = fhe.fhe_mul_relin(ctx, evk, x, y)
            assert (fhe.fhe_decrypt(ctx, sk, m) == (xv * yv) % 17).all()
            assert fhe.fhe_ct_shape(m)[2] == L - 1
            lt, eq = fhe.fhe_compare(ctx, evk, [x], [y])
            assert (fhe.fhe_decrypt(ctx, sk, lt) == (xv < yv)).all()
            for h in (x, y, m, lt, eq):
                fhe.fhe_ct_destroy(h)
            fhe.fhe_evk_destroy(evk)
            fhe.fhe_sk_destroy(sk)
            fhe.fhe_pk_destroy(pk)
        finally:
            fhe.fhe_ctx_destroy(ctx)
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_ctx_create(11, 17, 29, 4, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    assert e.value.code == -9  # FHE_EUNSUPPORTED


def test_malformed_calls_are_refused():
    from paper_2407_07308_gb300 import fhe

    U, lo, hi = CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"]
    for args, code in (((9, 17, 4, 2, U, lo, hi), -9),   # ring degree below the supported range
                       ((16, 17, 4, 2, U, lo, hi), -9),  # and above it
                       ((11, 15, 4, 2, U, lo, hi), -1),  # plaintext modulus not prime
                       ((11, 17, 4, 2, 17 * 131 * 257, lo, hi), -1)):  # primes need q = 1 mod 2N
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ctx_create(*args)
        assert e.value.code == code, args
    ctx = fhe.fhe_ctx_create(11, 17, 6, 2, U, lo, hi)
    other = fhe.fhe_ctx_create(11, 17, 6, 2, U, lo, hi)
    try:
        sk, pk = fhe.fhe_keygen(ctx, 1)
        evk = fhe.fhe_evk_create(ctx, sk, [], 2)
        sk2, pk2 = fhe.fhe_keygen(other, 3)
        ns = fhe.fhe_ctx_info(ctx).slots
        v = np.zeros((2, ns), dtype=np.uint64)
        x, y = fhe.fhe_encrypt(ctx, pk, v, 1), fhe.fhe_encrypt(ctx, pk, v, 2)
        x3 = fhe.fhe_encrypt(ctx, pk, np.zeros((3, ns), dtype=np.uint64), 3)
        z = fhe.fhe_encrypt(other, pk2, v, 4)

        def code_of(fn, *a):
            with pytest.raises(fhe.FheError) as e:
                fn(*a)
            return e.value.code

        assert code_of(fhe.fhe_encrypt, ctx, pk, np.zeros((0, ns), dtype=np.uint64), 5) == -1  # no rows
        assert code_of(fhe.fhe_compare, ctx, evk, [x], [x3]) == -2  # counts differ
        assert code_of(fhe.fhe_compare, ctx, evk, [x], [z]) == -1   # another context's handle
        assert code_of(fhe.fhe_compare, ctx, evk, [], []) == -1     # no digits
        assert code_of(fhe.fhe_mod_switch, ctx, x, 0) == -3         # below level 1
        assert code_of(fhe.fhe_mod_switch, ctx, x, 7) == -3         # above the ciphertext's level
        assert code_of(fhe.fhe_rotate, ctx, evk, x, 5) == -8        # no key for this element
        assert code_of(fhe.fhe_add, ctx, x, x3) == -2               # counts differ
        # the context still works after every refusal
        s = fhe.fhe_add(ctx, x, y)
        assert (fhe.fhe_decrypt(ctx, sk, s) == 0).all()
        for h in (x, y, x3, s):
            fhe.fhe_ct_destroy(h)
        fhe.fhe_ct_destroy(z)
        fhe.fhe_evk_destroy(evk)
        for h in (sk, sk2):
            fhe.fhe_sk_destroy(h)
        for h in (pk, pk2):
            fhe.fhe_pk_destroy(h)
    finally:
        fhe.fhe_ctx_destroy(ctx)
        fhe.fhe_ctx_destroy(other)
