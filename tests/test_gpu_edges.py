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


def test_slot_pack_mixed_levels_bitexact_and_refusals():
    """Compaction of inputs at different levels (sums are taken at the lower
    level): bit-exact with the oracle; an output array that is too small, a
    missing rotation key and a mask of the wrong shape are refused."""
    from oracle.circuits import slot_galois, slot_pack, slot_plan
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    p, logN, L = 17, 10, 6
    ns = 8
    useful = [[0, 1]] * 4
    n_out, pieces, dest = slot_plan(ns, useful)
    gal = slot_galois(ns, 2 ** logN, pieces)
    params = dict(logN=logN, p=p, L=L, K=2, **CHAIN50)
    g = GpuSetup(seed=61, galois=gal, **params)
    o = OracleSetup(seed=61, galois=gal, **params)
    try:
        rnd = np.random.default_rng(9)
        vals = rnd.integers(0, p, size=(4, 1, ns))
        xg = [g.encrypt_slots(vals[j], seed=900 + j) for j in range(4)]
        xo = [o.encrypt_slots(vals[j], seed=900 + j)[0] for j in range(4)]
        drops = {1: L - 2, 3: L - 1}
        for j, lv in drops.items():
            xg[j] = g.own(fhe.fhe_mod_switch(g.ctx, xg[j], lv))
            for _ in range(L - lv):
                xo[j] = o.o.modswitch(xo[j])
        mask = np.zeros((4, ns), dtype=bool)
        mask[:, :2] = True
        fhe.fhe_trace_enable(g.ctx, True)
        out = fhe.fhe_slot_pack(g.ctx, g.evk, xg, mask)
        for h in out:
            g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        ev = o.evaluator()
        out_o = slot_pack(ev, xo, useful)
        assert sorted(trace_g) == sorted(ev.trace)
        assert np.array_equal(g.export(out[0])[0], out_o[0].data)
        assert fhe.fhe_ct_shape(out[0])[2] == L - 2
        dec = g.decrypt(out[0])[0]
        assert [int(dec[dest[j][u]]) for j in range(4) for u in (0, 1)] == [int(vals[j, 0, u]) for j in range(4)
                                                                           for u in (0, 1)]
        # refusals
        arr = (fhe.c_void_p * 1)()
        handles = fhe._handles(xg)
        u8 = np.ascontiguousarray(mask.astype(np.uint8))
        spread = np.zeros((4, ns), dtype=bool)
        spread[:, 0] = True
        spread[0, :] = True  # input 0 full: 2 outputs
        assert fhe.lib().fhe_slot_pack(g.ctx, g.evk, handles, 4, fhe._ptr(np.ascontiguousarray(spread.astype(np.uint8))),
                                       arr, 1) == -1
        bare = fhe.fhe_evk_create(g.ctx, g.sk, [], 7)
        try:
            assert fhe.lib().fhe_slot_pack(g.ctx, bare, handles, 4, fhe._ptr(u8), arr, 1) == -8
        finally:
            fhe.fhe_evk_destroy(bare)
        with pytest.raises(ValueError):
            fhe.fhe_slot_pack(g.ctx, g.evk, xg, mask[:, :4])
    finally:
        g.close()


def test_extract_and_query_refusals_and_degenerate_cases():
    """Digit extraction: a digit count the ring has no slots of and a missing
    Frobenius key are refused.  Private query: op2 = 1 (the data itself is a
    candidate) and query types matching no code (answer 0)."""
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup

    p, logN = 17, 10
    g = GpuSetup(seed=63, logN=logN, p=p, L=8, K=2, **CHAIN50)
    try:
        ns = g.ns
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ext_galois(g.ctx, 3)
        assert e.value.code == -9
        ct = g.own(fhe.fhe_encrypt_ext(g.ctx, g.pk, np.zeros((1, ns, 2), dtype=np.uint64), 2, 5))
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_extract_digits(g.ctx, g.evk, ct, 2)  # no sigma_17 key in this evk
        assert e.value.code == -8
        rnd = np.random.default_rng(3)
        qv = np.array([[1, 0, 4, 5, 1, 6, 7, 1]], dtype=np.uint64)[:, :ns]
        dv = rnd.integers(0, p, size=(1, ns)).astype(np.uint64)
        ov = rnd.integers(0, p, size=(1, ns)).astype(np.uint64)
        q, data, op1 = (g.own(fhe.fhe_encrypt(g.ctx, g.pk, v, 40 + i)) for i, v in enumerate((qv, dv, ov)))
        out = g.own(fhe.fhe_private_query(g.ctx, g.evk, q, data, op1, 1, (2, 3, 1)))
        want = np.where(qv == 2, (dv + ov) % p, np.where(qv == 3, dv * ov % p, np.where(qv == 1, dv, 0)))
        assert (g.decrypt(out) == want).all()
        with pytest.raises(fhe.FheError):
            fhe.fhe_private_query(g.ctx, g.evk, q, data, op1, 0, (1, 2, 3))
    finally:
        g.close()


def test_checkpoint_resume_of_ciphertexts():
    """A batch imaged with fhe_ct_serialize and restored into a new context
    built from the same seeds gives, through a comparison, the bits of the
    original; images of another ring, a truncated image and an out-of-range
    residue are refused."""
    from paper_2407_07308_gb300 import fhe

    def make(p=17):
        ctx = fhe.fhe_ctx_create(11, p, 8, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
        sk, pk = fhe.fhe_keygen(ctx, 5)
        evk = fhe.fhe_evk_create(ctx, sk, [], 6)
        return ctx, sk, pk, evk

    def free(ctx, sk, pk, evk):
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
        fhe.fhe_ctx_destroy(ctx)

    a = make()
    ctx, sk, pk, evk = a
    ns = fhe.fhe_ctx_info(ctx).slots
    rnd = np.random.default_rng(2)
    xv, yv = rnd.integers(0, 9, size=(2, 3, ns))
    x, y = fhe.fhe_encrypt(ctx, pk, xv, 1), fhe.fhe_encrypt(ctx, pk, yv, 2)
    x3 = fhe.fhe_mod_switch(ctx, x, 5)
    images = [fhe.fhe_ct_serialize(ctx, h) for h in (x, y, x3)]
    lt = fhe.fhe_compare_lt(ctx, evk, [x], [y])
    want = fhe.fhe_ct_export_coeff(ctx, lt)
    for h in (x, y, x3, lt):
        fhe.fhe_ct_destroy(h)
    free(*a)
    b = make()  # resume: same seeds, new context
    ctx, sk, pk, evk = b
    other = make(131)
    try:
        x, y, x3 = (fhe.fhe_ct_deserialize(ctx, im) for im in images)
        assert fhe.fhe_ct_shape(x3)[2] == 5
        lt = fhe.fhe_compare_lt(ctx, evk, [x], [y])
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, lt), want)
        assert (fhe.fhe_decrypt(ctx, sk, lt) == (xv < yv)).all()
        assert fhe.fhe_ct_serialize(ctx, x) == images[0]
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ct_deserialize(other[0], images[0])
        assert e.value.code == -2
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ct_deserialize(ctx, images[0][:-8])
        assert e.value.code == -1
        bad = bytearray(images[0])
        bad[-8:] = (2 ** 64 - 1).to_bytes(8, "little")
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ct_deserialize(ctx, bytes(bad))
        assert e.value.code == -1
        for h in (x, y, x3, lt):
            fhe.fhe_ct_destroy(h)
    finally:
        free(*b)
        free(*other)



def test_pool_size_classes_reuse_nearby_sizes():
    """The pool hands out blocks in size classes of a quarter power of two: a
    983,040-byte ciphertext (3 x 2 x 5 limbs of 2^12 words) takes a 1 MiB
    block; once freed, that block serves a 1,048,576-byte ciphertext
    (4 x 2 x 4 limbs) without reserving more device memory, and both
    ciphertexts survive the round trip through the host."""
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(12, 17, 6, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        rng = np.random.default_rng(3)
        q = np.array(fhe.fhe_ctx_primes(ctx)[:6], dtype=np.uint64).reshape(1, 1, 6, 1)

        def data(count, level):
            x = rng.integers(0, 1 << 62, size=(count, 2, level, 4096), dtype=np.uint64)
            return np.ascontiguousarray(x % q[:, :, :level])

        fhe.fhe_ctx_sync(ctx)
        fhe.fhe_ctx_trim(ctx)
        r0, u0 = fhe.fhe_ctx_memory(ctx)
        a_data = data(3, 5)
        assert a_data.nbytes == 983040
        a = fhe.fhe_ct_import_coeff(ctx, a_data)
        fhe.fhe_ctx_sync(ctx)
        r1, u1 = fhe.fhe_ctx_memory(ctx)
        assert u1 - u0 == 1 << 20 and r1 - r0 == 1 << 20
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, a), a_data)
        fhe.fhe_ct_destroy(a)
        fhe.fhe_ctx_sync(ctx)
        r2, u2 = fhe.fhe_ctx_memory(ctx)
        assert u2 == u0
        e_data = data(4, 4)
        assert e_data.nbytes == 1 << 20
        e = fhe.fhe_ct_import_coeff(ctx, e_data)
        fhe.fhe_ctx_sync(ctx)
        r3, u3 = fhe.fhe_ctx_memory(ctx)
        assert r3 == r2 and u3 - u2 == 1 << 20  # a freed 1 MiB block, reused
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, e), e_data)
        fhe.fhe_ct_destroy(e)
    finally:
        fhe.fhe_ctx_destroy(ctx)
