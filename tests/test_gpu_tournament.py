"""GPU: device Philox against the oracle's, seeded key generation and
encryption, refresh, and the max/min tournament (bit-exact on a small ring,
plaintext-exact at the full N=2^15, p=257, d=2 configuration)."""
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


def test_philox_device_matches_oracle():
    from oracle.philox import block
    from paper_2407_07308_gb300 import fhe

    for seed, tag in ((0, 0), (123456789012345, 17), (2 ** 64 - 1, 1024)):
        got = fhe.fhe_philox_blocks(seed, tag, 300)
        for n in (0, 1, 2, 299):
            assert tuple(int(v) for v in got[n]) == block(seed, tag, n)


def test_seeded_keys_and_encryption_decrypt():
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(12, 257, 4, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        sk, pk = fhe.fhe_keygen(ctx, 7)
        evk = fhe.fhe_evk_create(ctx, sk, [5], 8)
        ns = fhe.fhe_ctx_info(ctx).slots
        rnd = random.Random(1)
        a = np.array([[rnd.randrange(257) for _ in range(ns)] for _ in range(3)], dtype=np.uint64)
        b = np.array([[rnd.randrange(257) for _ in range(ns)] for _ in range(3)], dtype=np.uint64)
        ca, cb = fhe.fhe_encrypt(ctx, pk, a, 11), fhe.fhe_encrypt(ctx, pk, b, 12)
        assert (fhe.fhe_decrypt(ctx, sk, ca) == a).all()
        prod = fhe.fhe_mul_relin(ctx, evk, ca, cb)
        assert (fhe.fhe_decrypt(ctx, sk, prod) == (a * b) % 257).all()
        rot = fhe.fhe_rotate(ctx, evk, ca, 5)
        cols = ns // 2
        want = np.array([[row[r * cols + (c + 1) % cols] for r in range(2) for c in range(cols)] for row in a])
        assert (fhe.fhe_decrypt(ctx, sk, rot) == want).all()
        # two seeds give different ciphertexts of the same plaintext
        cc = fhe.fhe_encrypt(ctx, pk, a, 13)
        assert not np.array_equal(fhe.fhe_ct_export_coeff(ctx, ca), fhe.fhe_ct_export_coeff(ctx, cc))
        for h in (ca, cb, cc, prod, rot):
            fhe.fhe_ct_destroy(h)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        fhe.fhe_ctx_destroy(ctx)


def test_refresh_explicit_bitexact():
    from paper_2407_07308_gb300 import fhe, synth
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    params = dict(logN=11, p=17, L=5, K=2, **CHAIN50)
    o = OracleSetup(seed=61, **params)
    g = GpuSetup(seed=61, **params)
    try:
        rows = [[(3 * i + s) % 17 for s in range(g.ns)] for i in range(2)]
        ct_o = o.encrypt_slots(rows, seed=5)
        ct_g = g.encrypt_slots(rows, seed=5)
        low_o = [o.o.modswitch(o.o.modswitch(c)) for c in ct_o]
        low_g = g.own(fhe.fhe_mod_switch(g.ctx, ct_g, 3))
        r = synth.EncRandomness(77, 2, g.N)
        out_g = g.own(fhe.fhe_refresh_explicit(g.ctx, g.sk, g.pk, low_g, r.u, r.e0, r.e1))
        ex = g.export(out_g)
        for i in range(2):
            want = o.o.encrypt(o.pk, o.o.decrypt_coeffs(low_o[i], o.s), r.u[i], r.e0[i], r.e1[i])
            assert np.array_equal(ex[i], want.data)
        assert g.decrypt(out_g).tolist() == rows
    finally:
        g.close()


def _digits(vals, b, d):
    return [[(v // b ** k) % b for v in row] for k in range(d) for row in [vals]]


def test_tournament_small_bitexact():
    from oracle.circuits import Tournament, galois_schedule
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    p, d, logN = 17, 1, 10
    galois = galois_schedule(8, 1 << logN)
    params = dict(logN=logN, p=p, L=21, K=3, **CHAIN50)
    o = OracleSetup(seed=71, galois=galois, **params)
    g = GpuSetup(seed=71, galois=galois, **params)
    try:
        assert fhe.fhe_tournament_galois(g.ctx) == galois
        rnd = random.Random(8)
        vals = [[rnd.randrange(9) for _ in range(g.ns)] for _ in range(2)]
        xg = g.encrypt_slots(vals, seed=90)
        mx, mn = fhe.fhe_tournament(g.ctx, g.evk, None, None, [xg], 1)
        for h in mx + mn:
            g.own(h)
        flat = [v for row in vals for v in row]
        assert g.decrypt(mx[0])[0].tolist() == [max(flat)] * g.ns
        assert g.decrypt(mn[0])[0].tolist() == [min(flat)] * g.ns
        xo = o.encrypt_slots(vals, seed=90)
        out = Tournament(o.evaluator(), d, g.ns, g.N).run([xo], True, True)
        assert np.array_equal(g.export(mx[0])[0], out["max"][0].data)
        assert np.array_equal(g.export(mn[0])[0], out["min"][0].data)
    finally:
        g.close()


def test_tournament_full_config_4096_values():
    """N=2^15, p=257, d=2 (values in [0, 129^2)), 20 x 50-bit + 4 special
    primes: max and min of 4096 values (10% duplicates) packed in 32
    ciphertexts of 128 slots, with refreshes between rounds."""
    from paper_2407_07308_gb300 import fhe, synth

    ctx = fhe.fhe_ctx_create(15, 257, 20, 4, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        sk, pk = fhe.fhe_keygen(ctx, 4)
        evk = fhe.fhe_evk_create(ctx, sk, fhe.fhe_tournament_galois(ctx), 5)
        g = synth.rng(4)
        vals = synth.values_with_duplicates(g, 4096, 129 ** 2, 0.10)
        b, d = 129, 2
        dig = synth.to_digits(vals, b, d)
        xs = [fhe.fhe_encrypt(ctx, pk, dig[k].reshape(32, 128).astype(np.uint64), 100 + k) for k in range(d)]
        mx, mn = fhe.fhe_tournament(ctx, evk, sk, pk, xs, 9)
        got_max = sum(fhe.fhe_decrypt(ctx, sk, mx[k]).astype(np.int64) * b ** k for k in range(d))
        got_min = sum(fhe.fhe_decrypt(ctx, sk, mn[k]).astype(np.int64) * b ** k for k in range(d))
        assert (got_max == vals.max()).all()
        assert (got_min == vals.min()).all()
        for h in xs + mx + mn:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        fhe.fhe_ctx_destroy(ctx)
