"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
identical seeded inputs.  Every comparison of ciphertext limbs is exact
(tolerance 0: integer arithmetic), decryptions are compared with plaintext
results, and the circuit-level operation traces must hold the same operations
at the same levels (the library runs independent operations of a circuit
together, so their order may differ from the oracle's)."""
import os
import random

import numpy as np
import pytest

from tests.params import CHAIN36, CHAIN50

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07308_gb300 import build

    build.build()


def _fhe():
    from paper_2407_07308_gb300 import fhe

    return fhe


def _pair(params, seed=1, galois=()):
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    o = OracleSetup(seed=seed, galois=galois, **params)
    g = GpuSetup(seed=seed, galois=galois, **params)
    assert g.primes == o.o.primes
    return o, g


def _same(oracle_ct, gpu_export, idx=0):
    want = oracle_ct.data
    got = gpu_export[idx]
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# NTT
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("logN,variant", [(10, 0), (10, 2), (11, 0), (11, 1), (12, 0), (12, 1), (12, 2), (12, 3),
                                           (13, 0), (13, 1), (13, 3), (14, 0), (14, 1), (14, 2), (14, 3), (15, 0),
                                           (15, 1), (15, 3), (15, 2)])
def test_ntt_forward_inverse_match_oracle(logN, variant):
    from oracle.bgv import Oracle

    fhe = _fhe()
    L, K = 3, 2
    o = Oracle(logN, 131, L, K, **CHAIN50)
    ctx = fhe.fhe_ctx_create(logN, 131, L, K, **{"prime_mod": CHAIN50["U"], "prime_lo": CHAIN50["lo"],
                                                   "prime_hi": CHAIN50["hi"]})
    try:
        fhe.fhe_ctx_ntt_variant(ctx, variant)
        N = 1 << logN
        g = np.random.default_rng(logN)
        # every prime, plus a ragged repeat pattern of prime indices
        pidx = [0, 1, 2, 3, 4, 2, 0]
        a = np.stack([g.integers(0, o.primes[i], size=N, dtype=np.uint64) for i in pidx])
        dev = torch.from_numpy(a.view(np.int64).copy()).cuda()
        fhe.fhe_ntt_forward(ctx, dev.data_ptr(), pidx, len(pidx))
        torch.cuda.synchronize()
        got = dev.cpu().numpy().view(np.uint64)
        for r, i in enumerate(pidx):
            assert np.array_equal(got[r], o.ntt(i, a[r])), (logN, r)
        fhe.fhe_ntt_inverse(ctx, dev.data_ptr(), pidx, len(pidx))
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), a)
        # inverse of arbitrary evaluation-domain data
        b = np.stack([g.integers(0, o.primes[i], size=N, dtype=np.uint64) for i in pidx])
        dev = torch.from_numpy(b.view(np.int64).copy()).cuda()
        fhe.fhe_ntt_inverse(ctx, dev.data_ptr(), pidx, len(pidx))
        torch.cuda.synchronize()
        got = dev.cpu().numpy().view(np.uint64)
        for r, i in enumerate(pidx):
            assert np.array_equal(got[r], o.intt(i, b[r]))
    finally:
        fhe.fhe_ctx_destroy(ctx)


def test_ntt_max_residues():
    """All-(q-1) input: the lazy butterflies' largest values."""
    from oracle.bgv import Oracle

    fhe = _fhe()
    o = Oracle(14, 131, 2, 1, **CHAIN50)
    ctx = fhe.fhe_ctx_create(14, 131, 2, 1, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        a = np.stack([np.full(1 << 14, q - 1, dtype=np.uint64) for q in o.primes])
        dev = torch.from_numpy(a.view(np.int64).copy()).cuda()
        fhe.fhe_ntt_forward(ctx, dev.data_ptr(), [0, 1, 2], 3)
        torch.cuda.synchronize()
        got = dev.cpu().numpy().view(np.uint64)
        for i in range(3):
            assert np.array_equal(got[i], o.ntt(i, a[i]))
    finally:
        fhe.fhe_ctx_destroy(ctx)


# ---------------------------------------------------------------------------
# keys, encryption, single operations
# ---------------------------------------------------------------------------

SMALL36 = dict(logN=12, p=17, L=4, K=1, **CHAIN36)
RAGGED50 = dict(logN=11, p=17, L=5, K=2, **CHAIN50)   # digits of 2, 2, 1 limbs
MID50 = dict(logN=14, p=131, L=10, K=3, **CHAIN50)


@pytest.mark.parametrize("params", [SMALL36, RAGGED50], ids=["n12_36b", "n11_50b"])
def test_encrypt_bitexact(params):
    o, g = _pair(params, seed=3)
    try:
        rnd = random.Random(1)
        rows = [[rnd.randrange(params["p"]) for _ in range(g.ns)] for _ in range(3)]
        cts_o = o.encrypt_slots(rows, seed=9)
        ct_g = g.encrypt_slots(rows, seed=9)
        ex = g.export(ct_g)
        for i in range(3):
            _same(cts_o[i], ex, i)
        assert g.decrypt(ct_g).tolist() == rows
    finally:
        g.close()


@pytest.mark.parametrize("params", [SMALL36, RAGGED50], ids=["n12_36b", "n11_50b"])
def test_single_ops_bitexact(params):
    fhe = _fhe()
    galois = (5, 2 * (1 << params["logN"]) - 1)
    o, g = _pair(params, seed=4, galois=galois)
    try:
        p = params["p"]
        rnd = random.Random(2)
        a = [rnd.randrange(p) for _ in range(g.ns)]
        b = [rnd.randrange(p) for _ in range(g.ns)]
        ca_o, cb_o = o.encrypt_slots([a, b], seed=11)
        ca_g, cb_g = g.encrypt_each([a, b], seed=11)
        oc = o.o
        X = g.ctx
        checks = [
            ("add", oc.add(ca_o, cb_o), fhe.fhe_add(X, ca_g, cb_g)),
            ("sub", oc.sub(ca_o, cb_o), fhe.fhe_sub(X, ca_g, cb_g)),
            ("neg", oc.neg(ca_o), fhe.fhe_neg(X, ca_g)),
            ("cmul", oc.mul_const(ca_o, -7), fhe.fhe_mul_const(X, ca_g, p - 7)),
            ("cadd", oc.add_const(ca_o, 3), fhe.fhe_add_const(X, ca_g, 3)),
            ("tensor", oc.tensor(ca_o, cb_o), fhe.fhe_mul(X, ca_g, cb_g)),
            ("modswitch", oc.modswitch(ca_o), fhe.fhe_mod_switch(X, ca_g, params["L"] - 1)),
            ("modswitch2", oc.modswitch(oc.modswitch(ca_o)), fhe.fhe_mod_switch(X, ca_g, params["L"] - 2)),
        ]
        d_o = oc.tensor(ca_o, cb_o)
        checks.append(("relin", oc.relin(d_o, o.rlk), fhe.fhe_relinearize(X, g.evk, checks[5][2])))
        ev = o.evaluator()
        checks.append(("mul_relin", ev.mul(ca_o, cb_o), fhe.fhe_mul_relin(X, g.evk, ca_g, cb_g)))
        for gal in galois:
            checks.append((f"rot{gal}", oc.rotate(ca_o, gal, o.gks[gal]), fhe.fhe_rotate(X, g.evk, ca_g, gal)))
        # a lower-level operand: relinearisation with a short last digit
        low_o = oc.modswitch(ca_o)
        low_g = fhe.fhe_mod_switch(X, ca_g, params["L"] - 1)
        dl_o = oc.tensor(low_o, low_o)
        dl_g = fhe.fhe_mul(X, low_g, low_g)
        checks.append(("relin_low", oc.relin(dl_o, o.rlk), fhe.fhe_relinearize(X, g.evk, dl_g)))
        for name, want, got in checks:
            g.own(got)
            ex = g.export(got)
            assert np.array_equal(ex[0], want.data), name
        g.own(low_g)
        g.own(dl_g)
    finally:
        g.close()


# ---------------------------------------------------------------------------
# comparison circuits
# ---------------------------------------------------------------------------

def _values(rnd, n, hi, dup=0.3):
    xs = [rnd.randrange(hi) for _ in range(n)]
    ys = [x if rnd.random() < dup else rnd.randrange(hi) for x in xs]
    return xs, ys


def _digits(vals, b, d):
    return [[(v // b ** k) % b for v in vals] for k in range(d)]


def _run_compare(params, d, count, seed, want_maxmin=False, check_bits=True):
    fhe = _fhe()
    o, g = _pair(params, seed=seed)
    try:
        p = params["p"]
        b = (p + 1) // 2
        rnd = random.Random(seed)
        xv, yv = zip(*[_values(rnd, g.ns, b ** d) for _ in range(count)])
        # digit k of every ciphertext of the batch: rows [count][ns]
        xd = [[_digits(xv[c], b, d)[k] for c in range(count)] for k in range(d)]
        yd = [[_digits(yv[c], b, d)[k] for c in range(count)] for k in range(d)]
        xg = [g.encrypt_slots(xd[k], seed=100 + k) for k in range(d)]
        yg = [g.encrypt_slots(yd[k], seed=200 + k) for k in range(d)]
        fhe.fhe_trace_enable(g.ctx, True)
        lt_g, eq_g = fhe.fhe_compare(g.ctx, g.evk, xg, yg)
        g.own(lt_g)
        g.own(eq_g)
        trace_g = fhe.fhe_trace_get(g.ctx)
        lt_dec, eq_dec = g.decrypt(lt_g), g.decrypt(eq_g)
        for c in range(count):
            assert lt_dec[c].tolist() == [int(a < e) for a, e in zip(xv[c], yv[c])]
            assert eq_dec[c].tolist() == [int(a == e) for a, e in zip(xv[c], yv[c])]
        if check_bits:
            # oracle on ciphertext 0 of the batch, same randomness
            xo = [o.encrypt_slots(xd[k], seed=100 + k)[0] for k in range(d)]
            yo = [o.encrypt_slots(yd[k], seed=200 + k)[0] for k in range(d)]
            ev = o.evaluator()
            lt_o, eq_o = ev.compare(xo, yo, True, True)
            assert sorted(trace_g) == sorted(ev.trace)
            _same(lt_o, g.export(lt_g), 0)
            _same(eq_o, g.export(eq_g), 0)
        if want_maxmin:
            mx, mn = fhe.fhe_max_min(g.ctx, g.evk, xg, yg)
            for h in mx + mn:
                g.own(h)
            mxd = [g.decrypt(h) for h in mx]
            mnd = [g.decrypt(h) for h in mn]
            for c in range(count):
                got_max = [sum(int(mxd[k][c][s]) * b ** k for k in range(d)) for s in range(g.ns)]
                got_min = [sum(int(mnd[k][c][s]) * b ** k for k in range(d)) for s in range(g.ns)]
                assert got_max == [max(a, e) for a, e in zip(xv[c], yv[c])]
                assert got_min == [min(a, e) for a, e in zip(xv[c], yv[c])]
            if check_bits:
                mx_o, mn_o = ev.max_min(xo, yo)
                for k in range(d):
                    _same(mx_o[k], g.export(mx[k]), 0)
                    _same(mn_o[k], g.export(mn[k]), 0)
    finally:
        g.close()


def test_compare_p17_d2_small_ring():
    _run_compare(dict(logN=10, p=17, L=7, K=2, **CHAIN50), d=2, count=3, seed=5, want_maxmin=True)


def test_compare_p17_d3_ragged_merge():
    _run_compare(dict(logN=10, p=17, L=8, K=3, **CHAIN50), d=3, count=2, seed=6)


def test_compare_p131_d1_small_ring():
    _run_compare(dict(logN=10, p=131, L=9, K=3, **CHAIN50), d=1, count=2, seed=7)


def test_compare_p257_d1_small_ring():
    _run_compare(dict(logN=10, p=257, L=9, K=4, **CHAIN50), d=1, count=2, seed=8)


def test_compare_small_config_full():
    """N=2^12, p=17, d=1, 4x36-bit + 1 special prime: one LT (and EQ)."""
    _run_compare(SMALL36, d=1, count=1, seed=1)


def test_batch_equals_singles():
    """A batch gives the same bits as each ciphertext on its own."""
    fhe = _fhe()
    from tests.gpu_setup import GpuSetup

    params = dict(logN=11, p=17, L=6, K=2, **CHAIN50)
    g = GpuSetup(seed=12, **params)
    try:
        rnd = random.Random(3)
        xs = [[rnd.randrange(9) for _ in range(g.ns)] for _ in range(4)]
        ys = [[rnd.randrange(9) for _ in range(g.ns)] for _ in range(4)]
        xb, yb = g.encrypt_slots(xs, seed=1), g.encrypt_slots(ys, seed=2)
        lt_b = g.own(fhe.fhe_compare_lt(g.ctx, g.evk, [xb], [yb]))
        ex_b = g.export(lt_b)
        xe, ye = g.encrypt_each(xs, seed=1), g.encrypt_each(ys, seed=2)
        for i in range(4):
            lt_i = g.own(fhe.fhe_compare_lt(g.ctx, g.evk, [xe[i]], [ye[i]]))
            assert np.array_equal(g.export(lt_i)[0], ex_b[i])
    finally:
        g.close()


@pytest.mark.parametrize("logN,variants", [(13, (0, 1, 2, 3)), (12, (0, 1, 2, 3)), (14, (0, 1, 2, 3))])
def test_ntt_variants_and_autotuner(logN, variants):
    """Every NTT variant gives the same bits through the whole compare path
    (16 ciphertexts, so the grouped row kernels run), and the autotuner
    returns one of them."""
    fhe = _fhe()
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=13, logN=logN, p=17, L=6, K=2, **CHAIN50)
    try:
        # which variant wins is a timing matter (the benchmark reports it);
        # here only that the autotuner returns one that exists
        v, ms = fhe.fhe_ctx_ntt_variant(g.ctx)
        if not os.environ.get("FHE_NTT_VARIANT"):  # a pinned variant skips the timings
            assert v in variants
            assert fhe.fhe_ctx_autotune(g.ctx, 64) in variants
        rnd = random.Random(4)
        xs = [[rnd.randrange(9) for _ in range(g.ns)] for _ in range(16)]
        ys = [[x if rnd.random() < 0.3 else rnd.randrange(9) for x in row] for row in xs]
        xb, yb = g.encrypt_slots(xs, seed=1), g.encrypt_slots(ys, seed=2)
        out = []
        for variant in variants:
            fhe.fhe_ctx_ntt_variant(g.ctx, variant)
            lt, eq = fhe.fhe_compare(g.ctx, g.evk, [xb], [yb])
            g.own(lt)
            g.own(eq)
            out.append((g.export(lt), g.export(eq)))
            lt_dec = g.decrypt(lt)
            for c in range(16):
                assert lt_dec[c].tolist() == [int(a < b) for a, b in zip(xs[c], ys[c])]
        for o in out[1:]:
            assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])
        with pytest.raises(fhe.FheError):
            fhe.fhe_ctx_ntt_variant(g.ctx, 4)
    finally:
        g.close()


def test_compare_plan_graph_matches_direct_and_is_isolated():
    """The captured (graph) form gives the bits of the direct call, replays
    deterministically, picks up inputs refreshed in place, and never aliases
    memory handed out after capture."""
    fhe = _fhe()
    from tests.gpu_setup import GpuSetup

    params = dict(logN=12, p=17, L=6, K=2, **CHAIN50)
    g = GpuSetup(seed=13, **params)
    try:
        rnd = random.Random(9)
        rows = lambda: [[rnd.randrange(9) for _ in range(g.ns)] for _ in range(4)]
        xs = [g.encrypt_slots(rows(), seed=1 + k) for k in range(2)]
        ys = [g.encrypt_slots(rows(), seed=3 + k) for k in range(2)]
        lt_d, eq_d = fhe.fhe_compare(g.ctx, g.evk, xs, ys)
        g.own(lt_d)
        g.own(eq_d)
        want_lt, want_eq = g.export(lt_d), g.export(eq_d)
        plan = fhe.fhe_compare_plan(g.ctx, g.evk, xs, ys)
        try:
            assert fhe.fhe_plan_nodes(plan) > 50
            for _ in range(2):
                fhe.fhe_plan_run(plan, g.ctx)
                assert np.array_equal(g.export(fhe.fhe_plan_result(plan, 0)), want_lt)
                assert np.array_equal(g.export(fhe.fhe_plan_result(plan, 1)), want_eq)
            # memory obtained after capture is not reused by the graph
            other = g.encrypt_slots(rows(), seed=99)
            before = g.export(other)
            fhe.fhe_plan_run(plan, g.ctx)
            fhe.fhe_ctx_sync(g.ctx)
            assert np.array_equal(g.export(other), before)
            # refresh one input in place: the replay follows it
            new_x0 = g.encrypt_slots(rows(), seed=50)
            fhe.fhe_ct_load_coeff(g.ctx, xs[0], g.export(new_x0))
            fhe.fhe_plan_run(plan, g.ctx)
            lt2, eq2 = fhe.fhe_compare(g.ctx, g.evk, xs, ys)
            g.own(lt2)
            g.own(eq2)
            assert np.array_equal(g.export(fhe.fhe_plan_result(plan, 0)), g.export(lt2))
            assert np.array_equal(g.export(fhe.fhe_plan_result(plan, 1)), g.export(eq2))
        finally:
            fhe.fhe_plan_destroy(plan)
    finally:
        g.close()


def test_ntt_batch_entry_matches_per_limb_entry():
    """fhe_ntt_forward_batch / fhe_ntt_inverse_batch over [count][nprimes][N]
    give the per-limb transforms of fhe_ntt_forward / fhe_ntt_inverse."""
    import torch

    fhe = _fhe()
    ctx = fhe.fhe_ctx_create(12, 17, 6, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        primes = fhe.fhe_ctx_primes(ctx)
        N, count, npr = 1 << 12, 5, 4
        rng = np.random.default_rng(3)
        host = np.stack([rng.integers(0, int(primes[i]), size=(count, N), dtype=np.uint64) for i in range(npr)], 1)
        a = torch.from_numpy(host.view(np.int64).copy()).cuda()
        b = a.clone()
        fhe.fhe_ntt_forward_batch(ctx, a.data_ptr(), count, npr)
        fhe.fhe_ntt_forward(ctx, b.data_ptr(), [i % npr for i in range(count * npr)], count * npr)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        fhe.fhe_ntt_inverse_batch(ctx, a.data_ptr(), count, npr)
        torch.cuda.synchronize()
        assert np.array_equal(a.cpu().numpy().view(np.uint64), host)
    finally:
        fhe.fhe_ctx_destroy(ctx)


@pytest.mark.parametrize("logN,p,L,K", [(12, 17, 6, 2), (13, 257, 9, 4), (14, 131, 10, 3)])
def test_fused_relin_modswitch_equals_separate_steps(logN, p, L, K):
    """Relinearise + modulus switch as one ModDown gives the residues of the
    two separate steps: product by product (every level) and through a whole
    comparison."""
    fhe = _fhe()
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=21, logN=logN, p=p, L=L, K=K, **CHAIN50)
    try:
        rnd = random.Random(logN + p)
        b = (p + 1) // 2
        xs = [[rnd.randrange(b) for _ in range(g.ns)] for _ in range(3)]
        ys = [[rnd.randrange(b) for _ in range(g.ns)] for _ in range(3)]
        x, y = g.encrypt_slots(xs, seed=1), g.encrypt_slots(ys, seed=2)
        for fused in (True, False):
            fhe.fhe_ctx_fused_modswitch(g.ctx, fused)
            a, res = x, []
            for _ in range(L - 1):  # repeated products down to level 1
                a = g.own(fhe.fhe_mul_relin(g.ctx, g.evk, a, y))
                res.append(g.export(a))
            lt, eq = fhe.fhe_compare(g.ctx, g.evk, [x], [y])
            g.own(lt)
            g.own(eq)
            res += [g.export(lt), g.export(eq)]
            if fused:
                first = res
        for u, v in zip(first, res):
            assert np.array_equal(u, v)
    finally:
        fhe.fhe_ctx_fused_modswitch(g.ctx, True)
        g.close()


@pytest.mark.parametrize("logN,p,L,K", [(12, 17, 12, 2), (13, 131, 10, 3)])
def test_multi_level_switch_equals_single_steps(logN, p, L, K):
    """Dropping k primes in one step (fhe_mod_switch to a level k below) gives
    the residues of k single-prime switches, for every k, and decrypts."""
    fhe = _fhe()
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=31, logN=logN, p=p, L=L, K=K, **CHAIN50)
    try:
        rnd = random.Random(p)
        rows = [[rnd.randrange(p) for _ in range(g.ns)] for _ in range(3)]
        x = g.encrypt_slots(rows, seed=5)
        single = {L: g.export(x)}
        cur = x
        for lv in range(L - 1, 0, -1):
            cur = g.own(fhe.fhe_mod_switch(g.ctx, cur, lv))
            single[lv] = g.export(cur)
        for lv in range(L - 1, 0, -1):
            direct = g.own(fhe.fhe_mod_switch(g.ctx, x, lv))
            assert np.array_equal(g.export(direct), single[lv]), lv
        assert np.array_equal(g.decrypt(direct), np.array(rows, dtype=np.uint64))
    finally:
        g.close()


@pytest.mark.parametrize("logN,p,L,K,d,count", [(10, 17, 8, 2, 2, 3), (10, 131, 10, 3, 1, 2)])
def test_compare_bivariate_full_digits_bitexact(logN, p, L, K, d, count):
    """The bivariate circuit on full digits in [0, p): LT and EQ of values
    in [0, p^d) decrypt to the plaintext comparison for every ciphertext of
    the batch; ciphertext 0 is bit-exact with the oracle and the op traces
    are equal."""
    fhe = _fhe()
    params = dict(logN=logN, p=p, L=L, K=K, **CHAIN50)
    o, g = _pair(params, seed=19)
    try:
        rnd = random.Random(p + d)
        xv, yv = zip(*[_values(rnd, g.ns, p ** d) for _ in range(count)])
        xd = [[_digits(xv[c], p, d)[k] for c in range(count)] for k in range(d)]
        yd = [[_digits(yv[c], p, d)[k] for c in range(count)] for k in range(d)]
        xg = [g.encrypt_slots(xd[k], seed=300 + k) for k in range(d)]
        yg = [g.encrypt_slots(yd[k], seed=400 + k) for k in range(d)]
        fhe.fhe_trace_enable(g.ctx, True)
        lt_g, eq_g = fhe.fhe_compare_bivariate(g.ctx, g.evk, xg, yg)
        g.own(lt_g)
        g.own(eq_g)
        trace_g = fhe.fhe_trace_get(g.ctx)
        lt_dec, eq_dec = g.decrypt(lt_g), g.decrypt(eq_g)
        for c in range(count):
            assert lt_dec[c].tolist() == [int(a < e) for a, e in zip(xv[c], yv[c])]
            assert eq_dec[c].tolist() == [int(a == e) for a, e in zip(xv[c], yv[c])]
        xo = [o.encrypt_slots(xd[k], seed=300 + k)[0] for k in range(d)]
        yo = [o.encrypt_slots(yd[k], seed=400 + k)[0] for k in range(d)]
        ev = o.evaluator()
        lt_o, eq_o = ev.compare(xo, yo, True, True, bivariate=True)
        assert sorted(trace_g) == sorted(ev.trace)
        _same(lt_o, g.export(lt_g), 0)
        _same(eq_o, g.export(eq_g), 0)
    finally:
        g.close()


def test_plaintext_operands_bitexact():
    """ct + pt, ct - pt, ct * pt with one slot vector for the whole batch:
    ciphertext 0 bit-exact with the oracle, every ciphertext decrypts to the
    slot-wise result."""
    fhe = _fhe()
    params = dict(logN=10, p=17, L=3, K=2, **CHAIN50)
    o, g = _pair(params, seed=27)
    try:
        rnd = random.Random(6)
        rows = [[rnd.randrange(17) for _ in range(g.ns)] for _ in range(2)]
        v = [rnd.randrange(17) for _ in range(g.ns)]
        x = g.encrypt_slots(rows, seed=7)
        xo = o.encrypt_slots(rows, seed=7)[0]
        ev = o.evaluator()
        for name, ref, f in (("add", ev.add_plain, lambda a, b: (a + b) % 17),
                             ("sub", ev.sub_plain, lambda a, b: (a - b) % 17),
                             ("mul", ev.mul_plain, lambda a, b: a * b % 17)):
            r = g.own(getattr(fhe, f"fhe_{name}_plain")(g.ctx, x, v))
            _same(ref(xo, v), g.export(r), 0)
            dec = g.decrypt(r)
            for c in range(2):
                assert dec[c].tolist() == [f(a, b) for a, b in zip(rows[c], v)]
    finally:
        g.close()


def test_sort_rows_bitexact():
    """Every row (cols = 4 values of 2 digits, ties included) of every
    ciphertext sorted; ciphertext 0 bit-exact with the oracle's sort and the
    op traces equal."""
    from oracle.circuits import sort_galois, sort_rows

    fhe = _fhe()
    p, d, logN = 17, 2, 10
    gal = sort_galois(p, 2 ** logN)
    params = dict(logN=logN, p=p, L=11, K=2, **CHAIN50)
    o, g = _pair(params, seed=29, galois=gal)
    try:
        assert fhe.fhe_sort_galois(g.ctx) == gal
        b = (p + 1) // 2
        rnd = random.Random(8)
        vals = [[rnd.randrange(b ** d) for _ in range(g.ns)] for _ in range(2)]
        vals[0][1] = vals[0][3]  # ties
        vals[1][4] = vals[1][5]
        dg = [[_digits(vals[c], b, d)[k] for c in range(2)] for k in range(d)]
        xg = [g.encrypt_slots(dg[k], seed=500 + k) for k in range(d)]
        fhe.fhe_trace_enable(g.ctx, True)
        out = fhe.fhe_sort(g.ctx, g.evk, xg)
        for h in out:
            g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        cols = g.ns // 2
        dec = [g.decrypt(h) for h in out]
        for c in range(2):
            got = [sum(int(dec[k][c][s]) * b ** k for k in range(d)) for s in range(g.ns)]
            assert got == sorted(vals[c][:cols]) + sorted(vals[c][cols:])
        xo = [o.encrypt_slots(dg[k], seed=500 + k)[0] for k in range(d)]
        ev = o.evaluator()
        out_o = sort_rows(ev, xo)
        assert sorted(trace_g) == sorted(ev.trace)
        for k in range(d):
            _same(out_o[k], g.export(out[k]), 0)
    finally:
        g.close()


@pytest.mark.parametrize("p,kind", [(17, "lead1"), (17, "lead2"), (17, "lead4"), (17, "stride4"),
                                    (17, "random"), (131, "lead1")])
def test_slot_pack_bitexact(p, kind):
    """Slot compaction (values in some slots, garbage elsewhere): every useful
    value decrypts where the plan puts it, each output bit-exact with the
    oracle's compaction, op traces equal."""
    from oracle.circuits import slot_galois, slot_pack, slot_plan
    from oracle.encoding import SlotStructure

    fhe = _fhe()
    logN = 10
    N = 2 ** logN
    ns = SlotStructure(p, N).ns
    rnd = random.Random(p + len(kind))
    if kind.startswith("lead"):
        used = int(kind[4:])
        useful = [list(range(used))] * (ns // used)
    elif kind == "stride4":
        useful = [[i for i in range(ns) if i % 4 == 3]] * 4
    else:
        useful = [sorted(rnd.sample(range(ns), rnd.randrange(1, ns))) for _ in range(5)]
    n_out, pieces, dest = slot_plan(ns, useful)
    gal = slot_galois(ns, N, pieces)
    params = dict(logN=logN, p=p, L=6, K=2, **CHAIN50)
    o, g = _pair(params, seed=31 + len(kind), galois=gal)
    try:
        mask = np.zeros((len(useful), ns), dtype=bool)
        for j, u_j in enumerate(useful):
            mask[j, u_j] = True
        assert fhe.fhe_slot_plan(g.ns, N, mask)[2] == gal
        vals = [[[rnd.randrange(p) for _ in range(ns)] for _ in range(2)] for _ in useful]
        xg = [g.encrypt_slots(vals[j], seed=600 + j) for j in range(len(useful))]
        fhe.fhe_trace_enable(g.ctx, True)
        outs = fhe.fhe_slot_pack(g.ctx, g.evk, xg, mask)
        for h in outs:
            g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        assert len(outs) == n_out
        dec = [g.decrypt(h) for h in outs]
        for j, u_j in enumerate(useful):
            for u in u_j:
                q, t = divmod(dest[j][u], ns)
                assert [int(dec[q][c][t]) for c in range(2)] == [vals[j][c][u] for c in range(2)]
        xo = [o.encrypt_slots(vals[j], seed=600 + j)[0] for j in range(len(useful))]
        ev = o.evaluator()
        outs_o = slot_pack(ev, xo, useful)
        assert sorted(trace_g) == sorted(ev.trace)
        for q in range(n_out):
            _same(outs_o[q], g.export(outs[q]), 0)
    finally:
        g.close()


@pytest.mark.parametrize("p,d,logN", [(17, 2, 10), (131, 2, 10), (131, 4, 10), (257, 2, 10)])
def test_extract_digits_bitexact(p, d, logN):
    """F_{p^d}-slot encryption bit-exact with the oracle's encoding; digit
    extraction bit-exact digit by digit, op traces equal; the digits decrypt
    to the inputs and fhe_decrypt_ext inverts the encoding."""
    from oracle.circuits import extract_digits
    from oracle.extension import ExtSlots

    fhe = _fhe()
    N = 2 ** logN
    xs = ExtSlots(p, N, d)
    params = dict(logN=logN, p=p, L=6, K=2, **CHAIN50)
    o, g = _pair(params, seed=43 + d, galois=xs.galois())
    try:
        assert fhe.fhe_ext_galois(g.ctx, d) == xs.galois()
        rnd = np.random.default_rng(p * d)
        digits = rnd.integers(0, p, size=(2, xs.ns, d))
        ct = g.encrypt_ext(digits, d, seed=700)
        assert (fhe.fhe_decrypt_ext(g.ctx, g.sk, ct, d) == digits).all()
        co = o.encrypt_coeffs([xs.encode(digits[c].tolist()) for c in range(2)], seed=700)[0]
        _same(co, g.export(ct), 0)
        fhe.fhe_trace_enable(g.ctx, True)
        out = fhe.fhe_extract_digits(g.ctx, g.evk, ct, d)
        for h in out:
            g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        for k in range(d):
            assert (g.decrypt(out[k]) == digits[:, :, k]).all()
        ev = o.evaluator()
        out_o = extract_digits(ev, co, d, xs)
        assert sorted(trace_g) == sorted(ev.trace)
        for k in range(d):
            _same(out_o[k], g.export(out[k]), 0)
    finally:
        g.close()


def test_extract_then_compare():
    """Operands sent as one F_{131^2}-slot ciphertext each (values below
    66^2): extraction on the device, then LT / EQ; decrypts to the integer
    comparison."""
    fhe = _fhe()
    from oracle.extension import ExtSlots

    p, d, logN = 131, 2, 11
    xs = ExtSlots(p, 2 ** logN, d)
    params = dict(logN=logN, p=p, L=11, K=3, **CHAIN50)
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=47, galois=xs.galois(), **params)
    try:
        b = (p + 1) // 2
        rnd = np.random.default_rng(5)
        xv = rnd.integers(0, b ** d, size=(3, g.ns))
        yv = rnd.integers(0, b ** d, size=(3, g.ns))
        yv[0] = xv[0]
        dig = lambda v: np.stack([(v // b ** k) % b for k in range(d)], axis=-1)  # noqa: E731
        cx = g.own(fhe.fhe_encrypt_ext(g.ctx, g.pk, dig(xv), d, 11))
        cy = g.own(fhe.fhe_encrypt_ext(g.ctx, g.pk, dig(yv), d, 12))
        dx = [g.own(h) for h in fhe.fhe_extract_digits(g.ctx, g.evk, cx, d)]
        dy = [g.own(h) for h in fhe.fhe_extract_digits(g.ctx, g.evk, cy, d)]
        lt, eq = fhe.fhe_compare(g.ctx, g.evk, dx, dy)
        g.own(lt)
        g.own(eq)
        assert (g.decrypt(lt) == (xv < yv)).all() and (g.decrypt(eq) == (xv == yv)).all()
    finally:
        g.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_private_query_bitexact(overlap):
    """Private query (branches straight-lined): bit-exact with the oracle,
    op traces equal, whether the comparison branch overlaps the arithmetic
    on the scheduler's streams or not; decrypts to the selected candidate."""
    from oracle.circuits import private_query

    fhe = _fhe()
    p, logN = 17, 10
    params = dict(logN=logN, p=p, L=8, K=2, **CHAIN50)
    o, g = _pair(params, seed=53)
    try:
        rnd = random.Random(6)
        rows = lambda hi: [[rnd.randrange(hi) for _ in range(g.ns)] for _ in range(2)]  # noqa: E731
        qv, dv, ov = rows(5), rows(p), rows(p)
        qv[0][:4] = [0, 1, 2, 3]
        qg, dg, og = (g.encrypt_slots(v, seed=800 + i) for i, v in enumerate((qv, dv, ov)))
        fhe.fhe_trace_enable(g.ctx, True)
        out = g.own(fhe.fhe_private_query(g.ctx, g.evk, qg, dg, og, 3, (1, 2, 3), overlap=overlap))
        trace_g = fhe.fhe_trace_get(g.ctx)
        dec = g.decrypt(out)
        for c in range(2):
            want = [((d + x) if t == 1 else (d * x) if t == 2 else d ** 3 if t == 3 else 0) % p
                    for t, d, x in zip(qv[c], dv[c], ov[c])]
            assert [int(v) for v in dec[c]] == want
        qo, do, oo = (o.encrypt_slots(v, seed=800 + i)[0] for i, v in enumerate((qv, dv, ov)))
        ev = o.evaluator()
        out_o = private_query(ev, qo, do, oo, 3, (1, 2, 3))
        assert sorted(trace_g) == sorted(ev.trace)
        _same(out_o, g.export(out), 0)
        fhe.fhe_trace_enable(g.ctx, False)
        # captured as a graph: every replay gives the same bits
        plan = fhe.fhe_private_query_plan(g.ctx, g.evk, qg, dg, og, 3, (1, 2, 3), serial=not overlap)
        try:
            for _ in range(2):
                fhe.fhe_plan_run(plan, g.ctx)
                assert np.array_equal(g.export(fhe.fhe_plan_result(plan, 0)), g.export(out))
        finally:
            fhe.fhe_plan_destroy(plan)
    finally:
        g.close()


def test_sort_joint_bitexact():
    """Sixteen values per row across four ciphertexts (p = 17, 4 columns),
    ties across ciphertexts: bit-exact with the oracle's joint sort, traces
    equal, decrypts to the sorted sequence; K cols > p is refused."""
    from oracle.circuits import sort_galois, sort_joint

    fhe = _fhe()
    p, d, logN, K = 17, 2, 10, 4
    gal = sort_galois(p, 2 ** logN)
    params = dict(logN=logN, p=p, L=11, K=2, **CHAIN50)
    o, g = _pair(params, seed=37, galois=gal)
    try:
        b = (p + 1) // 2
        cols = g.ns // 2
        rnd = random.Random(12)
        vals = [[rnd.randrange(b ** d) for _ in range(g.ns)] for _ in range(K)]
        vals[3][1] = vals[0][0]
        vals[2][6] = vals[1][5]
        dig = lambda v: [[(x // b ** k) % b for x in v] for k in range(d)]  # noqa: E731
        xg = [[g.encrypt_slots([dig(vals[a])[k]], seed=1000 + 10 * a + k) for k in range(d)] for a in range(K)]
        fhe.fhe_trace_enable(g.ctx, True)
        out = fhe.fhe_sort_joint(g.ctx, g.evk, xg)
        for hs in out:
            for h in hs:
                g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        fhe.fhe_trace_enable(g.ctx, False)
        dec = [[sum(int(g.decrypt(out[t][k])[0][s]) * b ** k for k in range(d)) for s in range(g.ns)] for t in range(K)]
        for r in range(2):
            seq = [vals[a][r * cols + c] for a in range(K) for c in range(cols)]
            assert [dec[t][r * cols + c] for t in range(K) for c in range(cols)] == sorted(seq)
        xo = [[o.encrypt_slots([dig(vals[a])[k]], seed=1000 + 10 * a + k)[0] for k in range(d)] for a in range(K)]
        ev = o.evaluator()
        out_o = sort_joint(ev, xo)
        assert sorted(trace_g) == sorted(ev.trace)
        for t in range(K):
            for k in range(d):
                _same(out_o[t][k], g.export(out[t][k]), 0)
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_sort_joint(g.ctx, g.evk, xg + [xg[0]])  # 5 x 4 columns > 17
        assert e.value.code == -1
    finally:
        g.close()


def test_sort_ranks_longer_than_p_bitexact():
    """Sequences longer than p (24 values per row at p = 17: six ciphertexts
    of 4 columns, ties included): the ranks and the comparison matrix
    bit-exact with the oracle, the ranks decrypting to the plaintext ranks
    mod p and the matrix to the plaintext comparisons."""
    from oracle.circuits import sort_galois, sort_ranks

    fhe = _fhe()
    p, d, logN, K = 17, 1, 10, 6
    gal = sort_galois(p, 2 ** logN)
    params = dict(logN=logN, p=p, L=8, K=2, **CHAIN50)
    o, g = _pair(params, seed=39, galois=gal)
    try:
        b = (p + 1) // 2
        cols = g.ns // 2
        rnd = random.Random(14)
        vals = [[rnd.randrange(b) for _ in range(g.ns)] for _ in range(K)]
        vals[5][1] = vals[0][2]
        vals[3][6] = vals[2][6]
        xg = [[g.encrypt_slots([vals[a]], seed=2000 + a)] for a in range(K)]
        fhe.fhe_trace_enable(g.ctx, True)
        ranks, mat = fhe.fhe_sort_ranks(g.ctx, g.evk, xg, matrix=True)
        for h in ranks + list(mat.values()):
            g.own(h)
        trace_g = fhe.fhe_trace_get(g.ctx)
        fhe.fhe_trace_enable(g.ctx, False)
        for r in range(2):
            seq = [vals[a][r * cols + c] for a in range(K) for c in range(cols)]
            assert len(seq) > p
            for a in range(K):
                got = g.decrypt(ranks[a])[0]
                for c in range(cols):
                    i = a * cols + c
                    want = sum(1 for j, v in enumerate(seq) if v < seq[i] or (v == seq[i] and j < i)) % p
                    assert got[r * cols + c] == want
        xo = [[o.encrypt_slots([vals[a]], seed=2000 + a)[0]] for a in range(K)]
        ev = o.evaluator()
        ranks_o, mat_o = sort_ranks(ev, xo)
        assert sorted(trace_g) == sorted(ev.trace)
        for a in range(K):
            _same(ranks_o[a], g.export(ranks[a]), 0)
        assert set(mat) == set(mat_o)
        for key in list(mat)[::5]:
            _same(mat_o[key], g.export(mat[key]), 0)
    finally:
        g.close()
