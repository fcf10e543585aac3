"""GPU parity on the rings and prime chains of every workload: the CUDA path
through its C ABI against the CPU oracle on identical seeded inputs, limb for
limb (tolerance 0: exact integer arithmetic).

- the tournament chain (N = 2^15, p = 257, 20 + 4 primes, five key-switching
  digits): one relinearised product, the rotations sigma_5 and sigma_{2N-1}
  and a three-prime modulus switch;
- the uneven workload's smallest ring (N = 2^13, p = 131 and 257, the same
  20 + 4 chain): the same operations, a product at a level with a short last
  digit, and a whole one-digit comparison from a lowered start level;
- the benchmark's batch (N = 2^14, p = 131, d = 2, 16 pairs): ciphertexts 0,
  7 and 15 of both the direct call and the captured plan the benchmark
  replays.
"""
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


def _fhe():
    from paper_2407_07308_gb300 import fhe

    return fhe


def _pair(params, seed, galois=()):
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import OracleSetup

    o = OracleSetup(seed=seed, galois=galois, **params)
    g = GpuSetup(seed=seed, galois=galois, **params)
    assert g.primes == o.o.primes
    return o, g


def _ops_bitexact(params, seed, low_level):
    """mul_relin, both rotations and a three-prime switch, at the top level
    and (product and rotation) again at `low_level`."""
    fhe = _fhe()
    N = 1 << params["logN"]
    galois = (5, 2 * N - 1)
    o, g = _pair(params, seed, galois)
    try:
        p, L = params["p"], params["L"]
        rnd = random.Random(seed)
        a = [rnd.randrange(p) for _ in range(g.ns)]
        b = [rnd.randrange(p) for _ in range(g.ns)]
        ca_o, cb_o = o.encrypt_slots([a, b], seed=11)
        ca_g, cb_g = g.encrypt_each([a, b], seed=11)
        ev = o.evaluator()
        oc, X = o.o, g.ctx
        checks = [("mul_relin", ev.mul(ca_o, cb_o), fhe.fhe_mul_relin(X, g.evk, ca_g, cb_g))]
        for gal in galois:
            checks.append((f"rot{gal}", oc.rotate(ca_o, gal, o.gks[gal]), fhe.fhe_rotate(X, g.evk, ca_g, gal)))
        checks.append(("switch3", oc.modswitch(oc.modswitch(oc.modswitch(ca_o))), fhe.fhe_mod_switch(X, ca_g, L - 3)))
        la_o, lb_o = ev.lower(ca_o, low_level), ev.lower(cb_o, low_level)
        la_g = g.own(fhe.fhe_mod_switch(X, ca_g, low_level))
        lb_g = g.own(fhe.fhe_mod_switch(X, cb_g, low_level))
        checks.append(("lowered", la_o, la_g))
        checks.append(("mul_relin_low", ev.mul(la_o, lb_o), fhe.fhe_mul_relin(X, g.evk, la_g, lb_g)))
        checks.append(("rot5_low", oc.rotate(la_o, 5, o.gks[5]), fhe.fhe_rotate(X, g.evk, la_g, 5)))
        for name, want, got in checks:
            if got is not la_g:
                g.own(got)
            assert np.array_equal(g.export(got)[0], want.data), name
        dec = g.decrypt(checks[0][2])[0].tolist()
        assert dec == [(x * y) % p for x, y in zip(a, b)]
    finally:
        g.close()


def test_tournament_chain_ops_bitexact():
    """N = 2^15, p = 257, 20 + 4 primes (dnum = 5); the low level 9 leaves a
    short last digit (9 = 4 + 4 + 1)."""
    _ops_bitexact(dict(logN=15, p=257, L=20, K=4, **CHAIN50), seed=41, low_level=9)


@pytest.mark.parametrize("p", [131, 257])
def test_uneven_ring_ops_bitexact(p):
    """N = 2^13 on the universal 20 + 4 chain (the uneven workload's smallest
    ring); low level 10 (= 4 + 4 + 2)."""
    _ops_bitexact(dict(logN=13, p=p, L=20, K=4, **CHAIN50), seed=42 + p, low_level=10)


@pytest.mark.parametrize("p,level", [(131, 9), (257, 11)])
def test_uneven_ring_compare_d1_bitexact(p, level):
    """One-digit LT and EQ on N = 2^13 (20 + 4 chain) from a lowered start
    level, 4 ciphertexts per batch: ciphertexts 0 and 3 bit-exact with the
    oracle, the trace equal, every slot against plaintext."""
    from tests.oracle_setup import compare_many

    fhe = _fhe()
    params = dict(logN=13, p=p, L=20, K=4, **CHAIN50)
    seed = 50 + p
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=seed, **params)
    try:
        b = (p + 1) // 2
        rnd = random.Random(seed)
        count = 4
        xv = [[rnd.randrange(b) for _ in range(g.ns)] for _ in range(count)]
        yv = [[x if rnd.random() < 0.3 else rnd.randrange(b) for x in row] for row in xv]
        xg = g.own(fhe.fhe_mod_switch(g.ctx, g.encrypt_slots(xv, seed=100), level))
        yg = g.own(fhe.fhe_mod_switch(g.ctx, g.encrypt_slots(yv, seed=200), level))
        fhe.fhe_trace_enable(g.ctx, True)
        lt, eq = fhe.fhe_compare(g.ctx, g.evk, [xg], [yg])
        g.own(lt)
        g.own(eq)
        trace = fhe.fhe_trace_get(g.ctx)
        fhe.fhe_trace_enable(g.ctx, False)
        lt_d, eq_d = g.decrypt(lt), g.decrypt(eq)
        for c in range(count):
            assert lt_d[c].tolist() == [int(x < y) for x, y in zip(xv[c], yv[c])]
            assert eq_d[c].tolist() == [int(x == y) for x, y in zip(xv[c], yv[c])]
        ex_lt, ex_eq = g.export(lt), g.export(eq)
        idx = (0, count - 1)
        res = compare_many([(params, seed, [xv], [yv], [100], [200], i, level) for i in idx])
        for i, (want_lt, want_eq, want_trace) in zip(idx, res):
            assert np.array_equal(ex_lt[i], want_lt), i
            assert np.array_equal(ex_eq[i], want_eq), i
            assert sorted(trace) == sorted(want_trace)
    finally:
        g.close()


def test_benchmark_batch_and_plan_bitexact():
    """The benchmark's workload: N = 2^14, p = 131, d = 2, 16 pairs, 10 + 3
    primes.  Ciphertexts 0, 7 and 15 of the direct call and of the captured
    plan (the form the benchmark times) bit-exact with the oracle; all 16
    against plaintext."""
    from tests.oracle_setup import compare_many
    from tests.gpu_setup import GpuSetup

    fhe = _fhe()
    params = dict(logN=14, p=131, L=10, K=3, **CHAIN50)
    seed, d, count = 2, 2, 16
    g = GpuSetup(seed=seed, **params)
    try:
        b = 66
        rnd = random.Random(seed)
        xv = [[rnd.randrange(b ** d) for _ in range(g.ns)] for _ in range(count)]
        yv = [[x if rnd.random() < 0.3 else rnd.randrange(b ** d) for x in row] for row in xv]
        xd = [[[(v // b ** k) % b for v in row] for row in xv] for k in range(d)]
        yd = [[[(v // b ** k) % b for v in row] for row in yv] for k in range(d)]
        xs = [g.encrypt_slots(xd[k], seed=100 + k) for k in range(d)]
        ys = [g.encrypt_slots(yd[k], seed=200 + k) for k in range(d)]
        fhe.fhe_trace_enable(g.ctx, True)
        lt, eq = fhe.fhe_compare(g.ctx, g.evk, xs, ys)
        g.own(lt)
        g.own(eq)
        trace = fhe.fhe_trace_get(g.ctx)
        fhe.fhe_trace_enable(g.ctx, False)
        direct = (g.export(lt), g.export(eq))
        plan = fhe.fhe_compare_plan(g.ctx, g.evk, xs, ys)
        try:
            fhe.fhe_plan_run(plan, g.ctx)
            fhe.fhe_ctx_sync(g.ctx)
            planned = (g.export(fhe.fhe_plan_result(plan, 0)), g.export(fhe.fhe_plan_result(plan, 1)))
        finally:
            fhe.fhe_plan_destroy(plan)
        lt_d, eq_d = g.decrypt(lt), g.decrypt(eq)
        for c in range(count):
            assert lt_d[c].tolist() == [int(x < y) for x, y in zip(xv[c], yv[c])]
            assert eq_d[c].tolist() == [int(x == y) for x, y in zip(xv[c], yv[c])]
        idx = (0, 7, 15)
        res = compare_many([(params, seed, xd, yd, [100 + k for k in range(d)], [200 + k for k in range(d)], i, None)
                            for i in idx])
        for i, (want_lt, want_eq, want_trace) in zip(idx, res):
            assert sorted(trace) == sorted(want_trace)
            for name, (got_lt, got_eq) in (("direct", direct), ("plan", planned)):
                assert np.array_equal(got_lt[i], want_lt), (name, i)
                assert np.array_equal(got_eq[i], want_eq), (name, i)
    finally:
        g.close()
