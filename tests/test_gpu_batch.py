"""GPU: uneven batches (fhe_batch_submit) give, job by job, the bits of the
same job run alone; mixed ring degrees, plaintext primes, digit counts and
levels in one submission."""
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


def test_uneven_batch_matches_alone():
    from paper_2407_07308_gb300 import fhe

    specs = [(12, 17), (13, 257)]  # (logN, p)
    ctxs = []
    rnd = random.Random(3)
    try:
        for logN, p in specs:
            ctx = fhe.fhe_ctx_create(logN, p, 12, 4, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
            sk, pk = fhe.fhe_keygen(ctx, 10 + logN)
            evk = fhe.fhe_evk_create(ctx, sk, [], 20 + logN)
            ctxs.append((ctx, sk, pk, evk, p, fhe.fhe_ctx_info(ctx).slots))
        jobs, meta, handles = [], [], []
        for i in range(10):
            ctx, sk, pk, evk, p, ns = ctxs[i % 2]
            b = (p + 1) // 2
            d = 1 + rnd.randrange(2)
            count = 1 + rnd.randrange(3)
            level = rnd.choice([12, 11, 10]) if p == 17 else 12
            xv = np.array([[rnd.randrange(b ** d) for _ in range(ns)] for _ in range(count)])
            yv = np.array([[x if rnd.random() < 0.3 else rnd.randrange(b ** d) for x in row] for row in xv])
            xs, ys = [], []
            for k in range(d):
                xk = fhe.fhe_encrypt(ctx, pk, (xv // b ** k) % b, 100 * i + k)
                yk = fhe.fhe_encrypt(ctx, pk, (yv // b ** k) % b, 100 * i + 50 + k)
                if level < 12:
                    xk2, yk2 = fhe.fhe_mod_switch(ctx, xk, level), fhe.fhe_mod_switch(ctx, yk, level)
                    handles += [xk, yk]
                    xk, yk = xk2, yk2
                xs.append(xk)
                ys.append(yk)
                handles += [xk, yk]
            kind = fhe.FHE_JOB_MAXMIN if i % 3 == 2 else fhe.FHE_JOB_COMPARE
            jobs.append(fhe.Job(ctx, evk, kind, xs, ys))
            meta.append((ctx, sk, evk, kind, xs, ys, xv, yv, b, d))
        batch = fhe.fhe_batch_submit(jobs)
        assert fhe.fhe_batch_wait(batch, 120000) == 0
        fhe.fhe_batch_destroy(batch)
        for job, (ctx, sk, evk, kind, xs, ys, xv, yv, b, d) in zip(jobs, meta):
            if kind == fhe.FHE_JOB_COMPARE:
                lt, eq = fhe.fhe_compare(ctx, evk, xs, ys)
                assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out0[0]), fhe.fhe_ct_export_coeff(ctx, lt))
                assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out1[0]), fhe.fhe_ct_export_coeff(ctx, eq))
                assert (fhe.fhe_decrypt(ctx, sk, job.out0[0]) == (xv < yv)).all()
                assert (fhe.fhe_decrypt(ctx, sk, job.out1[0]) == (xv == yv)).all()
                handles += [lt, eq] + job.out0 + job.out1
            else:
                mx, mn = fhe.fhe_max_min(ctx, evk, xs, ys)
                for k in range(d):
                    assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out0[k]),
                                          fhe.fhe_ct_export_coeff(ctx, mx[k]))
                    assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out1[k]),
                                          fhe.fhe_ct_export_coeff(ctx, mn[k]))
                got = sum(fhe.fhe_decrypt(ctx, sk, job.out0[k]).astype(np.int64) * b ** k for k in range(d))
                assert (got == np.maximum(xv, yv)).all()
                handles += mx + mn + job.out0 + job.out1
        for h in handles:
            fhe.fhe_ct_destroy(h)
    finally:
        for ctx, sk, pk, evk, _, _ in ctxs:
            fhe.fhe_evk_destroy(evk)
            fhe.fhe_sk_destroy(sk)
            fhe.fhe_pk_destroy(pk)
            fhe.fhe_ctx_destroy(ctx)


def test_batch_wait_timeout_is_bounded():
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(14, 131, 10, 3, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        sk, pk = fhe.fhe_keygen(ctx, 1)
        evk = fhe.fhe_evk_create(ctx, sk, [], 2)
        ns = fhe.fhe_ctx_info(ctx).slots
        v = np.zeros((16, ns), dtype=np.uint64)
        xs = [fhe.fhe_encrypt(ctx, pk, v, 3 + k) for k in range(2)]
        ys = [fhe.fhe_encrypt(ctx, pk, v, 5 + k) for k in range(2)]
        job = fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, xs, ys)
        batch = fhe.fhe_batch_submit([job])
        rc = fhe.fhe_batch_wait(batch, 0)
        assert rc in (0, -6)
        assert fhe.fhe_batch_wait(batch, 120000) == 0
        fhe.fhe_batch_destroy(batch)
        assert (fhe.fhe_decrypt(ctx, sk, job.out1[0]) == 1).all()
        for h in xs + ys + job.out0 + job.out1:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        fhe.fhe_ctx_destroy(ctx)


def test_recurring_batches_are_captured_and_match_alone():
    """The same group shapes submitted again are captured into a graph and
    replayed: every submission (direct, capture, replays, after eviction)
    gives each job the bits of the job alone, for new operand values each
    time."""
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(12, 17, 8, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        sk, pk = fhe.fhe_keygen(ctx, 7)
        evk = fhe.fhe_evk_create(ctx, sk, [], 8)
        ns = fhe.fhe_ctx_info(ctx).slots
        fhe.fhe_ctx_set_batch_graphs(ctx, 1)
        rnd = np.random.default_rng(5)
        shapes = {"a": [(1, 2, 8, fhe.FHE_JOB_COMPARE), (2, 1, 7, fhe.FHE_JOB_MAXMIN), (1, 1, 8, fhe.FHE_JOB_COMPARE)],
                  "b": [(2, 2, 8, fhe.FHE_JOB_COMPARE)]}
        launches = []
        for rep, name in enumerate(["a", "a", "a", "b", "b", "a", "a", "a"]):
            jobs, metas, hs = [], [], []
            for i, (d, count, level, kind) in enumerate(shapes[name]):
                xv = rnd.integers(0, 9 ** d, size=(count, ns))
                yv = np.where(rnd.random((count, ns)) < 0.3, xv, rnd.integers(0, 9 ** d, size=(count, ns)))
                xs, ys = [], []
                for k in range(d):
                    for vals, out, sd in ((xv, xs, 100 * rep + 10 * i + k), (yv, ys, 100 * rep + 10 * i + 5 + k)):
                        h = fhe.fhe_encrypt(ctx, pk, (vals // 9 ** k) % 9, sd)
                        if level < 8:
                            h2 = fhe.fhe_mod_switch(ctx, h, level)
                            hs.append(h)
                            h = h2
                        out.append(h)
                        hs.append(h)
                jobs.append(fhe.Job(ctx, evk, kind, xs, ys))
                metas.append((kind, xs, ys, xv, yv, d))
            l0 = fhe.fhe_ctx_launches(ctx)
            b = fhe.fhe_batch_submit(jobs)
            assert fhe.fhe_batch_wait(b, 120000) == 0
            fhe.fhe_batch_destroy(b)
            launches.append(fhe.fhe_ctx_launches(ctx) - l0)
            for job, (kind, xs, ys, xv, yv, d) in zip(jobs, metas):
                if kind == fhe.FHE_JOB_COMPARE:
                    lt, eq = fhe.fhe_compare(ctx, evk, xs, ys)
                    alone = [lt, eq]
                    got = job.out0 + job.out1
                    assert (fhe.fhe_decrypt(ctx, sk, job.out0[0]) == (xv < yv)).all()
                else:
                    mx, mn = fhe.fhe_max_min(ctx, evk, xs, ys)
                    alone = mx + mn
                    got = job.out0 + job.out1
                    m = sum(fhe.fhe_decrypt(ctx, sk, job.out0[k]).astype(np.int64) * 9 ** k for k in range(d))
                    assert (m == np.maximum(xv, yv)).all()
                for a, g in zip(alone, got):
                    assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, a), fhe.fhe_ct_export_coeff(ctx, g))
                hs += alone + got
            for h in hs:
                fhe.fhe_ct_destroy(h)
        # replays count the graph's nodes; the direct runs and captures do not
        # differ by much, so only check that every run launched work
        assert all(n > 0 for n in launches)
        fhe.fhe_ctx_set_batch_graphs(ctx, 0)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        fhe.fhe_ctx_destroy(ctx)


def test_level_aligned_batch_matches_lowered_alone():
    """FHE_BATCH_ALIGN_LEVELS: jobs of one (context, kind, digits) at
    different levels share a group at the lowest of them; each result equals
    the job run alone after switching its operands down to that level."""
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(12, 17, 12, 3, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    try:
        sk, pk = fhe.fhe_keygen(ctx, 3)
        evk = fhe.fhe_evk_create(ctx, sk, [], 4)
        ns = fhe.fhe_ctx_info(ctx).slots
        rnd = np.random.default_rng(8)
        jobs, meta, hs = [], [], []
        for i, (level, d, kind) in enumerate([(12, 2, fhe.FHE_JOB_COMPARE), (10, 2, fhe.FHE_JOB_COMPARE),
                                              (11, 2, fhe.FHE_JOB_COMPARE), (9, 1, fhe.FHE_JOB_MAXMIN),
                                              (12, 1, fhe.FHE_JOB_MAXMIN)]):
            xv = rnd.integers(0, 9 ** d, size=(2, ns))
            yv = np.where(rnd.random((2, ns)) < 0.3, xv, rnd.integers(0, 9 ** d, size=(2, ns)))
            xs, ys = [], []
            for k in range(d):
                for vals, out, sd in ((xv, xs, 10 * i + k), (yv, ys, 10 * i + 5 + k)):
                    h = fhe.fhe_encrypt(ctx, pk, (vals // 9 ** k) % 9, sd)
                    if level < 12:
                        h2 = fhe.fhe_mod_switch(ctx, h, level)
                        hs.append(h)
                        h = h2
                    out.append(h)
                    hs.append(h)
            jobs.append(fhe.Job(ctx, evk, kind, xs, ys))
            meta.append((kind, xs, ys, xv, yv, d))
        b = fhe.fhe_batch_submit(jobs, fhe.FHE_BATCH_ALIGN_LEVELS)
        assert fhe.fhe_batch_wait(b, 120000) == 0
        fhe.fhe_batch_destroy(b)
        lowest = {fhe.FHE_JOB_COMPARE: 10, fhe.FHE_JOB_MAXMIN: 9}
        for job, (kind, xs, ys, xv, yv, d) in zip(jobs, meta):
            lv = lowest[kind]
            xl = [fhe.fhe_mod_switch(ctx, h, lv) for h in xs]
            yl = [fhe.fhe_mod_switch(ctx, h, lv) for h in ys]
            hs += xl + yl
            if kind == fhe.FHE_JOB_COMPARE:
                alone = list(fhe.fhe_compare(ctx, evk, xl, yl))
                assert (fhe.fhe_decrypt(ctx, sk, job.out0[0]) == (xv < yv)).all()
            else:
                mx, mn = fhe.fhe_max_min(ctx, evk, xl, yl)
                alone = mx + mn
                got = sum(fhe.fhe_decrypt(ctx, sk, job.out0[k]).astype(np.int64) * 9 ** k for k in range(d))
                assert (got == np.maximum(xv, yv)).all()
            got_h = job.out0 + job.out1
            for a, g in zip(alone, got_h):
                assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, a), fhe.fhe_ct_export_coeff(ctx, g))
            hs += alone + got_h
        for h in hs:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        fhe.fhe_ctx_destroy(ctx)


def test_sort_jobs_in_batches_and_served():
    """Sort jobs beside compare jobs: in one batch submission (two sort jobs
    of one group, concatenated) and through the serving loop, each sort
    result has the bits of fhe_sort on the job alone; a sort job on a
    p = 3 mod 8 ring is refused."""
    from paper_2407_07308_gb300 import fhe

    p, logN, d = 17, 11, 2
    b = (p + 1) // 2
    ctx = fhe.fhe_ctx_create(logN, p, 12, 4, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    bad = fhe.fhe_ctx_create(logN, 131, 6, 2, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    handles = []
    try:
        sk, pk = fhe.fhe_keygen(ctx, 3)
        evk = fhe.fhe_evk_create(ctx, sk, fhe.fhe_sort_galois(ctx), 4)
        ns = fhe.fhe_ctx_info(ctx).slots
        rnd = np.random.default_rng(8)

        def operand(count, seed):
            v = rnd.integers(0, b ** d, size=(count, ns))
            hs = [fhe.fhe_encrypt(ctx, pk, (v // b ** k) % b, seed + k) for k in range(d)]
            handles.extend(hs)
            return v, hs

        (v1, s1), (v2, s2) = operand(2, 10), operand(1, 20)
        (xv, xs), (yv, ys) = operand(2, 30), operand(2, 40)
        alone, peaks = [], []
        for hs in (s1, s2):
            fhe.fhe_ctx_sync(ctx)
            fhe.fhe_ctx_memory_peak(ctx, reset=True)
            base = fhe.fhe_ctx_memory(ctx)[1]
            out = fhe.fhe_sort(ctx, evk, hs)
            fhe.fhe_ctx_sync(ctx)
            peaks.append(fhe.fhe_ctx_memory_peak(ctx) - base)
            alone.append([fhe.fhe_ct_export_coeff(ctx, h) for h in out])
            for h in out:
                fhe.fhe_ct_destroy(h)
        jobs = [fhe.Job(ctx, evk, fhe.FHE_JOB_SORT, s1, None), fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, xs, ys),
                fhe.Job(ctx, evk, fhe.FHE_JOB_SORT, s2, None)]
        for jb, pk_ in zip((jobs[0], jobs[2]), peaks):  # the admission estimate covers the measured peak
            assert fhe.fhe_job_footprint(jb) >= pk_, (fhe.fhe_job_footprint(jb), pk_)
        bt = fhe.fhe_batch_submit(jobs)
        assert fhe.fhe_batch_wait(bt, 120000) == 0
        fhe.fhe_batch_destroy(bt)
        for jb, want in zip((jobs[0], jobs[2]), alone):
            got = [fhe.fhe_ct_export_coeff(ctx, h) for h in jb.out0]
            assert all(np.array_equal(g_, w_) for g_, w_ in zip(got, want))
        cols = ns // 2
        dec = sum(fhe.fhe_decrypt(ctx, sk, jobs[0].out0[k]).astype(np.int64) * b ** k for k in range(d))
        assert (dec == np.concatenate([np.sort(v1[:, :cols], 1), np.sort(v1[:, cols:], 1)], 1)).all()
        assert (fhe.fhe_decrypt(ctx, sk, jobs[1].out0[0]) == (xv < yv)).all()
        for jb in jobs:
            for h in (jb.out0 or []) + (jb.out1 or []):
                fhe.fhe_ct_destroy(h)
        # served
        srv = fhe.fhe_server_start(hbm_budget=0)
        try:
            js = fhe.Job(ctx, evk, fhe.FHE_JOB_SORT, s2, None)
            t = fhe.fhe_server_submit(srv, js)
            done, info = fhe.fhe_server_poll(srv, t, 120000)
            assert done and info.error == 0
            got = [fhe.fhe_ct_export_coeff(ctx, h) for h in js.out0]
            assert all(np.array_equal(g_, w_) for g_, w_ in zip(got, alone[1]))
            for h in js.out0:
                fhe.fhe_ct_destroy(h)
            assert fhe.fhe_job_footprint(js) > 0
        finally:
            fhe.fhe_server_stop(srv)
        # refused on a ring without sortable rows
        bsk, bpk = fhe.fhe_keygen(bad, 5)
        bevk = fhe.fhe_evk_create(bad, bsk, [], 6)
        bx = fhe.fhe_encrypt(bad, bpk, np.zeros((1, 2), dtype=np.uint64), 7)
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_batch_submit([fhe.Job(bad, bevk, fhe.FHE_JOB_SORT, [bx], None)])
        assert e.value.code == -9
        fhe.fhe_ct_destroy(bx)
        fhe.fhe_evk_destroy(bevk)
        fhe.fhe_sk_destroy(bsk)
        fhe.fhe_pk_destroy(bpk)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        for h in handles:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_ctx_destroy(ctx)
        fhe.fhe_ctx_destroy(bad)


def test_fused_rings_mixed_degrees_match_alone_and_oracle():
    """FHE_BATCH_FUSE_RINGS: compare and max/min jobs of three contexts of one
    plaintext prime (N = 2^13, 2^14, 2^15; digit counts 1 and 2; start levels
    8, 7 and 6) in one submission, whose circuit runs every step as one launch
    over all ring degrees: each result equals the job alone, and ciphertext 0
    of one compare job per ring degree equals the CPU oracle limb for limb;
    the same shape submitted again is captured into one graph for the three
    contexts and replayed with identical bits."""
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup
    from tests.oracle_setup import compare_many

    p, L, K = 17, 8, 4
    setups = [GpuSetup(seed=60 + n, logN=n, p=p, L=L, K=K, **CHAIN50) for n in (13, 14, 15)]
    rnd = random.Random(61)
    try:
        jobs, meta, handles, oracle_jobs = [], [], [], []
        for i in range(9):
            g = setups[i % 3]
            b, ns = (p + 1) // 2, g.ns
            d = 1 + (i // 3) % 2
            count = 2 + i % 2
            level = L - (i % 3)
            xv = [[rnd.randrange(b ** d) for _ in range(ns)] for _ in range(count)]
            yv = [[x if rnd.random() < 0.3 else rnd.randrange(b ** d) for x in row] for row in xv]
            xd = [[[(v // b ** k) % b for v in row] for row in xv] for k in range(d)]
            yd = [[[(v // b ** k) % b for v in row] for row in yv] for k in range(d)]
            sx = [700 + 10 * i + k for k in range(d)]
            sy = [800 + 10 * i + k for k in range(d)]
            xs = [g.encrypt_slots(xd[k], seed=sx[k]) for k in range(d)]
            ys = [g.encrypt_slots(yd[k], seed=sy[k]) for k in range(d)]
            if level < L:
                xs = [g.own(fhe.fhe_mod_switch(g.ctx, h, level)) for h in xs]
                ys = [g.own(fhe.fhe_mod_switch(g.ctx, h, level)) for h in ys]
            kind = fhe.FHE_JOB_MAXMIN if i in (4, 8) else fhe.FHE_JOB_COMPARE
            jobs.append(fhe.Job(g.ctx, g.evk, kind, xs, ys))
            meta.append((g, kind, xs, ys, np.array(xv), np.array(yv), b, d))
            if kind == fhe.FHE_JOB_COMPARE and i < 3:
                params = dict(logN=(13, 14, 15)[i], p=p, L=L, K=K, **CHAIN50)
                oracle_jobs.append((i, (params, 60 + params["logN"], xd, yd, sx, sy, 0,
                                        level if level < L else None)))
        batch = fhe.fhe_batch_submit(jobs, fhe.FHE_BATCH_FUSE_RINGS)
        assert fhe.fhe_batch_wait(batch, 300000) == 0
        for i in range(len(jobs)):
            assert fhe.fhe_batch_job_done(batch, i)
        fhe.fhe_batch_destroy(batch)
        # the same shape twice more: captured into one graph for the three
        # contexts, then replayed; identical bits every time
        first = [[m[0].export(h) for h in (job.out0 or []) + (job.out1 or []) if h] for job, m in zip(jobs, meta)]
        for rep in range(2):
            again = [fhe.Job(m[0].ctx, m[0].evk, m[1], m[2], m[3]) for m in meta]
            bt = fhe.fhe_batch_submit(again, fhe.FHE_BATCH_FUSE_RINGS)
            assert fhe.fhe_batch_wait(bt, 300000) == 0
            fhe.fhe_batch_destroy(bt)
            for job, m, want in zip(again, meta, first):
                outs = [h for h in (job.out0 or []) + (job.out1 or []) if h]
                for h in outs:
                    m[0].own(h)
                assert all(np.array_equal(m[0].export(h), w) for h, w in zip(outs, want)), rep
        for job, (g, kind, xs, ys, xv, yv, b, d) in zip(jobs, meta):
            outs = [h for h in (job.out0 or []) + (job.out1 or []) if h]
            for h in outs:
                g.own(h)
            if kind == fhe.FHE_JOB_COMPARE:
                lt, eq = fhe.fhe_compare(g.ctx, g.evk, xs, ys)
                g.own(lt)
                g.own(eq)
                assert np.array_equal(g.export(job.out0[0]), g.export(lt))
                assert np.array_equal(g.export(job.out1[0]), g.export(eq))
                assert (g.decrypt(job.out0[0]) == (xv < yv)).all()
                assert (g.decrypt(job.out1[0]) == (xv == yv)).all()
            else:
                mx, mn = fhe.fhe_max_min(g.ctx, g.evk, xs, ys)
                for h in mx + mn:
                    g.own(h)
                for k in range(d):
                    assert np.array_equal(g.export(job.out0[k]), g.export(mx[k]))
                    assert np.array_equal(g.export(job.out1[k]), g.export(mn[k]))
                got = sum(g.decrypt(job.out0[k]).astype(np.int64) * b ** k for k in range(d))
                assert (got == np.maximum(xv, yv)).all()
        res = compare_many([oj for _, oj in oracle_jobs])
        for (i, _), (want_lt, want_eq, _) in zip(oracle_jobs, res):
            g = meta[i][0]
            assert np.array_equal(g.export(jobs[i].out0[0])[0], want_lt), i
            assert np.array_equal(g.export(jobs[i].out1[0])[0], want_eq), i
    finally:
        for g in setups:
            g.close()
