"""GPU: the serving loop (fhe_server_*) returns, request by request, the bits
of the same request run alone; requests arrive from another thread while
earlier batches run; admission keeps the estimated footprint of the admitted
requests within the budget, and the estimate covers what a request really
allocates."""
import random
import threading
import time

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


def _contexts(fhe, specs, L=10, K=3):
    import gc

    out = []
    for logN, p in specs:
        # the allocator object is a temporary here: the binding keeps its
        # callbacks alive for the context's lifetime
        ctx = fhe.fhe_ctx_create(logN, p, L, K, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"],
                                 allocator=fhe.torch_allocator(0))
        gc.collect()
        sk, pk = fhe.fhe_keygen(ctx, 30 + logN + p)
        evk = fhe.fhe_evk_create(ctx, sk, [], 40 + logN + p)
        out.append((ctx, sk, pk, evk, p, fhe.fhe_ctx_info(ctx).slots))
    return out


def _close(fhe, ctxs):
    for ctx, sk, pk, evk, _, _ in ctxs:
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
        fhe.fhe_ctx_destroy(ctx)


def _request(fhe, rnd, i, c, L, handles):
    ctx, sk, pk, evk, p, ns = c
    b = (p + 1) // 2
    d = 1 + rnd.randrange(2)
    count = 1 + rnd.randrange(3)
    level = rnd.choice([L, L - 1])
    xv = np.array([[rnd.randrange(b ** d) for _ in range(ns)] for _ in range(count)])
    yv = np.array([[x if rnd.random() < 0.3 else rnd.randrange(b ** d) for x in row] for row in xv])
    xs, ys = [], []
    for k in range(d):
        xk = fhe.fhe_encrypt(ctx, pk, (xv // b ** k) % b, 1000 * i + k)
        yk = fhe.fhe_encrypt(ctx, pk, (yv // b ** k) % b, 1000 * i + 500 + k)
        if level < L:
            handles += [xk, yk]
            xk, yk = fhe.fhe_mod_switch(ctx, xk, level), fhe.fhe_mod_switch(ctx, yk, level)
        xs.append(xk)
        ys.append(yk)
        handles += [xk, yk]
    kind = fhe.FHE_JOB_MAXMIN if i % 4 == 3 else fhe.FHE_JOB_COMPARE
    return fhe.Job(ctx, evk, kind, xs, ys), (c, kind, xs, ys, xv, yv, b, d)


def _check_alone(fhe, job, meta, handles):
    (ctx, sk, pk, evk, p, ns), kind, xs, ys, xv, yv, b, d = meta
    if kind == fhe.FHE_JOB_COMPARE:
        lt, eq = fhe.fhe_compare(ctx, evk, xs, ys)
        handles += [lt, eq] + job.out0 + job.out1
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out0[0]), fhe.fhe_ct_export_coeff(ctx, lt))
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out1[0]), fhe.fhe_ct_export_coeff(ctx, eq))
        assert (fhe.fhe_decrypt(ctx, sk, job.out0[0]) == (xv < yv)).all()
        assert (fhe.fhe_decrypt(ctx, sk, job.out1[0]) == (xv == yv)).all()
    else:
        mx, mn = fhe.fhe_max_min(ctx, evk, xs, ys)
        handles += mx + mn + job.out0 + job.out1
        for k in range(d):
            assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out0[k]), fhe.fhe_ct_export_coeff(ctx, mx[k]))
            assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, job.out1[k]), fhe.fhe_ct_export_coeff(ctx, mn[k]))
        got = sum(fhe.fhe_decrypt(ctx, sk, job.out1[k]).astype(np.int64) * b ** k for k in range(d))
        assert (got == np.minimum(xv, yv)).all()


def test_server_mix_matches_alone_within_budget():
    from paper_2407_07308_gb300 import fhe

    L = 10
    ctxs = _contexts(fhe, [(11, 17), (12, 257)], L=L)
    handles = []
    rnd = random.Random(9)
    try:
        reqs = [_request(fhe, rnd, i, ctxs[i % 2], L, handles) for i in range(12)]
        foot = [fhe.fhe_job_footprint(j) for j, _ in reqs]
        assert min(foot) > 0
        budget = int(2.5 * max(foot))
        srv = fhe.fhe_server_start(hbm_budget=budget)
        tickets = [None] * len(reqs)

        def client():
            for i, (j, _) in enumerate(reqs):
                tickets[i] = fhe.fhe_server_submit(srv, j)
                time.sleep(rnd.random() * 0.004)

        th = threading.Thread(target=client)
        th.start()
        th.join()
        infos = []
        for t in tickets:
            done, info = fhe.fhe_server_poll(srv, t, 120000)
            assert done and info.state == fhe.FHE_REQ_DONE and info.error == 0
            assert info.t_submit_ms <= info.t_start_ms <= info.t_done_ms
            infos.append(info)
        st = fhe.fhe_server_stats(srv)
        assert st.completed == len(reqs) and st.failed == 0 and st.queued == 0 and st.running == 0
        assert 1 <= st.batches <= len(reqs)
        assert st.admitted_peak_bytes <= budget and st.admitted_bytes == 0
        with pytest.raises(fhe.FheError):
            fhe.fhe_server_poll(srv, tickets[0])  # retired
        fhe.fhe_server_stop(srv)
        for j, meta in reqs:
            _check_alone(fhe, j, meta, handles)
    finally:
        for h in handles:
            fhe.fhe_ct_destroy(h)
        _close(fhe, ctxs)


@pytest.mark.parametrize("logN,p,d,count,kind", [(13, 131, 1, 1, 1), (13, 131, 2, 3, 1), (12, 17, 3, 2, 2),
                                                 (12, 257, 2, 4, 2)])
def test_footprint_covers_peak(logN, p, d, count, kind):
    """What one request allocates (the pool's peak) stays within its
    estimate; a budget below the estimate refuses it."""
    from paper_2407_07308_gb300 import fhe

    L = 10
    ctxs = _contexts(fhe, [(logN, p)], L=L)
    ctx, sk, pk, evk, _, ns = ctxs[0]
    b = (p + 1) // 2
    hs = []
    try:
        rng = np.random.default_rng(logN + p + d)
        xv = rng.integers(0, b ** d, size=(count, ns))
        yv = rng.integers(0, b ** d, size=(count, ns))
        xs = [fhe.fhe_encrypt(ctx, pk, (xv // b ** k) % b, 10 + k) for k in range(d)]
        ys = [fhe.fhe_encrypt(ctx, pk, (yv // b ** k) % b, 20 + k) for k in range(d)]
        hs += xs + ys
        job = fhe.Job(ctx, evk, kind, xs, ys)
        foot = fhe.fhe_job_footprint(job)
        srv = fhe.fhe_server_start(hbm_budget=foot - 1)
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_server_submit(srv, job)
        assert e.value.code == -5  # FHE_EBUDGET
        fhe.fhe_server_stop(srv)
        fhe.fhe_ctx_sync(ctx)
        base = fhe.fhe_ctx_memory(ctx)[1]
        fhe.fhe_ctx_memory_peak(ctx, reset=True)
        srv = fhe.fhe_server_start(hbm_budget=foot)
        t = fhe.fhe_server_submit(srv, job)
        done, info = fhe.fhe_server_poll(srv, t, 120000)
        assert done and info.error == 0 and info.est_bytes == foot
        fhe.fhe_server_stop(srv)
        hs += job.out0 + job.out1
        peak = fhe.fhe_ctx_memory_peak(ctx)
        print(f"footprint {foot / 1e6:.1f} MB, peak {(peak - base) / 1e6:.1f} MB")
        assert 0 < peak - base <= foot
    finally:
        for h in hs:
            fhe.fhe_ct_destroy(h)
        _close(fhe, ctxs)


def test_lowest_level_p257_decrypts():
    """p = 257 at N = 2^14: one digit compared from level 10, where the
    polynomial's last product falls on the second prime, decrypts
    correctly."""
    from paper_2407_07308_gb300 import fhe

    ctxs = _contexts(fhe, [(14, 257)], L=20, K=4)
    ctx, sk, pk, evk, _, ns = ctxs[0]
    hs = []
    try:
        rng = np.random.default_rng(1)
        xv = rng.integers(0, 129, size=(4, ns))
        yv = np.where(rng.random((4, ns)) < 0.3, xv, rng.integers(0, 129, size=(4, ns)))
        x0, y0 = fhe.fhe_encrypt(ctx, pk, xv, 1), fhe.fhe_encrypt(ctx, pk, yv, 2)
        x, y = fhe.fhe_mod_switch(ctx, x0, 10), fhe.fhe_mod_switch(ctx, y0, 10)
        lt, eq = fhe.fhe_compare(ctx, evk, [x], [y])
        hs += [x0, y0, x, y, lt, eq]
        assert (fhe.fhe_decrypt(ctx, sk, lt) == (xv < yv)).all()
        assert (fhe.fhe_decrypt(ctx, sk, eq) == (xv == yv)).all()
    finally:
        for h in hs:
            fhe.fhe_ct_destroy(h)
        _close(fhe, ctxs)


def test_errors_are_reported_and_context_recovers():
    """A device allocation that fails mid-circuit (host-side injection) and a
    context memory budget that is too small end the call with FHE_ENOMEM /
    FHE_EBUDGET; the context keeps working, and a served request that fails
    reports its error while the next ones are served."""
    from paper_2407_07308_gb300 import fhe

    ctxs = _contexts(fhe, [(12, 17)], L=8, K=2)
    ctx, sk, pk, evk, _, ns = ctxs[0]
    hs = []
    try:
        rng = np.random.default_rng(3)
        xv, yv = rng.integers(0, 9, size=(2, ns)), rng.integers(0, 9, size=(2, ns))
        x, y = fhe.fhe_encrypt(ctx, pk, xv, 1), fhe.fhe_encrypt(ctx, pk, yv, 2)
        hs += [x, y]
        lt0, eq0 = fhe.fhe_compare(ctx, evk, [x], [y])
        hs += [lt0, eq0]
        ref = fhe.fhe_ct_export_coeff(ctx, lt0)
        fhe.fhe_ctx_sync(ctx)
        fhe.fhe_ctx_set_budget(ctx, 1)  # nothing new fits
        with pytest.raises(fhe.FheError) as e:
            for _ in range(3):  # cached blocks may serve the first call
                a, b = fhe.fhe_compare(ctx, evk, [x], [y])
                hs += [a, b]
        assert e.value.code == -5
        fhe.fhe_ctx_set_budget(ctx, 0)
        fhe.fhe_ctx_memory_peak(ctx, reset=True)
        # fail the 3rd new block from now on, after dropping the cache
        fhe.fhe_ctx_trim(ctx)
        fhe.fhe_ctx_inject_alloc_failure(ctx, 2)
        with pytest.raises(fhe.FheError) as e:
            a, b = fhe.fhe_compare(ctx, evk, [x], [y])
            hs += [a, b]
        assert e.value.code == -4
        fhe.fhe_ctx_inject_alloc_failure(ctx, -1)
        lt1, eq1 = fhe.fhe_compare(ctx, evk, [x], [y])
        hs += [lt1, eq1]
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, lt1), ref)
        # the server: one failing request, then normal service
        srv = fhe.fhe_server_start()
        fhe.fhe_ctx_trim(ctx)
        fhe.fhe_ctx_inject_alloc_failure(ctx, 0)
        j1 = fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, [x], [y])
        t1 = fhe.fhe_server_submit(srv, j1)
        done, info = fhe.fhe_server_poll(srv, t1, 60000)
        assert done and info.error == -4
        fhe.fhe_ctx_inject_alloc_failure(ctx, -1)
        j2 = fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, [x], [y])
        t2 = fhe.fhe_server_submit(srv, j2)
        done, info = fhe.fhe_server_poll(srv, t2, 60000)
        assert done and info.error == 0
        hs += j2.out0 + j2.out1
        assert np.array_equal(fhe.fhe_ct_export_coeff(ctx, j2.out0[0]), ref)
        st = fhe.fhe_server_stats(srv)
        assert st.completed == 2 and st.failed == 1
        fhe.fhe_server_stop(srv)
    finally:
        fhe.fhe_ctx_inject_alloc_failure(ctx, -1)
        for h in hs:
            if h:
                fhe.fhe_ct_destroy(h)
        _close(fhe, ctxs)


def test_queued_request_is_canceled():
    """A request held back by the memory budget is canceled while the one
    before it runs: it reports done with FHE_ECANCELED and no outputs; the
    running one completes; canceling a finished request answers FHE_EBUSY."""
    from paper_2407_07308_gb300 import fhe

    ctx = fhe.fhe_ctx_create(14, 131, 10, 3, CHAIN50["U"], CHAIN50["lo"], CHAIN50["hi"])
    handles = []
    try:
        sk, pk = fhe.fhe_keygen(ctx, 1)
        evk = fhe.fhe_evk_create(ctx, sk, [], 2)
        ns = fhe.fhe_ctx_info(ctx).slots
        rnd = np.random.default_rng(3)
        xv, yv = rnd.integers(0, 66 ** 2, size=(2, 16, ns))
        ops = []
        for vals, sd in ((xv, 10), (yv, 20)):
            hs = [fhe.fhe_encrypt(ctx, pk, (vals // 66 ** k) % 66, sd + k) for k in range(2)]
            handles += hs
            ops.append(hs)
        j1 = fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, ops[0], ops[1])
        j2 = fhe.Job(ctx, evk, fhe.FHE_JOB_COMPARE, ops[0], ops[1])
        srv = fhe.fhe_server_start(hbm_budget=fhe.fhe_job_footprint(j1))  # one request at a time
        try:
            t1 = fhe.fhe_server_submit(srv, j1)
            t2 = fhe.fhe_server_submit(srv, j2)
            t0 = time.time()
            while fhe.fhe_server_poll(srv, t1, 0)[1].state == fhe.FHE_REQ_QUEUED and time.time() - t0 < 10:
                time.sleep(0.0005)
            assert fhe.fhe_server_cancel(srv, t2) == 0  # j2 waits for j1's memory
            assert fhe.fhe_server_cancel(srv, t1) == -11  # admitted: runs to completion
            done, info = fhe.fhe_server_poll(srv, t2, 0)
            assert done and info.error == -10
            done, info = fhe.fhe_server_poll(srv, t1, 120000)
            assert done and info.error == 0
            assert (fhe.fhe_decrypt(ctx, sk, j1.out0[0]) == (xv < yv)).all()
            assert j2.out0[0].value is None  # nothing written
            with pytest.raises(fhe.FheError):  # retired once reported done
                fhe.fhe_server_cancel(srv, t1)
        finally:
            fhe.fhe_server_stop(srv)
        for h in j1.out0 + j1.out1:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_evk_destroy(evk)
        fhe.fhe_sk_destroy(sk)
        fhe.fhe_pk_destroy(pk)
    finally:
        for h in handles:
            fhe.fhe_ct_destroy(h)
        fhe.fhe_ctx_destroy(ctx)
