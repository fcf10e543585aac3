// batch.cu -- many comparison requests of uneven shape in one submission.
//
// Jobs are grouped by (context, keys, kind, digits, level); each group's
// operands are concatenated into one ciphertext batch, so one kernel launch
// serves the whole group.  All groups of a context run as one circuit under
// the dependency scheduler (c->multistream), so groups of different levels
// and digit counts overlap on the device; different contexts (ring degrees,
// plaintext primes) run on their own streams.  Results are sliced back into
// per-job handles.  Completion is tracked with one event per context;
// fhe_batch_wait polls them with a deadline and never blocks without bound.
#include <string.h>

#include <chrono>
#include <map>
#include <thread>
#include <tuple>

#include "fhe_internal.h"

struct fhe_batch {
    std::vector<std::pair<fhe_ctx *, cudaEvent_t>> done;
};

namespace {

struct Group {
    const fhe_evk *evk;
    int kind, d, level;
    std::vector<int> jobs;
    std::vector<fhe_ct *> X, Y;              // concatenated operands (owned when built)
    std::vector<bool> own_x;
    std::vector<fhe_ct *> out0, out1;        // group outputs (owned, sliced to jobs)
};

}  // namespace

int batch_check_job(const fhe_job &j)
{
    if (!j.ctx || !j.evk || j.evk->ctx != j.ctx || !j.x || !j.y || j.d < 1) return FHE_EINVAL;
    if (j.kind != FHE_JOB_COMPARE && j.kind != FHE_JOB_MAXMIN) return FHE_EINVAL;
    if (!j.out0 && !j.out1) return FHE_EINVAL;
    const fhe_ct *a = j.x[0];
    if (!a) return FHE_EINVAL;
    for (int k = 0; k < j.d; k++) {
        const fhe_ct *u = j.x[k], *v = j.y[k];
        if (!u || !v || u->ctx != j.ctx || v->ctx != j.ctx) return FHE_EINVAL;
        if (u->npoly != 2 || v->npoly != 2 || u->count != a->count || v->count != a->count ||
            u->level != a->level || v->level != a->level)
            return fhe_fail(j.ctx, FHE_EMISMATCH, "batch job: operands differ in shape or level");
    }
    return 0;
}

namespace {

// concatenation of the jobs' digit-k operands (one allocation, one copy per part)
int gather(fhe_ctx *c, const fhe_job *jobs, const std::vector<int> &ids, int k, bool ys, fhe_ct **out, bool *owned)
{
    if (ids.size() == 1) {
        *out = const_cast<fhe_ct *>(ys ? jobs[ids[0]].y[k] : jobs[ids[0]].x[k]);
        *owned = false;
        return 0;
    }
    const fhe_ct *first = ys ? jobs[ids[0]].y[k] : jobs[ids[0]].x[k];
    int total = 0;
    for (int id : ids) total += (ys ? jobs[id].y[k] : jobs[id].x[k])->count;
    int err = 0;
    fhe_ct *r = ct_new(c, total, first->npoly, first->level, &err);
    if (!r) return err;
    size_t off = 0;
    for (int id : ids) {
        const fhe_ct *part = ys ? jobs[id].y[k] : jobs[id].x[k];
        cudaMemcpyAsync((char *)r->d + off, part->d, part->bytes, cudaMemcpyDeviceToDevice, c->stream);
        off += part->bytes;
    }
    *out = r;
    *owned = true;
    return 0;
}

int run_context(fhe_ctx *c, const fhe_job *jobs, const std::vector<int> &ids)
{
    std::map<std::tuple<const fhe_evk *, int, int, int, bool, bool>, Group> groups;
    for (int id : ids) {
        const fhe_job &j = jobs[id];
        auto key = std::make_tuple(j.evk, j.kind, j.d, j.x[0]->level, j.out0 != nullptr, j.out1 != nullptr);
        Group &g = groups[key];
        g.evk = j.evk;
        g.kind = j.kind;
        g.d = j.d;
        g.level = j.x[0]->level;
        g.jobs.push_back(id);
    }
    int err = 0;
    // operands
    for (auto &kv : groups) {
        Group &g = kv.second;
        g.X.assign(g.d, nullptr);
        g.Y.assign(g.d, nullptr);
        g.own_x.assign(2 * g.d, false);
        g.out0.assign(g.kind == FHE_JOB_MAXMIN ? g.d : 1, nullptr);
        g.out1.assign(g.kind == FHE_JOB_MAXMIN ? g.d : 1, nullptr);
        for (int k = 0; k < g.d && !err; k++) {
            bool o1 = false, o2 = false;
            err = gather(c, jobs, g.jobs, k, false, &g.X[k], &o1);
            if (!err) err = gather(c, jobs, g.jobs, k, true, &g.Y[k], &o2);
            g.own_x[k] = o1;
            g.own_x[g.d + k] = o2;
        }
        if (err) break;
    }
    // one circuit per key set; with multistream the groups overlap
    std::map<const fhe_evk *, std::vector<MultiItem>> by_evk;
    if (!err)
        for (auto &kv : groups) {
            Group &g = kv.second;
            const fhe_job &j0 = jobs[g.jobs[0]];
            MultiItem it;
            it.x = g.X.data();
            it.y = g.Y.data();
            it.d = g.d;
            it.maxmin = g.kind == FHE_JOB_MAXMIN;
            it.out0 = j0.out0 ? g.out0.data() : nullptr;
            it.out1 = j0.out1 ? g.out1.data() : nullptr;
            by_evk[g.evk].push_back(it);
        }
    c->multistream = true;
    for (auto &kv : by_evk) {
        if (err) break;
        err = circuit_multi(c, kv.first, kv.second);
    }
    c->multistream = false;
    // results back to the jobs
    for (auto &kv : groups) {
        Group &g = kv.second;
        int off = 0;
        for (int id : g.jobs) {
            const fhe_job &j = jobs[id];
            const int cnt = j.x[0]->count;
            for (int s = 0; s < 2 && !err; s++) {
                fhe_ct **dst = s == 0 ? j.out0 : j.out1;
                std::vector<fhe_ct *> &src = s == 0 ? g.out0 : g.out1;
                if (!dst) continue;
                for (size_t k = 0; k < src.size() && !err; k++) {
                    if (!src[k]) continue;
                    if (g.jobs.size() == 1) {
                        dst[k] = src[k];
                        src[k] = nullptr;
                    } else {
                        err = op_slice(c, src[k], off, cnt, &dst[k]);
                    }
                }
            }
            off += cnt;
        }
        for (fhe_ct *x : g.out0) fhe_ct_destroy(x);
        for (fhe_ct *x : g.out1) fhe_ct_destroy(x);
        for (int k = 0; k < 2 * g.d; k++)
            if (g.own_x[k]) fhe_ct_destroy(k < g.d ? g.X[k] : g.Y[k - g.d]);
    }
    return err;
}

}  // namespace

extern "C" int fhe_batch_submit(const fhe_job *jobs, int n, fhe_batch **out)
{
    if (!jobs || n < 1 || !out) return FHE_EINVAL;
    for (int i = 0; i < n; i++) {
        int e = batch_check_job(jobs[i]);
        if (e) return e;
    }
    std::vector<fhe_ctx *> order;
    std::map<fhe_ctx *, std::vector<int>> by_ctx;
    for (int i = 0; i < n; i++) {
        if (!by_ctx.count(jobs[i].ctx)) order.push_back(jobs[i].ctx);
        by_ctx[jobs[i].ctx].push_back(i);
    }
    fhe_batch *B = new fhe_batch;
    int err = 0;
    for (fhe_ctx *c : order) {
        std::lock_guard<std::mutex> g(c->mu);
        err = run_context(c, jobs, by_ctx[c]);
        cudaEvent_t ev = nullptr;
        if (!err) err = fhe_cuda_check(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch event");
        if (!err) err = fhe_cuda_check(c, cudaEventRecord(ev, c->stream), "batch event");
        if (ev) B->done.push_back({c, ev});
        if (err) break;
    }
    if (err) {
        fhe_batch_destroy(B);
        return err;
    }
    *out = B;
    return 0;
}

extern "C" int fhe_batch_wait(fhe_batch *B, int timeout_ms)
{
    if (!B) return FHE_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        bool all = true;
        for (auto &d : B->done) {
            const cudaError_t q = cudaEventQuery(d.second);
            if (q == cudaErrorNotReady) {
                all = false;
                break;
            }
            if (q != cudaSuccess) return fhe_cuda_check(d.first, q, "batch wait");
        }
        if (all) return 0;
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms) return FHE_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" void fhe_batch_destroy(fhe_batch *B)
{
    if (!B) return;
    for (auto &d : B->done) {
        cudaEventSynchronize(d.second);
        cudaEventDestroy(d.second);
    }
    delete B;
}
