// batch.cu -- many comparison requests of uneven shape in one submission.
//
// Jobs are grouped by (context, keys, kind, digits, level); each group's
// operands are concatenated into one ciphertext batch, so one kernel launch
// serves the whole group.  All groups of a context run as one circuit under
// the dependency scheduler (c->multistream), so groups of different levels
// and digit counts overlap on the device; different contexts (ring degrees,
// plaintext primes) run on their own streams.  Results are sliced back into
// per-job handles.  A context that receives a submission of the same group
// shapes again captures the circuit once into a CUDA graph with its own
// operand and result buffers and from then on copies the operands in,
// replays the graph and slices the results out.  Completion is tracked with
// one event per context; fhe_batch_wait polls them with a deadline and never
// blocks without bound.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <set>
#include <mutex>
#include <thread>
#include <tuple>

#include "fhe_internal.h"

struct fhe_batch {
    std::vector<std::pair<fhe_ctx *, cudaEvent_t>> done;  // every event of the batch
    std::vector<int> job_event;                          // per job: its index into done
};

// Whether job i of the batch has its results (its context's compare phase,
// or for a sort job its sort phase, has completed): 1 done, 0 not yet, or a
// negative error.
int batch_job_done(fhe_batch *B, int i)
{
    if (!B || i < 0 || i >= (int)B->job_event.size()) return FHE_EINVAL;
    const auto &d = B->done[B->job_event[i]];
    const cudaError_t q = cudaEventQuery(d.second);
    if (q == cudaErrorNotReady) return 0;
    return q == cudaSuccess ? 1 : fhe_cuda_check(d.first, q, "batch job");
}

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
    const bool sort = j.kind == FHE_JOB_SORT;
    if (!j.ctx || !j.evk || j.evk->ctx != j.ctx || !j.x || (!sort && !j.y) || j.d < 1) return FHE_EINVAL;
    if (j.kind != FHE_JOB_COMPARE && j.kind != FHE_JOB_MAXMIN && !sort) return FHE_EINVAL;
    if (!j.out0 && !j.out1) return FHE_EINVAL;
    if (sort && (!j.out0 || j.out1)) return FHE_EINVAL;
    if (sort && (!j.ctx->slots_linear || j.ctx->ns < 4))
        return fhe_fail(j.ctx, FHE_EUNSUPPORTED, "batch job: sorting needs p = 1 mod 4");
    const fhe_ct *a = j.x[0];
    if (!a) return FHE_EINVAL;
    for (int k = 0; k < j.d; k++) {
        const fhe_ct *u = j.x[k], *v = sort ? a : j.y[k];
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

using GroupMap = std::map<std::tuple<const fhe_evk *, int, int, int, bool, bool>, Group>;

GroupMap make_groups(const fhe_job *jobs, const std::vector<int> &ids)
{
    GroupMap groups;
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
    return groups;
}

// shape of a context's submission: per group (keys, kind, digits, level,
// ciphertexts, wanted outputs)
std::vector<u64> signature(const fhe_job *jobs, const GroupMap &groups)
{
    std::vector<u64> sig;
    for (auto &kv : groups) {
        const Group &g = kv.second;
        u64 cnt = 0;
        for (int id : g.jobs) cnt += jobs[id].x[0]->count;
        const fhe_job &j0 = jobs[g.jobs[0]];
        sig.insert(sig.end(), {(u64)(uintptr_t)g.evk, (u64)g.kind, (u64)g.d, (u64)g.level, cnt,
                               (u64)(j0.out0 != nullptr), (u64)(j0.out1 != nullptr)});
    }
    return sig;
}

std::vector<MultiItem> items_for(Group &g, const fhe_job &j0, std::vector<fhe_ct *> &X, std::vector<fhe_ct *> &Y,
                                 std::vector<fhe_ct *> &O0, std::vector<fhe_ct *> &O1)
{
    O0.assign(g.kind == FHE_JOB_MAXMIN ? g.d : 1, nullptr);
    O1.assign(g.kind == FHE_JOB_MAXMIN ? g.d : 1, nullptr);
    MultiItem it;
    it.x = X.data();
    it.y = Y.data();
    it.d = g.d;
    it.maxmin = g.kind == FHE_JOB_MAXMIN;
    it.out0 = j0.out0 ? O0.data() : nullptr;
    it.out1 = j0.out1 ? O1.data() : nullptr;
    return {it};
}

// results of group g (held in src0/src1) back to its jobs: a slice per job,
// or (direct, one job) the handles themselves
int scatter(fhe_ctx *c, const fhe_job *jobs, const Group &g, std::vector<fhe_ct *> &src0,
            std::vector<fhe_ct *> &src1, bool transfer)
{
    int err = 0, off = 0;
    for (int id : g.jobs) {
        const fhe_job &j = jobs[id];
        const int cnt = j.x[0]->count;
        for (int s = 0; s < 2 && !err; s++) {
            fhe_ct **dst = s == 0 ? j.out0 : j.out1;
            std::vector<fhe_ct *> &src = s == 0 ? src0 : src1;
            if (!dst) continue;
            for (size_t k = 0; k < src.size() && !err; k++) {
                if (!src[k]) continue;
                if (transfer && g.jobs.size() == 1) {
                    dst[k] = src[k];
                    src[k] = nullptr;
                } else {
                    err = op_slice(c, src[k], off, cnt, &dst[k]);
                }
            }
        }
        off += cnt;
    }
    return err;
}

// each job's digit-k operands into the plan's buffer (one copy per part)
void fill(fhe_ctx *c, const fhe_job *jobs, const Group &g, int k, bool ys, fhe_ct *dst)
{
    size_t off = 0;
    for (int id : g.jobs) {
        const fhe_ct *part = ys ? jobs[id].y[k] : jobs[id].x[k];
        cudaMemcpyAsync((char *)dst->d + off, part->d, part->bytes, cudaMemcpyDeviceToDevice, c->stream);
        off += part->bytes;
    }
}

void plan_free(fhe_ctx *c, BatchPlan *P)
{
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    for (auto *v : {&P->X, &P->Y, &P->O0, &P->O1})
        for (auto &g : *v)
            for (fhe_ct *x : g) fhe_ct_destroy(x);
    for (auto &kv : P->held)
        for (void *p : kv.second) c->pool.put(p);
    for (auto &m : P->mheld)
        for (auto &kv : m.second)
            for (void *p : kv.second) m.first->pool.put(p);
    delete P;
}

// Fused-ring plans (batch graphs of several contexts of one plaintext
// prime), kept across calls like a context's own plans; released with any
// member context (and when memory runs out).
std::recursive_mutex g_fam_mu;
std::vector<BatchPlan *> g_fam_plans;
std::map<std::vector<u64>, int> g_fam_seen;
std::set<std::vector<u64>> g_fam_nocap;  // shapes whose capture ran out of memory
u64 g_fam_clock = 0;
constexpr int FAM_PLAN_CAP = 4;

// Captures the circuit of these groups into a new plan (nothing runs).
int capture(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups, const std::vector<u64> &sig, BatchPlan **out)
{
    BatchPlan *P = new BatchPlan;
    P->sig = sig;
    int err = 0;
    std::map<const fhe_evk *, std::vector<MultiItem>> by_evk;
    for (auto &kv : groups) {
        Group &g = kv.second;
        int cnt = 0;
        for (int id : g.jobs) cnt += jobs[id].x[0]->count;
        P->X.emplace_back();
        P->Y.emplace_back();
        P->O0.emplace_back();
        P->O1.emplace_back();
        for (int k = 0; k < g.d && !err; k++) {
            fhe_ct *a = ct_new(c, cnt, 2, g.level, &err);
            fhe_ct *b = a ? ct_new(c, cnt, 2, g.level, &err) : nullptr;
            P->X.back().push_back(a);
            P->Y.back().push_back(b);
        }
        if (err) break;
    }
    if (!err) {
        size_t gi = 0;
        for (auto &kv : groups) {
            Group &g = kv.second;
            auto it = items_for(g, jobs[g.jobs[0]], P->X[gi], P->Y[gi], P->O0[gi], P->O1[gi]);
            by_evk[g.evk].push_back(it[0]);
            gi++;
        }
    }
    cudaStream_t user = c->stream, cap = nullptr;
    if (!err) err = fhe_cuda_check(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    if (!err) {
        const bool prof = c->prof_on;
        c->prof_on = false;
        c->pool.cap_free = &P->held;
        c->pool.in_capture = true;
        c->stream = cap;
        c->pool.stream = cap;
        err = fhe_cuda_check(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed), "begin capture");
        if (!err) {
            c->capturing = true;
            for (auto &kv : by_evk) {
                if (err) break;
                err = circuit_multi(c, kv.first, kv.second);
            }
            c->capturing = false;
            cudaGraph_t gr = nullptr;
            const int e2 = fhe_cuda_check(c, cudaStreamEndCapture(cap, &gr), "end capture");
            if (!err) err = e2;
            P->graph = gr;
        }
        c->stream = user;
        c->pool.stream = user;
        c->pool.cap_free = nullptr;
        c->pool.in_capture = false;
        c->prof_on = prof;
        cudaStreamDestroy(cap);
    }
    if (!err) err = fhe_cuda_check(c, cudaGraphInstantiate(&P->exec, P->graph, 0), "graph instantiate");
    if (!err) {
        size_t n = 0;
        cudaGraphGetNodes(P->graph, nullptr, &n);
        P->nodes = (int)n;
    }
    if (err) {
        plan_free(c, P);
        return err;
    }
    *out = P;
    return 0;
}

int replay_in(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups, BatchPlan *P);

int replay(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups, BatchPlan *P)
{
    c->bplan_active = P;
    const int err = replay_in(c, jobs, groups, P);
    c->bplan_active = nullptr;
    return err;
}

int replay_in(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups, BatchPlan *P)
{
    size_t gi = 0;
    for (auto &kv : groups) {
        const Group &g = kv.second;
        for (int k = 0; k < g.d; k++) {
            fill(c, jobs, g, k, false, P->X[gi][k]);
            fill(c, jobs, g, k, true, P->Y[gi][k]);
        }
        gi++;
    }
    int err = fhe_cuda_check(c, cudaGraphLaunch(P->exec, c->stream), "batch graph launch");
    c->launches += P->nodes;
    P->last = ++c->bplan_clock;
    gi = 0;
    for (auto &kv : groups) {
        if (err) break;
        err = scatter(c, jobs, kv.second, P->O0[gi], P->O1[gi], false);
        gi++;
    }
    return err;
}

// each group's operands concatenated (one batch per digit)
int gather_groups(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups)
{
    int err = 0;
    for (auto &kv : groups) {
        Group &g = kv.second;
        g.X.assign(g.d, nullptr);
        g.Y.assign(g.d, nullptr);
        g.own_x.assign(2 * g.d, false);
        for (int k = 0; k < g.d && !err; k++) {
            bool o1 = false, o2 = false;
            err = gather(c, jobs, g.jobs, k, false, &g.X[k], &o1);
            if (!err && g.kind != FHE_JOB_SORT) err = gather(c, jobs, g.jobs, k, true, &g.Y[k], &o2);
            g.own_x[k] = o1;
            g.own_x[g.d + k] = o2;
        }
        if (err) break;
    }
    return err;
}

// results back to the jobs; the group buffers freed
int scatter_groups(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups, int err)
{
    for (auto &kv : groups) {
        Group &g = kv.second;
        if (!err) err = scatter(c, jobs, g, g.out0, g.out1, true);
        for (fhe_ct *x : g.out0) fhe_ct_destroy(x);
        for (fhe_ct *x : g.out1) fhe_ct_destroy(x);
        for (int k = 0; k < 2 * g.d && k < (int)g.own_x.size(); k++)
            if (g.own_x[k]) fhe_ct_destroy(k < g.d ? g.X[k] : g.Y[k - g.d]);
        g.out0.clear();
        g.out1.clear();
        g.own_x.clear();
    }
    return err;
}

int run_direct(fhe_ctx *c, const fhe_job *jobs, GroupMap &groups)
{
    int err = gather_groups(c, jobs, groups);
    // one circuit per key set; with multistream the groups overlap
    std::map<const fhe_evk *, std::vector<MultiItem>> by_evk;
    if (!err)
        for (auto &kv : groups) {
            Group &g = kv.second;
            if (g.kind == FHE_JOB_SORT) continue;
            auto it = items_for(g, jobs[g.jobs[0]], g.X, g.Y, g.out0, g.out1);
            by_evk[g.evk].push_back(it[0]);
        }
    c->multistream = true;
    for (auto &kv : by_evk) {
        if (err) break;
        err = circuit_multi(c, kv.first, kv.second);
    }
    // sorting groups: one sort circuit each (rows are independent, so the
    // concatenated group sorts every job's rows)
    for (auto &kv : groups) {
        Group &g = kv.second;
        if (err || g.kind != FHE_JOB_SORT) continue;
        g.out0.assign(g.d, nullptr);
        std::vector<const fhe_ct *> X(g.X.begin(), g.X.end());
        err = circuit_sort(c, g.evk, X.data(), g.d, g.out0.data());
    }
    c->multistream = false;
    return scatter_groups(c, jobs, groups, err);
}

// The items of a family's groups (family order), with the keys of each; the
// item of the first member that has one leads the circuit (items[0]).
void family_items(const std::vector<fhe_ctx *> &fam, const fhe_job *jobs, std::vector<GroupMap> &gm,
                  std::vector<std::vector<fhe_ct *>> *X, std::vector<std::vector<fhe_ct *>> *Y,
                  std::vector<std::vector<fhe_ct *>> *O0, std::vector<std::vector<fhe_ct *>> *O1,
                  std::vector<const fhe_evk *> &evks, std::vector<MultiItem> &items)
{
    size_t gi = 0;
    for (size_t i = 0; i < fam.size(); i++)
        for (auto &kv : gm[i]) {
            Group &g = kv.second;
            auto it = X ? items_for(g, jobs[g.jobs[0]], (*X)[gi], (*Y)[gi], (*O0)[gi], (*O1)[gi])
                        : items_for(g, jobs[g.jobs[0]], g.X, g.Y, g.out0, g.out1);
            items.push_back(it[0]);
            evks.push_back(g.evk);
            gi++;
        }
}

// shape of a family's submission: the members and each one's group shapes
std::vector<u64> family_signature(const std::vector<fhe_ctx *> &fam, const fhe_job *jobs,
                                  const std::vector<GroupMap> &gm)
{
    std::vector<u64> sig;
    for (size_t i = 0; i < fam.size(); i++) {
        const std::vector<u64> s = signature(jobs, gm[i]);
        sig.push_back((u64)(uintptr_t)fam[i]);
        sig.push_back(s.size());
        sig.insert(sig.end(), s.begin(), s.end());
    }
    return sig;
}

// Captures a family's circuit into a new plan (nothing runs): operand and
// result buffers per group in each member's pool; every member's pool keeps
// what the capture frees (the plan reuses it on every replay).  The members'
// streams are the leader's (run_family).
int capture_family(const std::vector<fhe_ctx *> &fam, const fhe_job *jobs, std::vector<GroupMap> &gm,
                   const std::vector<u64> &sig, BatchPlan **out)
{
    fhe_ctx *lead = fam[0];
    BatchPlan *P = new BatchPlan;
    P->sig = sig;
    P->members = fam;
    int err = 0;
    for (size_t i = 0; i < fam.size() && !err; i++)
        for (auto &kv : gm[i]) {
            Group &g = kv.second;
            int cnt = 0;
            for (int id : g.jobs) cnt += jobs[id].x[0]->count;
            P->X.emplace_back();
            P->Y.emplace_back();
            P->O0.emplace_back();
            P->O1.emplace_back();
            for (int k = 0; k < g.d && !err; k++) {
                fhe_ct *a = ct_new(fam[i], cnt, 2, g.level, &err);
                fhe_ct *b = a ? ct_new(fam[i], cnt, 2, g.level, &err) : nullptr;
                P->X.back().push_back(a);
                P->Y.back().push_back(b);
            }
        }
    std::vector<const fhe_evk *> evks;
    std::vector<MultiItem> items;
    if (!err) family_items(fam, jobs, gm, &P->X, &P->Y, &P->O0, &P->O1, evks, items);
    cudaStream_t user = lead->stream, cap = nullptr;
    if (!err) err = fhe_cuda_check(lead, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    if (!err) {
        std::vector<bool> prof;
        for (fhe_ctx *m : fam) {
            prof.push_back(m->prof_on);
            m->prof_on = false;
            m->pool.cap_free = &P->mheld[m];
            m->pool.in_capture = true;
            m->stream = cap;
            m->pool.stream = cap;
            m->capturing = true;
        }
        err = fhe_cuda_check(lead, cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed), "begin capture");
        if (!err) {
            err = circuit_multi_ctx(evks, items);
            cudaGraph_t gr = nullptr;
            const int e2 = fhe_cuda_check(lead, cudaStreamEndCapture(cap, &gr), "end capture");
            if (!err) err = e2;
            P->graph = gr;
        }
        for (size_t i = 0; i < fam.size(); i++) {
            fhe_ctx *m = fam[i];
            m->capturing = false;
            m->stream = user;
            m->pool.stream = user;
            m->pool.cap_free = nullptr;
            m->pool.in_capture = false;
            m->prof_on = prof[i];
        }
        cudaStreamDestroy(cap);
    }
    if (!err) err = fhe_cuda_check(lead, cudaGraphInstantiate(&P->exec, P->graph, 0), "graph instantiate");
    if (!err) {
        size_t n = 0;
        cudaGraphGetNodes(P->graph, nullptr, &n);
        P->nodes = (int)n;
    }
    if (err) {
        plan_free(lead, P);
        return err;
    }
    *out = P;
    return 0;
}

// operands in, one graph launch on the leader's stream, results sliced out
int replay_family(const std::vector<fhe_ctx *> &fam, const fhe_job *jobs, std::vector<GroupMap> &gm, BatchPlan *P)
{
    for (fhe_ctx *m : fam) m->bplan_active = P;  // kept if memory runs out meanwhile
    size_t gi = 0;
    for (size_t i = 0; i < fam.size(); i++)
        for (auto &kv : gm[i]) {
            const Group &g = kv.second;
            for (int k = 0; k < g.d; k++) {
                fill(fam[i], jobs, g, k, false, P->X[gi][k]);
                fill(fam[i], jobs, g, k, true, P->Y[gi][k]);
            }
            gi++;
        }
    int err = fhe_cuda_check(fam[0], cudaGraphLaunch(P->exec, fam[0]->stream), "fused batch graph launch");
    fam[0]->launches += P->nodes;
    P->last = ++g_fam_clock;
    gi = 0;
    for (size_t i = 0; i < fam.size(); i++)
        for (auto &kv : gm[i]) {
            if (!err) err = scatter(fam[i], jobs, kv.second, P->O0[gi], P->O1[gi], false);
            gi++;
        }
    for (fhe_ctx *m : fam) m->bplan_active = nullptr;
    return err;
}

// The compare and max/min jobs of contexts that share a device and a
// plaintext prime, in one circuit (fused launches across ring degrees,
// digit counts and levels); their sort jobs afterwards, per context.  Every
// member context works on the leader's stream meanwhile: the leader first
// waits for what the others have queued, and they wait for the leader at
// the end.  A submission shape the family has served before is captured
// (once) into a graph and replayed.  The caller holds every member's lock.
int run_family(const std::vector<fhe_ctx *> &fam_in, const fhe_job *jobs,
               std::map<fhe_ctx *, std::vector<int>> &by_ctx)
{
    // members with compare jobs first (the first of them leads the circuit)
    std::vector<fhe_ctx *> fam;
    for (int pass = 0; pass < 2; pass++)
        for (fhe_ctx *m : fam_in) {
            bool cmp = false;
            for (int id : by_ctx[m]) cmp = cmp || jobs[id].kind != FHE_JOB_SORT;
            if (cmp == (pass == 0)) fam.push_back(m);
        }
    fhe_ctx *lead = fam[0];
    const cudaStream_t ls = lead->stream;
    std::vector<cudaStream_t> saved;
    int err = 0;
    auto follow = [&](cudaStream_t waiter, cudaStream_t on) {  // waiter waits for work queued on `on`
        cudaEvent_t ev = nullptr;
        int e = fhe_cuda_check(lead, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "fuse event");
        if (!e) e = fhe_cuda_check(lead, cudaEventRecord(ev, on), "fuse event");
        if (!e) e = fhe_cuda_check(lead, cudaStreamWaitEvent(waiter, ev, 0), "fuse wait");
        if (ev) cudaEventDestroy(ev);
        return e;
    };
    for (fhe_ctx *m : fam) {
        saved.push_back(m->stream);
        if (m == lead) continue;
        if (!err) err = follow(ls, m->stream);
        m->stream = ls;
        m->pool.stream = ls;
    }
    std::vector<GroupMap> gm(fam.size());
    std::vector<GroupMap> sorts(fam.size());
    bool any = false;
    for (size_t i = 0; i < fam.size(); i++) {
        std::vector<int> cmp, srt;
        for (int id : by_ctx[fam[i]]) (jobs[id].kind == FHE_JOB_SORT ? srt : cmp).push_back(id);
        gm[i] = make_groups(jobs, cmp);
        sorts[i] = make_groups(jobs, srt);
        any = any || !cmp.empty();
    }
    bool done = false;
    if (!err && any && lead->bplan_cap > 0) {
        std::lock_guard<std::recursive_mutex> g(g_fam_mu);
        const std::vector<u64> sig = family_signature(fam, jobs, gm);
        BatchPlan *P = nullptr;
        for (BatchPlan *Q : g_fam_plans)
            if (Q->sig == sig) P = Q;
        if (!P && g_fam_seen[sig]++ > 0 && !g_fam_nocap.count(sig)) {
            // evict the least recently used plan of this family's members
            // (their locks are held here) once the family has FAM_PLAN_CAP
            std::vector<size_t> mine;
            for (size_t q = 0; q < g_fam_plans.size(); q++) {
                bool ours = true;
                for (fhe_ctx *m : g_fam_plans[q]->members)
                    ours = ours && std::find(fam.begin(), fam.end(), m) != fam.end();
                if (ours) mine.push_back(q);
            }
            if ((int)mine.size() >= FAM_PLAN_CAP) {
                size_t lru = mine[0];
                for (size_t q : mine)
                    if (g_fam_plans[q]->last < g_fam_plans[lru]->last) lru = q;
                cudaDeviceSynchronize();
                plan_free(lead, g_fam_plans[lru]);
                g_fam_plans.erase(g_fam_plans.begin() + lru);
            }
            err = capture_family(fam, jobs, gm, sig, &P);
            if (err == FHE_ENOMEM) {
                // a graph keeps every intermediate of the circuit: the
                // members' own batch graphs and cached blocks go back to the
                // device, and the capture is tried once more
                cudaDeviceSynchronize();
                cudaGetLastError();  // the failed allocation's error is not sticky
                for (fhe_ctx *m : fam) {
                    batch_plans_release(m);
                    m->pool.trim();
                }
                err = capture_family(fam, jobs, gm, sig, &P);
            }
            if (err == FHE_ENOMEM) {
                // too large to hold as a graph: this shape runs directly
                cudaDeviceSynchronize();
                cudaGetLastError();
                for (fhe_ctx *m : fam) m->pool.trim();
                g_fam_nocap.insert(sig);
                P = nullptr;
                err = 0;
            }
            if (!err && P) g_fam_plans.push_back(P);
        }
        if (!err && P) {
            err = replay_family(fam, jobs, gm, P);
            done = true;
        }
        if (g_fam_seen.size() > 1024) g_fam_seen.clear();
        if (g_fam_nocap.size() > 1024) g_fam_nocap.clear();
    }
    if (!err && any && !done) {
        std::vector<const fhe_evk *> evks;
        std::vector<MultiItem> items;
        for (size_t i = 0; i < fam.size() && !err; i++) err = gather_groups(fam[i], jobs, gm[i]);
        if (!err) family_items(fam, jobs, gm, nullptr, nullptr, nullptr, nullptr, evks, items);
        if (!err) {
            const bool ms = lead->multistream;
            lead->multistream = true;
            err = circuit_multi_ctx(evks, items);
            lead->multistream = ms;
        }
        for (size_t i = 0; i < fam.size(); i++) err = scatter_groups(fam[i], jobs, gm[i], err);
    }
    for (size_t i = 0; i < fam.size() && !err; i++)
        if (!sorts[i].empty()) err = run_direct(fam[i], jobs, sorts[i]);
    for (size_t i = 0; i < fam.size(); i++) {
        fhe_ctx *m = fam[i];
        if (m == lead) continue;
        m->stream = saved[i];
        m->pool.stream = saved[i];
        const int e = follow(m->stream, ls);
        if (!err) err = e;
    }
    return err;
}

// A submission whose shape the context has served before is captured (once)
// and replayed; a new shape runs directly under the multi-stream scheduler.
int run_context(fhe_ctx *c, const fhe_job *jobs, const std::vector<int> &ids)
{
    GroupMap groups = make_groups(jobs, ids);
    bool sort = false;
    for (auto &kv : groups) sort = sort || kv.second.kind == FHE_JOB_SORT;
    if (c->bplan_cap <= 0 || sort) return run_direct(c, jobs, groups);  // sorting is not captured
    const std::vector<u64> sig = signature(jobs, groups);
    for (BatchPlan *P : c->bplans)
        if (P->sig == sig) return replay(c, jobs, groups, P);
    if (c->bseen.size() > 1024) c->bseen.clear();
    if (c->bseen[sig]++ == 0) return run_direct(c, jobs, groups);
    if ((int)c->bplans.size() >= c->bplan_cap) {  // evict the least recently used
        auto lru = std::min_element(c->bplans.begin(), c->bplans.end(),
                                    [](const BatchPlan *a, const BatchPlan *b) { return a->last < b->last; });
        cudaStreamSynchronize(c->stream);
        plan_free(c, *lru);
        c->bplans.erase(lru);
    }
    BatchPlan *P = nullptr;
    const int err = capture(c, jobs, groups, sig, &P);
    if (err) return err;
    c->bplans.push_back(P);
    return replay(c, jobs, groups, P);
}

}  // namespace

// Frees every captured batch of the context except `keep` (the caller has
// made sure none of them is running).
void batch_plans_release(fhe_ctx *c, const BatchPlan *keep)
{
    std::vector<BatchPlan *> kept;
    for (BatchPlan *P : c->bplans)
        if (P == keep)
            kept.push_back(P);
        else
            plan_free(c, P);
    c->bplans = kept;
    if (!keep) c->bseen.clear();
}

// Fused-ring plans that hold memory of c (a context being destroyed): they
// may run on another member's stream, so the whole device is drained first.
// They are freed only here and by run_family (which holds every member's
// lock): the memory-pressure paths leave them alone, since another thread may
// hold the other members.
void batch_family_release(fhe_ctx *c)
{
    std::lock_guard<std::recursive_mutex> g(g_fam_mu);
    bool synced = false;
    for (size_t i = 0; i < g_fam_plans.size();) {
        BatchPlan *P = g_fam_plans[i];
        if (std::find(P->members.begin(), P->members.end(), c) == P->members.end()) {
            i++;
            continue;
        }
        if (!synced) cudaDeviceSynchronize(), synced = true;
        plan_free(c, P);
        g_fam_plans.erase(g_fam_plans.begin() + i);
    }
}

extern "C" int fhe_ctx_set_batch_graphs(fhe_ctx *c, int max_plans)
{
    if (!c || max_plans < 0) return FHE_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    cudaStreamSynchronize(c->stream);
    batch_plans_release(c);
    c->bplan_cap = max_plans;
    return 0;
}

namespace {

// Level alignment: within each (context, keys, kind, digits, outputs) the
// jobs above the lowest level get copies of their operands switched down to
// it (several primes at once), so that they share one group.  The copies are
// released after the circuit has been enqueued (stream-ordered reuse).
struct Aligned {
    std::vector<fhe_job> jobs;
    std::vector<std::vector<const fhe_ct *>> ops;  // per job: x[0..d), y[0..d)
    std::vector<fhe_ct *> owned;
    ~Aligned()
    {
        for (fhe_ct *x : owned) fhe_ct_destroy(x);
    }
};

int align_levels(const fhe_job *jobs, int n, Aligned &A)
{
    std::map<std::tuple<fhe_ctx *, const fhe_evk *, int, int, bool, bool>, int> lowest;
    for (int i = 0; i < n; i++) {
        const fhe_job &j = jobs[i];
        auto key = std::make_tuple(j.ctx, j.evk, j.kind, j.d, j.out0 != nullptr, j.out1 != nullptr);
        auto it = lowest.find(key);
        const int lv = j.x[0]->level;
        if (it == lowest.end() || lv < it->second) lowest[key] = lv;
    }
    A.jobs.assign(jobs, jobs + n);
    A.ops.resize(n);
    // every operand above its target, per context: switched down in merged
    // rounds (at most FHE_MAXK primes a step, one launch per step for all)
    struct Want {
        const fhe_ct **slot;
        const fhe_ct *cur;
        int target;
    };
    std::map<fhe_ctx *, std::vector<Want>> want;
    for (int i = 0; i < n; i++) {
        fhe_job &j = A.jobs[i];
        const int target =
            lowest[std::make_tuple(j.ctx, j.evk, j.kind, j.d, j.out0 != nullptr, j.out1 != nullptr)];
        std::vector<const fhe_ct *> &ops = A.ops[i];
        ops.assign(2 * j.d, nullptr);
        const int nops = j.kind == FHE_JOB_SORT ? j.d : 2 * j.d;
        for (int k = 0; k < nops; k++) {
            const fhe_ct *src = k < j.d ? j.x[k] : j.y[k - j.d];
            ops[k] = src;
            if (src->level > target) want[j.ctx].push_back(Want{&ops[k], src, target});
        }
        j.x = ops.data();
        j.y = ops.data() + j.d;
    }
    for (auto &kv : want) {
        fhe_ctx *c = kv.first;
        std::lock_guard<std::mutex> g(c->mu);
        for (;;) {
            std::vector<SwitchItem> items;
            std::vector<Want *> who;
            for (Want &w : kv.second)
                if (w.cur->level > w.target) {
                    items.push_back(SwitchItem{c, w.cur, std::min(w.cur->level - w.target, FHE_MAXK), nullptr});
                    who.push_back(&w);
                }
            if (items.empty()) break;
            const int e = op_modswitch_many(items);
            if (e) return e;
            for (size_t t = 0; t < items.size(); t++) {
                A.owned.push_back(items[t].out);
                who[t]->cur = items[t].out;
                *who[t]->slot = items[t].out;
            }
        }
    }
    return 0;
}

}  // namespace

extern "C" int fhe_batch_submit(const fhe_job *jobs, int n, fhe_batch **out)
{
    return fhe_batch_submit_ex(jobs, n, 0, out);
}

extern "C" int fhe_batch_submit_ex(const fhe_job *jobs, int n, int flags, fhe_batch **out)
{
    FHE_RANGE("fhe_batch_submit_ex");
    if (!jobs || n < 1 || !out || (flags & ~(FHE_BATCH_ALIGN_LEVELS | FHE_BATCH_FUSE_RINGS))) return FHE_EINVAL;
    for (int i = 0; i < n; i++) {
        int e = batch_check_job(jobs[i]);
        if (e) return e;
    }
    Aligned A;
    if (flags & FHE_BATCH_ALIGN_LEVELS) {
        const int e = align_levels(jobs, n, A);
        if (e) return e;
        jobs = A.jobs.data();
    }
    std::vector<fhe_ctx *> order;
    std::map<fhe_ctx *, std::vector<int>> by_ctx;
    for (int i = 0; i < n; i++) {
        if (!by_ctx.count(jobs[i].ctx)) order.push_back(jobs[i].ctx);
        by_ctx[jobs[i].ctx].push_back(i);
    }
    // families of contexts that run in one circuit (FHE_BATCH_FUSE_RINGS:
    // one device and plaintext prime), in order of first appearance
    std::vector<std::vector<fhe_ctx *>> fams;
    for (fhe_ctx *c : order) {
        bool placed = false;
        if (flags & FHE_BATCH_FUSE_RINGS)
            for (auto &f : fams)
                if (f[0]->p == c->p && f[0]->device == c->device) {
                    f.push_back(c);
                    placed = true;
                    break;
                }
        if (!placed) fams.push_back({c});
    }
    fhe_batch *B = new fhe_batch;
    B->job_event.assign(n, 0);
    int err = 0;
    // Two phases per family: its compare and max/min jobs, then its sort jobs
    // (long circuits), each followed by one event per context, so that a
    // job completes with its own phase rather than with the whole batch.
    for (auto &fam : fams) {
        std::vector<fhe_ctx *> lock_order(fam);
        std::sort(lock_order.begin(), lock_order.end());
        std::vector<std::unique_lock<std::mutex>> locks;
        for (fhe_ctx *c : lock_order) locks.emplace_back(c->mu);
        for (int phase = 0; phase < 2 && !err; phase++) {
            std::map<fhe_ctx *, std::vector<int>> ids;
            bool any = false;
            for (fhe_ctx *c : fam)
                for (int id : by_ctx[c])
                    if ((jobs[id].kind == FHE_JOB_SORT) == (phase == 1)) ids[c].push_back(id), any = true;
            if (!any) continue;
            if (fam.size() == 1)
                err = run_context(fam[0], jobs, ids[fam[0]]);
            else
                err = run_family(fam, jobs, ids);
            for (fhe_ctx *c : fam) {
                if (!ids.count(c)) continue;
                cudaEvent_t ev = nullptr;
                if (!err) err = fhe_cuda_check(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch event");
                if (!err) err = fhe_cuda_check(c, cudaEventRecord(ev, c->stream), "batch event");
                if (ev) {
                    for (int id : ids[c]) B->job_event[id] = (int)B->done.size();
                    B->done.push_back({c, ev});
                }
            }
        }
        if (err) break;
    }
    if (err) {
        fhe_batch_destroy(B);
        return err;
    }
    *out = B;
    return 0;
}

extern "C" int fhe_batch_job_done(fhe_batch *B, int i) { return batch_job_done(B, i); }

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
