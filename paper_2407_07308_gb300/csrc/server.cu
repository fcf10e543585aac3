// server.cu -- a serving loop over the batch path: requests arrive from any
// thread, a worker thread admits them in arrival order while an estimate of
// the device memory they will hold fits a budget, and submits every admitted
// request as one uneven batch (continuous batching: the next batch is
// enqueued while the previous one still runs, so the device never waits for
// the host).  Each request retires as soon as its own job has its results
// (per-job completion events of the batch), and its memory estimate leaves
// the admitted total then.  Keys and contexts stay resident; the server owns
// no ciphertexts.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "fhe_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    fhe_job job;
    std::vector<const fhe_ct *> x, y;  // copies of the caller's handle arrays
    size_t est = 0;
    int state = FHE_REQ_QUEUED, error = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct InFlight {
    fhe_batch *batch;
    std::vector<Request *> reqs;
};

int ceil_log2(u64 v)
{
    int r = 0;
    while ((1ull << r) < v) r++;
    return r;
}

}  // namespace

struct fhe_server {
    fhe_server_config cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<InFlight> inflight;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    size_t admitted = 0, admitted_peak = 0;
    long long batches = 0, completed = 0, failed = 0;
    bool stopping = false;
    Clock::time_point t0;
    std::thread worker;

    double now() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
    void run();
    void reap(std::unique_lock<std::mutex> &lk);
};

// Device bytes a request adds while it runs (a conservative model of the
// comparison circuit under the dependency scheduler, whose 8 streams keep
// the blocks they free until the circuit joins, so that scratch is seldom
// reused inside one circuit): for every ciphertext product -- M = B/2 +
// ceil(log2 p) + ceil((p-1)/B) per digit for the Paterson-Stockmeyer
// evaluation, 2 per merge node, 1 per digit for max/min -- the tensor
// (3l limbs), the key-switching scratch (l + dnum (l + K) + 2 (l + K) + 2K
// limbs: coefficient copy, ModUp digits, the two accumulators, their special
// part), the relinearised and switched results (4l limbs), all at the input
// level l; plus the per-digit working set of powers and partial sums and the
// outputs; a sort holds FHE_SORT_MERGE comparisons at a time.  A limb is N
// words per ciphertext of the batch; B = 4 for p < 64, else 16.  The pool
// rounds every block up to its size class (less than 25% more), so the sum
// is scaled by 5/4.
extern "C" uint64_t fhe_job_footprint(const fhe_job *j)
{
    if (!j || !j->ctx || !j->x || !j->x[0] || j->d < 1) return 0;
    const fhe_ctx *c = j->ctx;
    const fhe_ct *a = j->x[0];
    const u64 W = 8ull * c->N * a->count;  // one limb of every ciphertext
    const u64 l = a->level, K = c->K, d = j->d;
    const u64 B = c->p < 64 ? 4 : 16;
    const u64 dnum = (l + K - 1) / K;
    const u64 per_mult = (3 * l + l + dnum * (l + K) + 2 * (l + K) + 2 * K + 4 * l) * W;
    const u64 M = B / 2 + ceil_log2(c->p) + (c->p - 1 + B - 1) / B;
    const u64 mults = d * M + 2 * (d - 1) + (j->kind == FHE_JOB_MAXMIN ? d : 0);
    const u64 ct = 2 * l * W;
    u64 est = mults * per_mult;
    est += d * (B / 2 + ceil_log2(c->p) + 4) * ct;
    est += (j->kind == FHE_JOB_MAXMIN ? 2 * d : 2) * ct;
    if (j->kind == FHE_JOB_SORT)  // FHE_SORT_MERGE shifts' comparisons at a time, plus the
        // rotated operands, the rank, the selection powers and the d accumulated outputs
        est = FHE_SORT_MERGE * est + (ceil_log2(c->p) + 3 * d + 4) * ct + 2 * per_mult;
    return est + est / 4;
}

// Each request retires when its own job has its results (not when the whole
// submission has); a submission is released once all its requests have.
void fhe_server::reap(std::unique_lock<std::mutex> &)
{
    for (size_t i = 0; i < inflight.size();) {
        InFlight &f = inflight[i];
        bool all = true, any = false;
        const double t = now();
        for (size_t j = 0; j < f.reqs.size(); j++) {
            Request *q = f.reqs[j];
            if (q->state == FHE_REQ_DONE) continue;
            const int r = batch_job_done(f.batch, (int)j);
            if (r == 0) {
                all = false;
                continue;
            }
            q->state = FHE_REQ_DONE;
            q->error = r < 0 ? r : 0;
            q->t_done = t;
            admitted -= q->est;
            completed++;
            if (r < 0) failed++;
            any = true;
        }
        if (any) cv_done.notify_all();
        if (!all) {
            i++;
            continue;
        }
        fhe_batch_destroy(f.batch);
        inflight.erase(inflight.begin() + i);
    }
}

void fhe_server::run()
{
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        reap(lk);
        std::vector<Request *> take;
        while (!queue.empty()) {
            Request *q = queue.front();
            if (cfg.max_batch > 0 && (int)take.size() >= cfg.max_batch) break;
            // a request never waits for an empty server, so one that fits the
            // budget alone always runs
            if (cfg.hbm_budget && admitted + q->est > cfg.hbm_budget && admitted > 0) break;
            queue.pop_front();
            admitted += q->est;
            take.push_back(q);
        }
        admitted_peak = std::max(admitted_peak, admitted);
        if (take.empty()) {
            if (stopping && queue.empty() && inflight.empty()) break;
            cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 50));
            continue;
        }
        const double t = now();
        std::vector<fhe_job> jobs;
        for (Request *q : take) {
            q->state = FHE_REQ_RUNNING;
            q->t_start = t;
            jobs.push_back(q->job);
        }
        lk.unlock();
        fhe_batch *b = nullptr;
        int err = fhe_batch_submit_ex(jobs.data(), (int)jobs.size(), cfg.batch_flags, &b);
        lk.lock();
        batches++;
        if (err) {
            // the whole submission failed before or while it was enqueued:
            // each request reports the error
            const double td = now();
            for (Request *q : take) {
                q->state = FHE_REQ_DONE;
                q->error = err;
                q->t_done = td;
                admitted -= q->est;
                completed++;
                failed++;
            }
            cv_done.notify_all();
            continue;
        }
        inflight.push_back({b, take});
    }
}

extern "C" int fhe_server_start(const fhe_server_config *cfg, fhe_server **out)
{
    if (!out) return FHE_EINVAL;
    fhe_server *s = new fhe_server;
    memset(&s->cfg, 0, sizeof(s->cfg));
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_batch < 0) {
        delete s;
        return FHE_EINVAL;
    }
    s->t0 = Clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return 0;
}

extern "C" int fhe_server_submit(fhe_server *s, const fhe_job *job, uint64_t *ticket)
{
    if (!s || !job || !ticket) return FHE_EINVAL;
    const int e = batch_check_job(*job);
    if (e) return e;
    auto q = std::make_unique<Request>();
    q->job = *job;
    q->x.assign(job->x, job->x + job->d);
    if (job->y)
        q->y.assign(job->y, job->y + job->d);
    else
        q->y.assign(job->d, nullptr);  // sort jobs take one operand
    q->job.x = q->x.data();
    q->job.y = q->y.data();
    q->est = fhe_job_footprint(job);
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stopping) return FHE_EINVAL;
    if (s->cfg.hbm_budget && q->est > s->cfg.hbm_budget) return FHE_EBUDGET;
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs[q->ticket] = std::move(q);
    s->cv_work.notify_one();
    return 0;
}

extern "C" int fhe_server_cancel(fhe_server *s, uint64_t ticket)
{
    if (!s) return FHE_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FHE_EINVAL;
    Request *q = it->second.get();
    if (q->state != FHE_REQ_QUEUED) return FHE_EBUSY;
    auto pos = std::find(s->queue.begin(), s->queue.end(), q);
    if (pos == s->queue.end()) return FHE_EBUSY;
    s->queue.erase(pos);
    q->state = FHE_REQ_DONE;
    q->error = FHE_ECANCELED;
    q->t_done = s->now();
    s->completed++;
    s->failed++;
    s->cv_done.notify_all();
    return 0;
}

extern "C" int fhe_server_poll(fhe_server *s, uint64_t ticket, int timeout_ms, fhe_request_info *info)
{
    if (!s) return FHE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FHE_EINVAL;
    Request *q = it->second.get();
    if (timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [q] { return q->state == FHE_REQ_DONE; });
    if (info) {
        info->state = q->state;
        info->error = q->error;
        info->t_submit_ms = q->t_submit;
        info->t_start_ms = q->t_start;
        info->t_done_ms = q->t_done;
        info->est_bytes = q->est;
    }
    if (q->state != FHE_REQ_DONE) return 0;
    s->reqs.erase(it);  // a request reported done is retired
    return 1;
}

extern "C" int fhe_server_stats(fhe_server *s, fhe_server_status *st)
{
    if (!s || !st) return FHE_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    st->queued = (long long)s->queue.size();
    long long running = 0;
    for (auto &f : s->inflight)
        for (Request *q : f.reqs) running += q->state == FHE_REQ_RUNNING;
    st->running = running;
    st->completed = s->completed;
    st->failed = s->failed;
    st->batches = s->batches;
    st->admitted_bytes = s->admitted;
    st->admitted_peak_bytes = s->admitted_peak;
    return 0;
}

extern "C" int fhe_server_stop(fhe_server *s)
{
    if (!s) return FHE_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stopping = true;
        s->cv_work.notify_one();
    }
    s->worker.join();
    delete s;
    return 0;
}
