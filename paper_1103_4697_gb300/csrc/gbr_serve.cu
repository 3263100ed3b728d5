// Serving for libgbres: continuous batching of resultant and gcd requests.
//
// gbr_submit deep-copies a job into the queue and returns a ticket.  Worker
// threads (one CUDA stream and one child context each, all sharing the parent
// context's device arena) repeatedly take their share of the queued jobs (a
// third of the queue, at least 32) as far as the device-memory budget allows,
// group them by kind, and run them as device batches; gbr_wait_any hands out
// finished jobs in completion order.
// Because several workers run at once on separate streams, a batch that
// arrives while another is on the GPU is admitted as soon as memory allows and
// overlaps with it.  Residues stay in device memory for the whole life of a
// batch; only inputs go in and final limbs come out.  Every wait in this file
// is on a host condition variable; nothing spins on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>

#include "gbr_core.h"

namespace gbr {

struct ServeJob {
    uint64_t ticket = 0;
    int32_t kind = 0, var = 1;
    std::vector<uint64_t> a, b;      // coefficient words (bivariate) or int64 (univariate)
    gbr_bipoly f{}, g{};
    gbr_upoly p{}, q{};
    size_t est = 0;                  // device bytes reserved while in flight
    int status = GBR_EAGAIN;
    bool done = false;
    double t_done = 0.0;             // completion time, seconds on the steady clock
    gbr_bigpoly result{-1, 0, nullptr, nullptr};
};

static double steady_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<ServeJob>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<ServeJob>> jobs;
    std::deque<uint64_t> completions;   // tickets in completion order (gbr_wait_any)
    std::vector<std::thread> threads;
    std::vector<gbr_ctx *> workers;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t inflight = 0, cap = 0;
    gbr_serve_stats stats{};
};

static const int kWorkers = 3;
static const int kMaxBatch = 8192;
static const size_t kMinShare = 32;   // a worker takes at least this many queued jobs

static size_t estimate_bytes(const ServeJob &j) {
    if (j.kind == GBR_JOB_GCD) {
        int64_t dp = j.p.deg, dq = j.q.deg;
        int64_t k = (std::max(dp, dq) + 140) / 31 + 8;
        int64_t S = std::min(dp, dq) + dp + dq + 3;
        return (size_t)(k * S * 4 * 2 + (dp + dq + 2) * 8 * 2 + 4096);
    }
    gbr_res_info info{};
    // the per-entry bound alone: never fewer primes than the plan takes, and cheap
    if (resultant_info_impl(&j.f, j.kind == GBR_JOB_DISC ? &j.f : &j.g, j.var, j.kind == GBR_JOB_DISC, &info, false) ||
        info.m < 0 || info.n < 0)
        return 4096;
    int64_t P = info.deg_bound + 1, k = info.primes, L = info.limbs;
    int64_t S = (int64_t)(info.m + 1 + info.n + 1) * (std::max(j.f.deg_x, j.f.deg_y) + 1);
    int64_t in = (int64_t)j.a.size() * 8 + (int64_t)j.b.size() * 8;
    // residues, values and their denominators (up to 2 P points on roots of unity),
    // coefficients mod p, output limbs
    return (size_t)(k * S * 4 + 5 * k * P * 4 + P * L * 4 + P + in + 8192);
}

// marks j finished (caller holds S->mu) and queues its ticket for gbr_wait_any
static void mark_done(ServeState *S, ServeJob &j, int status) {
    j.status = status;
    j.done = true;
    j.t_done = steady_s();
    S->completions.push_back(j.ticket);
    S->stats.completed++;
}

static void finish(ServeState *S, const std::shared_ptr<ServeJob> &j, int status, const gbr_bigpoly *r) {
    std::lock_guard<std::mutex> g(S->mu);
    if (r) j->result = *r;
    S->inflight -= j->est;
    mark_done(S, *j, status);
}

// a failing job's detail text goes to the parent context, where gbr_last_error finds it
static void parent_error(gbr_ctx *w, int st) {
    if (!w->parent) return;
    std::string msg;
    {
        std::lock_guard<std::mutex> g(w->err_mu);
        msg = w->err;
    }
    w->parent->fail(st, ("serving job: " + msg).c_str());
}

static void run_group(gbr_ctx *w, ServeState *S, std::vector<std::shared_ptr<ServeJob>> &grp) {
    if (grp.empty()) return;
    NvtxScope call("gbr: serving batch");
    const int n = (int)grp.size();
    std::vector<gbr_bigpoly> out(n);
    int st;
    const int kind = grp[0]->kind, var = grp[0]->var;
    if (kind == GBR_JOB_GCD) {
        std::vector<gbr_upoly> p(n), q(n);
        for (int i = 0; i < n; ++i) {
            p[i] = grp[i]->p;
            q[i] = grp[i]->q;
        }
        st = gbr_gcd_batch(w, n, p.data(), q.data(), out.data());
    } else {
        std::vector<gbr_bipoly> f(n), g(n);
        for (int i = 0; i < n; ++i) {
            f[i] = grp[i]->f;
            g[i] = grp[i]->g;
        }
        st = kind == GBR_JOB_DISC ? gbr_discriminant_res_batch(w, n, f.data(), var, out.data())
                                  : gbr_resultant_batch(w, n, f.data(), g.data(), var, out.data());
    }
    if (st == GBR_OK) {
        for (int i = 0; i < n; ++i) finish(S, grp[i], GBR_OK, &out[i]);
    } else if (n > 1) {
        // isolate the failing job(s): run them one at a time
        for (auto &j : grp) {
            std::vector<std::shared_ptr<ServeJob>> one{j};
            run_group(w, S, one);
        }
        return;
    } else {
        parent_error(w, st);
        finish(S, grp[0], st, nullptr);
    }
    S->cv_done.notify_all();
}

static void worker_loop(gbr_ctx *parent, int wi) {
    ServeState *S = parent->serve;
    gbr_ctx *w = S->workers[wi];
    while (true) {
        std::vector<std::shared_ptr<ServeJob>> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop) return;
            // admission by memory: take queued jobs while they fit the budget, at most
            // a worker's share of the queue (so a burst spreads over the workers'
            // streams and overlaps on the device instead of waiting in one batch)
            const size_t share = std::max<size_t>(kMinShare, (S->queue.size() + kWorkers - 1) / kWorkers);
            while (!S->queue.empty() && (int)batch.size() < kMaxBatch && batch.size() < share) {
                auto &j = S->queue.front();
                if (j->est > S->cap) {   // can never fit: fail it now
                    mark_done(S, *j, GBR_ENOMEM);
                    S->queue.pop_front();
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->inflight + j->est > S->cap) break;
                S->inflight += j->est;
                batch.push_back(j);
                S->queue.pop_front();
            }
            if (batch.empty()) {
                // the head job waits for memory held by other workers' batches
                S->stats.waits_for_memory++;
                S->cv_done.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            S->stats.batches++;
            S->stats.max_batch = std::max<int64_t>(S->stats.max_batch, (int64_t)batch.size());
            S->stats.peak_bytes = std::max<int64_t>(S->stats.peak_bytes, (int64_t)S->inflight);
            if (!S->queue.empty()) S->cv_work.notify_one();   // let another worker admit the rest
        }
        // group by (kind, var) and run each group as one device batch
        std::stable_sort(batch.begin(), batch.end(), [](const std::shared_ptr<ServeJob> &x, const std::shared_ptr<ServeJob> &y) {
            return x->kind != y->kind ? x->kind < y->kind : x->var < y->var;
        });
        size_t i = 0;
        while (i < batch.size()) {
            size_t j = i;
            std::vector<std::shared_ptr<ServeJob>> grp;
            while (j < batch.size() && batch[j]->kind == batch[i]->kind && batch[j]->var == batch[i]->var)
                grp.push_back(batch[j++]);
            run_group(w, S, grp);
            i = j;
        }
        S->cv_work.notify_one();
    }
}

static int ensure_started(gbr_ctx *c) {
    if (c->serve) return GBR_OK;
    ServeState *S = new (std::nothrow) ServeState();
    if (!S) return GBR_ENOMEM;
    S->cap = (size_t)(c->budget * 0.7);
    for (int i = 0; i < kWorkers; ++i) {
        gbr_ctx *w = gbr_make_worker(c);
        if (!w) {
            for (gbr_ctx *x : S->workers) gbr_destroy_worker(x);
            delete S;
            return c->fail(GBR_EDEVICE, "could not create a serving stream");
        }
        S->workers.push_back(w);
    }
    c->serve = S;
    for (int i = 0; i < kWorkers; ++i) S->threads.emplace_back(worker_loop, c, i);
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

void gbr_serve_shutdown(gbr_ctx *c) {
    if (!c || !c->serve) return;
    ServeState *S = c->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto &j : S->queue) mark_done(S, *j, GBR_ECANCELED);
        S->queue.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (auto &t : S->threads) t.join();
    for (gbr_ctx *w : S->workers) gbr_destroy_worker(w);
    for (auto &kv : S->jobs)
        if (kv.second->done && kv.second->status == GBR_OK) gbr_free_result(c, &kv.second->result);
    delete S;
    c->serve = nullptr;
}

static bool copy_bipoly(const gbr_bipoly &src, std::vector<uint64_t> &buf, gbr_bipoly &dst) {
    if (!src.coef || src.deg_x < 0 || src.deg_y < 0 || src.words < 1 || src.words > GBR_MAX_WORDS) return false;
    size_t n = (size_t)(src.deg_x + 1) * (src.deg_y + 1) * src.words;
    buf.assign((const uint64_t *)src.coef, (const uint64_t *)src.coef + n);
    dst = src;
    dst.coef = buf.data();
    return true;
}

static bool copy_upoly(const gbr_upoly &src, std::vector<uint64_t> &buf, gbr_upoly &dst) {
    if (!src.coef || src.deg < 0 || src.words != 1) return false;
    buf.assign((const uint64_t *)src.coef, (const uint64_t *)src.coef + (size_t)(src.deg + 1));
    dst = src;
    dst.coef = buf.data();
    return true;
}

extern "C" int gbr_submit(gbr_ctx *c, const gbr_job *job, uint64_t *ticket) {
    if (!c || !job || !ticket) return GBR_EINVAL;
    auto j = std::make_shared<ServeJob>();
    j->kind = job->kind;
    j->var = job->var;
    bool ok;
    if (job->kind == GBR_JOB_GCD) {
        ok = copy_upoly(job->p, j->a, j->p) && copy_upoly(job->q, j->b, j->q);
    } else if (job->kind == GBR_JOB_RESULTANT) {
        ok = (job->var == 0 || job->var == 1) && copy_bipoly(job->f, j->a, j->f) && copy_bipoly(job->g, j->b, j->g);
    } else if (job->kind == GBR_JOB_DISC) {
        ok = (job->var == 0 || job->var == 1) && copy_bipoly(job->f, j->a, j->f);
        j->g = j->f;
    } else {
        ok = false;
    }
    if (!ok) return GBR_EINVAL;
    j->est = estimate_bytes(*j);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        int st = ensure_started(c);
        if (st) return st;
    }
    ServeState *S = c->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        j->ticket = S->next_ticket++;
        S->jobs[j->ticket] = j;
        S->queue.push_back(j);
        S->stats.submitted++;
    }
    S->cv_work.notify_one();
    *ticket = j->ticket;
    return GBR_OK;
}

extern "C" int gbr_poll(gbr_ctx *c, uint64_t ticket, gbr_bigpoly *out, int timeout_ms) {
    if (!c || !out) return GBR_EINVAL;
    if (!c->serve) return GBR_ENOTFOUND;
    ServeState *S = c->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return GBR_ENOTFOUND;
    std::shared_ptr<ServeJob> j = it->second;
    auto ready = [&] { return j->done; };
    if (!ready()) {
        if (timeout_ms == 0) return GBR_EAGAIN;
        if (timeout_ms < 0) S->cv_done.wait(lk, ready);
        else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return GBR_ETIMEOUT;
    }
    int st = j->status;
    if (st == GBR_OK) {
        *out = j->result;
        j->result = gbr_bigpoly{-1, 0, nullptr, nullptr};
    }
    S->jobs.erase(ticket);
    return st;
}

extern "C" int gbr_wait_any(gbr_ctx *c, int timeout_ms, uint64_t *ticket, gbr_bigpoly *out, double *t_done) {
    if (!c || !ticket || !out) return GBR_EINVAL;
    if (!c->serve) return GBR_ENOTFOUND;
    ServeState *S = c->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    // tickets already consumed by gbr_poll are skipped
    auto ready = [&] {
        while (!S->completions.empty() && !S->jobs.count(S->completions.front())) S->completions.pop_front();
        return !S->completions.empty() || S->jobs.empty();
    };
    if (!ready()) {
        if (timeout_ms == 0) return GBR_EAGAIN;
        if (timeout_ms < 0) S->cv_done.wait(lk, ready);
        else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return GBR_ETIMEOUT;
    }
    if (S->completions.empty()) return GBR_ENOTFOUND;   // nothing outstanding
    const uint64_t t = S->completions.front();
    S->completions.pop_front();
    auto it = S->jobs.find(t);
    std::shared_ptr<ServeJob> j = it->second;
    *ticket = t;
    if (t_done) *t_done = j->t_done;
    const int st = j->status;
    if (st == GBR_OK) {
        *out = j->result;
        j->result = gbr_bigpoly{-1, 0, nullptr, nullptr};
    }
    S->jobs.erase(it);
    return st;
}

extern "C" double gbr_clock(void) { return steady_s(); }

extern "C" int gbr_get_serve_stats(gbr_ctx *c, gbr_serve_stats *out) {
    if (!c || !out) return GBR_EINVAL;
    if (!c->serve) {
        *out = gbr_serve_stats{};
        return GBR_OK;
    }
    std::lock_guard<std::mutex> g(c->serve->mu);
    *out = c->serve->stats;
    return GBR_OK;
}
