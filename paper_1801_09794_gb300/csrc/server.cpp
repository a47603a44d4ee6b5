// Serving loop: continuous batching of independent NLFEAST requests.
//
// A request is one whole run of Algorithm 1 (create + contour + solve) on its
// own handle and CUDA stream, in two stages:
//   * a factoring thread takes requests in submission order while fewer than
//     max_active are in flight and their summed device-memory footprint stays
//     within the budget (a request that exceeds the budget on its own is taken
//     when nothing else is in flight), creates their handles, and factors the
//     node matrices of everything it took in one grouped launch sequence
//     (feast_nl_set_contour_group: requests of different n share each launch);
//     requests that cannot be grouped (complex128 factors, n > 4096) are
//     factored one by one;
//   * worker threads (max_active of them) solve factored requests, each on its
//     request's stream, and copy the kept pairs out.
// Requests in flight overlap on the GPU: one request's latency-bound reduced
// stage runs beside another's solves or a group's factorisation.  A node's
// factors are the same bits in a group as alone, and every kernel reduces in a
// fixed order, so a request's results do not depend on what else is in flight.
#include "../../include/feast_nl.h"

#include <algorithm>
#include <chrono>
#include <complex>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    feast_nl_request r;
    std::vector<feast_nl_term> terms;   // the caller's terms (buffers stay the caller's)
    int64_t footprint = 0;
    int state = 0;                      // 0 queued, 1 running, 2 done
    int waiters = 0;                    // threads blocked in feast_nl_server_wait on it
    int status = 0;
    feast_nl_handle* h = nullptr;       // from creation to the end of the solve
    feast_nl_info info{};
    int m = 0;                          // kept pairs
    std::vector<double> lam, relres;    // 2 m, m
    std::vector<std::complex<double>> X;  // n x m row-major
    std::string error;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

}  // namespace

struct feast_nl_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_ready, cv_done;
    std::deque<uint64_t> queue;          // submitted, not yet taken
    std::deque<Request*> ready;          // factored, waiting for a worker
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int64_t budget = 0, in_use = 0;
    int max_active = 1, active = 0, max_seen = 0, max_group = 0;
    int preparing = 0;                   // groups being created and factored
    int group_limit = 64;                // largest group factored together
    int64_t completed = 0;
    bool stop = false;
    std::thread factorer;
    std::vector<std::thread> workers;
};

namespace {

// Marks a request done and releases its share of the budget.
void finish(feast_nl_server* s, Request* q) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->t_done = now_ms();
        q->state = 2;
        s->in_use -= q->footprint;
        s->active -= 1;
        s->completed += 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void fail_request(Request* q, int st) {
    q->status = st;
    q->error = feast_nl_last_error();
    if (q->h) feast_nl_destroy(q->h);
    q->h = nullptr;
}

// Creates the handles of a taken group and factors their nodes (grouped where
// possible); returns the requests that are ready to solve.
std::vector<Request*> prepare_group(feast_nl_server* s, const std::vector<Request*>& group) {
    std::vector<Request*> ok, grouped;
    // handles in parallel: each creation copies its coefficients in and
    // estimates their norms on its own stream, waiting on the host in between
    std::vector<int> cst(group.size(), FEAST_NL_OK);
    std::vector<std::string> cerr(group.size());
    {
        std::vector<std::thread> ts;
        for (size_t i = 0; i < group.size(); ++i)
            ts.emplace_back([&, i] {
                Request* q = group[i];
                const feast_nl_request& r = q->r;
                cst[i] = feast_nl_create(&q->h, r.n, r.nterms, q->terms.data(), r.precision, nullptr);
                if (cst[i] != FEAST_NL_OK) cerr[i] = feast_nl_last_error();
            });
        for (auto& t : ts) t.join();
    }
    for (size_t i = 0; i < group.size(); ++i) {
        Request* q = group[i];
        if (cst[i] != FEAST_NL_OK) {
            q->status = cst[i];
            q->error = cerr[i];
            q->h = nullptr;
            finish(s, q);
            continue;
        }
        if (q->r.precision != FEAST_NL_FP64 && q->r.n <= 4096) grouped.push_back(q);
        else ok.push_back(q);
    }
    if (grouped.size() == 1) {           // nothing to share a launch with
        ok.push_back(grouped[0]);
        grouped.clear();
    }
    // one by one: complex128 factors, large n, or a group of one
    for (auto it = ok.begin(); it != ok.end();) {
        const feast_nl_request& r = (*it)->r;
        const int st = feast_nl_set_contour((*it)->h, r.c_re, r.c_im, r.ra, r.rb, r.nc, r.rule);
        if (st != FEAST_NL_OK) { fail_request(*it, st); finish(s, *it); it = ok.erase(it); }
        else ++it;
    }
    if (!grouped.empty()) {
        const size_t k = grouped.size();
        std::vector<feast_nl_handle*> hs(k);
        std::vector<double> cre(k), cim(k), ra(k), rb(k);
        std::vector<int32_t> nc(k);
        bool same_rule = true;
        for (size_t i = 0; i < k; ++i) {
            const feast_nl_request& r = grouped[i]->r;
            hs[i] = grouped[i]->h;
            cre[i] = r.c_re; cim[i] = r.c_im; ra[i] = r.ra; rb[i] = r.rb; nc[i] = r.nc;
            same_rule = same_rule && r.rule == grouped[0]->r.rule;
        }
        int st = FEAST_NL_EINVAL;
        if (same_rule)
            st = feast_nl_set_contour_group((int32_t)k, hs.data(), cre.data(), cim.data(), ra.data(),
                                            rb.data(), nc.data(), grouped[0]->r.rule, nullptr);
        if (st == FEAST_NL_OK) {
            ok.insert(ok.end(), grouped.begin(), grouped.end());
        } else {
            // one by one, so that a failing request does not take the others down
            for (Request* q : grouped) {
                const feast_nl_request& r = q->r;
                const int st1 = feast_nl_set_contour(q->h, r.c_re, r.c_im, r.ra, r.rb, r.nc, r.rule);
                if (st1 != FEAST_NL_OK) { fail_request(q, st1); finish(s, q); }
                else ok.push_back(q);
            }
        }
    }
    return ok;
}

void factor_loop(feast_nl_server* s) {
    for (;;) {
        std::vector<Request*> group;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty() || s->active >= s->max_active) return false;
                const Request& head = *s->reqs[s->queue.front()];
                return s->active == 0 || s->in_use + head.footprint <= s->budget;
            });
            if (s->stop) return;
            // the head and every following request that still fits
            while (!s->queue.empty() && s->active < s->max_active &&
                   (int)group.size() < s->group_limit) {
                Request* q = s->reqs[s->queue.front()].get();
                if (s->active > 0 && s->in_use + q->footprint > s->budget) break;
                s->queue.pop_front();
                s->in_use += q->footprint;
                s->active += 1;
                s->max_seen = std::max(s->max_seen, s->active);
                q->state = 1;
                q->t_start = now_ms();
                group.push_back(q);
            }
            s->max_group = std::max(s->max_group, (int)group.size());
        }
        // the group is prepared on a thread of its own, so that the next group
        // can be taken (and factored on the GPU alongside) while it runs
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->preparing += 1;
        }
        std::thread([s, group] {
            const std::vector<Request*> ok = prepare_group(s, group);
            // notified under the lock: once it is released this thread no
            // longer touches the server (destroy may then free it)
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request* q : ok) s->ready.push_back(q);
            s->preparing -= 1;
            s->cv_ready.notify_all();
            s->cv_done.notify_all();
        }).detach();
    }
}

// Solves one factored request and copies its kept pairs out.
void solve_request(Request& q) {
    const feast_nl_request& r = q.r;
    int st = feast_nl_solve(q.h, r.m0, r.tol, r.maxit, r.seed, nullptr, &q.info);
    if (st == FEAST_NL_OK || st == FEAST_NL_ENOT_CONVERGED || st == FEAST_NL_ETOO_MANY) {
        q.lam.assign(2 * (size_t)r.m0, 0.0);
        q.relres.assign((size_t)r.m0, 0.0);
        q.X.assign((size_t)r.n * r.m0, std::complex<double>(0.0, 0.0));
        int m = 0;
        const int g = feast_nl_get_eigpairs(q.h, r.m0, &m, q.lam.data(), q.X.data(), q.relres.data(), 0);
        if (g != FEAST_NL_OK) st = g;
        q.m = m;
    }
    if (st != FEAST_NL_OK) q.error = feast_nl_last_error();
    q.status = st;
    feast_nl_destroy(q.h);
    q.h = nullptr;
}

void worker_loop(feast_nl_server* s) {
    for (;;) {
        Request* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_ready.wait(lk, [&] { return s->stop || !s->ready.empty(); });
            if (s->ready.empty()) return;       // stop, nothing left
            q = s->ready.front();
            s->ready.pop_front();
        }
        solve_request(*q);
        finish(s, q);
    }
}

}  // namespace

extern "C" {

int64_t feast_nl_request_footprint(const feast_nl_request* r) {
    if (!r || r->n < 1 || r->nterms < 1 || !r->terms) return -1;
    const int64_t n = r->n, m = std::max<int64_t>(r->m0, 1), nc = std::max<int32_t>(r->nc, 1);
    int64_t dense = 0;
    for (int t = 0; t < r->nterms; ++t)
        if (r->terms[t].A) ++dense;
    const int64_t lu = (r->precision == FEAST_NL_FP64) ? 16 : 8;
    int64_t b = dense * 16 * n * n;                      // A_t, complex128
    b += nc * lu * n * n;                                // node factors
    if (r->precision == FEAST_NL_FP32_I8) b += dense * 7 * 2 * (n + 128) * (2 * n + 32);  // digit slices
    b += nc * lu * n * m;                                // node right-hand sides
    b += (int64_t)16 * n * m * (r->nterms + 8);          // subspace blocks
    b += (int64_t)64 << 20;                              // small blocks, reduced problem, slack
    return b;
}

int feast_nl_server_create(feast_nl_server** out, int32_t max_active, int64_t hbm_budget) {
    if (!out || max_active < 1 || max_active > 64 || hbm_budget < 1) return FEAST_NL_EINVAL;
    feast_nl_server* s = new (std::nothrow) feast_nl_server();
    if (!s) return FEAST_NL_ENOMEM;
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->factorer = std::thread(factor_loop, s);
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return FEAST_NL_OK;
}

int feast_nl_server_submit(feast_nl_server* s, const feast_nl_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return FEAST_NL_EINVAL;
    const int64_t fp = feast_nl_request_footprint(r);
    if (fp < 0 || r->m0 < 1 || r->nc < 1) return FEAST_NL_EINVAL;
    auto q = std::make_unique<Request>();
    q->r = *r;
    q->terms.assign(r->terms, r->terms + r->nterms);
    q->r.terms = nullptr;
    q->footprint = fp;
    q->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FEAST_NL_EINVAL;
        const uint64_t t = s->next_ticket++;
        s->reqs[t] = std::move(q);
        s->queue.push_back(t);
        *ticket = t;
    }
    s->cv_work.notify_all();
    return FEAST_NL_OK;
}

int feast_nl_server_poll(feast_nl_server* s, uint64_t ticket, int32_t* state) {
    if (!s || !state) return FEAST_NL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FEAST_NL_EINVAL;
    *state = it->second->state;
    return FEAST_NL_OK;
}

int feast_nl_server_wait(feast_nl_server* s, uint64_t ticket, feast_nl_info* info,
                         double* latency_ms) {
    if (!s) return FEAST_NL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FEAST_NL_EINVAL;
    Request* q = it->second.get();
    ++q->waiters;                       // fetch refuses the ticket while this is non-zero
    s->cv_done.wait(lk, [&] { return q->state == 2; });
    --q->waiters;
    if (info) *info = q->info;
    if (latency_ms) *latency_ms = q->t_done - q->t_submit;
    return q->status;
}

int feast_nl_server_fetch(feast_nl_server* s, uint64_t ticket, int32_t capacity, int32_t* m_out,
                          double* lambda, void* X, double* relres, int32_t inside_only) {
    if (!s || !m_out || capacity < 0) return FEAST_NL_EINVAL;
    std::unique_ptr<Request> q;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state != 2) return FEAST_NL_EINVAL;
        if (it->second->waiters > 0) return FEAST_NL_EINVAL;   // another thread still waits on it
        q = std::move(it->second);
        s->reqs.erase(it);
    }
    const feast_nl_request& r = q->r;
    int out = 0;
    for (int i = 0; i < q->m && out < capacity; ++i) {
        const double re = q->lam[2 * i], im = q->lam[2 * i + 1];
        const double dx = (re - r.c_re) / r.ra, dy = (im - r.c_im) / r.rb;
        if (inside_only && !(dx * dx + dy * dy < 1.0)) continue;
        if (lambda) { lambda[2 * out] = re; lambda[2 * out + 1] = im; }
        if (relres) relres[out] = q->relres[i];
        if (X) {
            auto* Xo = static_cast<std::complex<double>*>(X);
            for (int64_t row = 0; row < r.n; ++row) Xo[row * capacity + out] = q->X[row * r.m0 + i];
        }
        ++out;
    }
    *m_out = out;
    return q->status;
}

int feast_nl_server_set_group_limit(feast_nl_server* s, int32_t limit) {
    if (!s || limit < 1) return FEAST_NL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->group_limit = limit;
    return FEAST_NL_OK;
}

int feast_nl_server_stats(feast_nl_server* s, int32_t* max_concurrent, int64_t* completed,
                          int32_t* max_group) {
    if (!s) return FEAST_NL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (max_concurrent) *max_concurrent = s->max_seen;
    if (completed) *completed = s->completed;
    if (max_group) *max_group = s->max_group;
    return FEAST_NL_OK;
}

void feast_nl_server_destroy(feast_nl_server* s) {
    if (!s) return;
    {
        // finish what was submitted, then stop the workers
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->queue.empty() && s->active == 0 && s->preparing == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_ready.notify_all();
    if (s->factorer.joinable()) s->factorer.join();
    for (auto& t : s->workers) t.join();
    delete s;
}

}  // extern "C"
