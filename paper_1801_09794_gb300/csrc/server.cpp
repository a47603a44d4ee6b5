// Serving loop: continuous batching of independent NLFEAST requests.
//
// A request is one whole run of Algorithm 1 (create + set_contour + solve) on
// its own handle and CUDA stream.  Worker threads (max_active of them) take
// requests in submission order; the head of the queue is admitted while the
// summed device-memory footprint of the running requests stays within the
// budget (a request that exceeds the budget on its own runs when nothing else
// does).  Requests in flight overlap on the GPU: one request's latency-bound
// reduced eigenvalue stage (one CTA) runs beside another's node
// factorisations and solves.  Each request's arithmetic is the same as when it
// runs alone (every kernel reduces in a fixed order), so its results do not
// depend on what else is in flight.
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
    int status = 0;
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
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int64_t budget = 0, in_use = 0;
    int active = 0, max_seen = 0;
    int64_t completed = 0;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// Runs one request to completion on its own handle; fills its results.
void run_request(Request& q) {
    feast_nl_handle* h = nullptr;
    const feast_nl_request& r = q.r;
    int st = feast_nl_create(&h, r.n, r.nterms, q.terms.data(), r.precision, nullptr);
    if (st == FEAST_NL_OK)
        st = feast_nl_set_contour(h, r.c_re, r.c_im, r.ra, r.rb, r.nc, r.rule);
    if (st == FEAST_NL_OK) {
        st = feast_nl_solve(h, r.m0, r.tol, r.maxit, r.seed, nullptr, &q.info);
        if (st == FEAST_NL_OK || st == FEAST_NL_ENOT_CONVERGED || st == FEAST_NL_ETOO_MANY) {
            q.lam.assign(2 * (size_t)r.m0, 0.0);
            q.relres.assign((size_t)r.m0, 0.0);
            q.X.assign((size_t)r.n * r.m0, std::complex<double>(0.0, 0.0));
            int m = 0;
            const int g = feast_nl_get_eigpairs(h, r.m0, &m, q.lam.data(), q.X.data(),
                                                q.relres.data(), 0);
            if (g != FEAST_NL_OK) st = g;
            q.m = m;
        }
    }
    if (st != FEAST_NL_OK) q.error = feast_nl_last_error();
    q.status = st;
    if (h) feast_nl_destroy(h);
}

void worker_loop(feast_nl_server* s) {
    for (;;) {
        Request* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty()) return false;
                const Request& head = *s->reqs[s->queue.front()];
                return s->active == 0 || s->in_use + head.footprint <= s->budget;
            });
            if (s->stop && s->queue.empty()) return;
            if (s->stop) return;
            const uint64_t t = s->queue.front();
            s->queue.pop_front();
            q = s->reqs[t].get();
            s->in_use += q->footprint;
            s->active += 1;
            s->max_seen = std::max(s->max_seen, s->active);
            q->state = 1;
            q->t_start = now_ms();
        }
        run_request(*q);
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
    s->cv_done.wait(lk, [&] { return q->state == 2; });
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

int feast_nl_server_stats(feast_nl_server* s, int32_t* max_concurrent, int64_t* completed) {
    if (!s) return FEAST_NL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (max_concurrent) *max_concurrent = s->max_seen;
    if (completed) *completed = s->completed;
    return FEAST_NL_OK;
}

void feast_nl_server_destroy(feast_nl_server* s) {
    if (!s) return;
    {
        // finish what was submitted, then stop the workers
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->queue.empty() && s->active == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

}  // extern "C"
