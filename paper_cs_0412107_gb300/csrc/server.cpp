// server.cpp -- the serving loop: estimate requests admitted into a pool by
// device memory and run with continuous batching.
//
// Callers submit requests from any thread; each carries its matrix (copied),
// its cycle schedule and the estimate it wants.  One engine thread owns the
// pool: it admits queued requests in arrival order while a slot and arena
// memory are free (a request that does not fit waits; nothing behind it
// overtakes it), advances every admitted matrix one step at a time -- so a
// request admitted while others are running shares their kernels from the
// next step on -- and completes a request as soon as its matrix has run its
// cycles: the estimate is read back, the slot and its memory are released and
// the waiting caller is woken.  Latency is measured from submission to the
// moment the result is ready.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mcinv.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    int64_t n = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    uint32_t matrix_id = 0;
    int64_t burnin = 0, samples = 0;
    mcinv_kind kind = MCINV_EST_DIAG;
    std::vector<double> q;
    int64_t ticket = -1;
    Clock::time_point submitted, admitted, done;
    bool finished = false;
    mcinv_status status = MCINV_OK;
    std::string error;
    std::vector<double> out, se;
};

}  // namespace

struct mcinv_server_ctx {
    mcinv_pool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;            // waiting for admission
    std::map<int64_t, std::shared_ptr<Request>> running;   // admitted, by ticket
    std::map<int64_t, std::shared_ptr<Request>> requests;  // every request not yet collected
    std::vector<double> latencies_ms;
    int64_t next_id = 1, completed = 0, steps = 0;
    double busy_s = 0.0;
    Clock::time_point started;
    bool stop = false;
    std::thread engine;
    std::string err;
};

static void engine_loop(mcinv_server_ctx *S)
{
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->running.empty(); });
        if (S->stop) return;
        // admission: arrival order, as long as the head fits
        while (!S->queue.empty()) {
            std::shared_ptr<Request> r = S->queue.front();
            int64_t ticket = -1;
            const mcinv_status st = mcinv_pool_submit(S->pool, r->n, r->row_ptr.data(), r->col.data(), r->val.data(),
                                                      r->matrix_id, r->burnin, r->samples,
                                                      r->kind == MCINV_EST_BLOCK ? 1 : 0, &ticket);
            if (st == MCINV_E_NOMEM && !S->running.empty()) break;  // wait for members to finish
            S->queue.pop_front();
            if (st != MCINV_OK) {
                r->status = st;
                r->error = mcinv_pool_last_error(S->pool);
                r->finished = true;
                r->done = Clock::now();
                S->cv_done.notify_all();
                continue;
            }
            r->ticket = ticket;
            r->admitted = Clock::now();
            S->running[ticket] = r;
        }
        if (S->running.empty()) continue;
        // one step for every member, outside the lock (the pool is only touched here)
        lk.unlock();
        const Clock::time_point t0 = Clock::now();
        mcinv_status st = mcinv_pool_step(S->pool);
        lk.lock();
        S->steps++;
        std::vector<std::shared_ptr<Request>> finished;
        for (auto it = S->running.begin(); it != S->running.end();) {
            int32_t done = 0;
            if (st == MCINV_OK) mcinv_pool_poll(S->pool, it->first, &done);
            if (st != MCINV_OK || done) {
                finished.push_back(it->second);
                it = S->running.erase(it);
            } else {
                ++it;
            }
        }
        lk.unlock();
        for (auto &r : finished) {
            if (st == MCINV_OK) {
                const size_t cnt = r->kind == MCINV_EST_DIAG ? (size_t)r->n
                                   : r->kind == MCINV_EST_TRACE ? 1
                                                                : (size_t)r->n * (size_t)r->n;
                r->out.resize(cnt);
                r->se.resize(cnt);
                r->status = mcinv_pool_estimate(S->pool, r->ticket, r->kind, r->q.empty() ? nullptr : r->q.data(),
                                                 r->out.data(), r->se.data());
            } else {
                r->status = st;
            }
            if (r->status != MCINV_OK) r->error = mcinv_pool_last_error(S->pool);
            mcinv_pool_release(S->pool, r->ticket);
        }
        const Clock::time_point t1 = Clock::now();
        lk.lock();
        S->busy_s += std::chrono::duration<double>(t1 - t0).count();
        for (auto &r : finished) {
            r->finished = true;
            r->done = t1;
            S->completed++;
            S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->done - r->submitted).count());
        }
        if (!finished.empty()) S->cv_done.notify_all();
    }
}

extern "C" mcinv_status mcinv_server_create(mcinv_server_t *out, const mcinv_pool_options *opt)
{
    if (!out) return MCINV_E_ARG;
    *out = nullptr;
    mcinv_server_ctx *S = new (std::nothrow) mcinv_server_ctx;
    if (!S) return MCINV_E_NOMEM;
    const mcinv_status st = mcinv_pool_create(&S->pool, opt);
    if (st != MCINV_OK) {
        delete S;
        return st;
    }
    S->started = Clock::now();
    S->engine = std::thread(engine_loop, S);
    *out = S;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_server_submit(mcinv_server_t S, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                            const double *val, uint32_t matrix_id, int64_t burnin, int64_t samples,
                                            mcinv_kind kind, const double *q_diag, int64_t *request)
{
    if (!S || !request || n <= 0 || !row_ptr || !col || !val) return MCINV_E_ARG;
    if (kind == MCINV_EST_TRACE && !q_diag) return MCINV_E_ARG;
    auto r = std::make_shared<Request>();
    r->n = n;
    r->row_ptr.assign(row_ptr, row_ptr + n + 1);
    const int64_t nnz = row_ptr[n];
    if (nnz < 0) return MCINV_E_ARG;
    r->col.assign(col, col + nnz);
    r->val.assign(val, val + nnz);
    r->matrix_id = matrix_id;
    r->burnin = burnin;
    r->samples = samples;
    r->kind = kind;
    if (q_diag) r->q.assign(q_diag, q_diag + n);
    r->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->requests[r->id] = r;
    S->queue.push_back(r);
    S->cv_work.notify_one();
    *request = r->id;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_server_wait(mcinv_server_t S, int64_t request, double timeout_s, double *out,
                                          double *se_out, double *latency_ms)
{
    if (!S) return MCINV_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(request);
    if (it == S->requests.end()) return MCINV_E_ARG;
    std::shared_ptr<Request> r = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->finished; });
    if (!ok) return MCINV_E_TIMEOUT;
    S->requests.erase(request);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->done - r->submitted).count();
    if (r->status != MCINV_OK) {
        S->err = r->error;
        return r->status;
    }
    if (out) std::memcpy(out, r->out.data(), r->out.size() * sizeof(double));
    if (se_out) std::memcpy(se_out, r->se.data(), r->se.size() * sizeof(double));
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_server_stats(mcinv_server_t S, mcinv_server_stats_t *st)
{
    if (!S || !st) return MCINV_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = S->completed;
    st->queued = (int64_t)S->queue.size();
    st->running = (int64_t)S->running.size();
    st->steps = S->steps;
    std::vector<double> l = S->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)std::floor(q * (l.size() - 1) + 0.5))]; };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = l.back();
    }
    st->elapsed_s = std::chrono::duration<double>(Clock::now() - S->started).count();
    st->busy_s = S->busy_s;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_server_reset_stats(mcinv_server_t S)
{
    if (!S) return MCINV_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies_ms.clear();
    S->completed = 0;
    S->steps = 0;
    S->busy_s = 0.0;
    S->started = Clock::now();
    return MCINV_OK;
}

extern "C" const char *mcinv_server_last_error(mcinv_server_t S) { return S ? S->err.c_str() : ""; }

extern "C" void mcinv_server_destroy(mcinv_server_t S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->engine.joinable()) S->engine.join();
    mcinv_pool_destroy(S->pool);
    delete S;
}
