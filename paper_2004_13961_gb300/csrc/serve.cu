// serve.cu -- continuous batching of solve requests on one GPU.
//
// Requests wait in a queue until a worker slot is free and their device
// footprint (lsg_footprint_bytes) fits the remaining HBM budget; among the
// queued requests that fit, the one with the smallest footprint is admitted
// (the earliest on ties), so short solves are not held behind large ones --
// unless the oldest queued request has waited longer than the aging bound, in
// which case it alone is admitted next (as soon as it fits), so large requests
// are not starved.  Each admitted request runs on its own stream -- setup
// (tables, M, ILU(0)), load vector, PCG -- with its vectors in stream-ordered
// device memory, so the kernels of all in-flight requests overlap on the
// device; a finished request releases its context on its own stream (no
// device-wide synchronisation) and frees its slot and budget for the next one
// at once.  Latency runs from submit to the solution in host memory.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <stdlib.h>
#include <string.h>

#include "lsg_internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Pending {
    lsg_request req;
    std::vector<double> a, b, f;
    size_t fp;
    clk::time_point t0;
};

}  // namespace

struct lsg_server {
    size_t budget = 0, used = 0;
    double aging_ms = 2000.0;
    int max_inflight = 1, active = 0, device = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::vector<lsg_result> done;
    std::vector<std::thread> workers;
};

static void run_one(lsg_server *S, Pending &p, lsg_result &res)
{
    res.id = p.req.id;
    res.u = nullptr;
    res.n = 0;
    memset(&res.info, 0, sizeof res.info);
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        res.info.status = LSG_ERR_CUDA;
        return;
    }
    const lsg_request &q = p.req;
    lsg_ctx *ctx = nullptr;
    int st = lsg_setup_ex(&ctx, q.d, q.N, q.T, q.Q, p.a.data(), p.b.data(), q.precision, LSG_SETUP_SHARED_GPU,
                          (lsg_stream_t)s);
    if (st == LSG_OK) {
        const long long n = lsg_query(ctx, LSG_Q_UNKNOWNS);
        // F and u live on the device (stream-ordered allocations from the pool)
        double *dF = nullptr, *du = nullptr;
        double *u = (double *)malloc(sizeof(double) * n);
        if (!u || cudaMallocAsync((void **)&dF, sizeof(double) * n, s) != cudaSuccess ||
            cudaMallocAsync((void **)&du, sizeof(double) * n, s) != cudaSuccess) {
            cudaGetLastError();
            st = LSG_ERR_NOMEM;
        } else {
            st = lsg_load_vector(ctx, p.f.data(), dF, (lsg_stream_t)s);
            if (st == LSG_OK && cudaMemsetAsync(du, 0, sizeof(double) * n, s) != cudaSuccess) st = LSG_ERR_CUDA;
            if (st == LSG_OK) st = lsg_pcg_solve(ctx, dF, du, q.rtol, q.kmax, &res.info, (lsg_stream_t)s);
            if ((st == LSG_OK || st == LSG_ERR_NOT_CONVERGED) &&
                (cudaMemcpyAsync(u, du, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
                st = LSG_ERR_CUDA;
        }
        if (dF) cudaFreeAsync(dF, s);
        if (du) cudaFreeAsync(du, s);
        res.u = u;
        res.n = u ? n : 0;
    }
    if (ctx) lsg_destroy(ctx);  // ordered on s
    cudaStreamDestroy(s);
    res.info.status = st;
    res.latency_ms = std::chrono::duration<double, std::milli>(clk::now() - p.t0).count();
}

static void worker(lsg_server *S)
{
    for (;;) {
        Pending p;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) return;
                // smallest footprint first among the queued requests that fit (ties:
                // the earliest), so short solves are not held behind large ones; a
                // request older than the aging bound goes next, alone (the queue is in
                // arrival order, so the front is the oldest)
                auto it = S->queue.end();
                const bool aged = !S->queue.empty() &&
                                  std::chrono::duration<double, std::milli>(clk::now() - S->queue.front().t0).count() >
                                      S->aging_ms;
                if (aged) {
                    if (S->used + S->queue.front().fp <= S->budget) it = S->queue.begin();
                } else {
                    for (auto jt = S->queue.begin(); jt != S->queue.end(); ++jt)
                        if (S->used + jt->fp <= S->budget && (it == S->queue.end() || jt->fp < it->fp)) it = jt;
                }
                if (it != S->queue.end()) {
                    p = std::move(*it);
                    S->queue.erase(it);
                    S->used += p.fp;
                    S->active += 1;
                    break;
                }
                // wake up for the aging bound too: a queued request may become the oldest
                S->cv.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
        lsg_result res;
        run_one(S, p, res);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= p.fp;
            S->active -= 1;
            S->done.push_back(res);
        }
        S->cv.notify_all();
    }
}

extern "C" {

int lsg_server_create(lsg_server **srv, size_t hbm_budget, int max_inflight)
{
    if (!srv || hbm_budget == 0 || max_inflight < 1 || max_inflight > 256) return LSG_ERR_ARG;
    lsg_server *S = new lsg_server();
    S->budget = hbm_budget;
    S->max_inflight = max_inflight;
    cudaGetDevice(&S->device);
    for (int i = 0; i < max_inflight; ++i) S->workers.emplace_back(worker, S);
    *srv = S;
    return LSG_OK;
}

int lsg_server_set_aging(lsg_server *S, double ms)
{
    if (!S || !(ms > 0.0)) return LSG_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->aging_ms = ms;
    return LSG_OK;
}

int lsg_server_submit(lsg_server *S, const lsg_request *req)
{
    if (!S || !req || !req->a || !req->b || !req->f) return LSG_ERR_ARG;
    int Q = req->Q <= 0 ? req->N + 2 : req->Q;
    size_t fp = lsg_footprint_bytes(req->d, req->N, req->T, Q, req->precision);
    if (fp == 0) return LSG_ERR_ARG;
    long long n = 1;
    for (int i = 0; i < req->d; ++i) n *= req->N - 1;
    fp += 2 * sizeof(double) * (size_t)n;  // the request's F and u on the device
    if (fp > S->budget) return LSG_ERR_NOMEM;
    Pending p;
    p.req = *req;
    p.req.Q = Q;
    long long nq = 1;
    for (int i = 0; i < req->d; ++i) nq *= Q;
    p.a.assign(req->a, req->a + nq);
    p.b.assign(req->b, req->b + nq);
    p.f.assign(req->f, req->f + nq);
    p.req.a = p.req.b = p.req.f = nullptr;
    p.fp = fp;
    p.t0 = clk::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->queue.push_back(std::move(p));
    }
    S->cv.notify_all();
    return LSG_OK;
}

int lsg_server_poll(lsg_server *S, lsg_result *out, int max, int *count)
{
    if (!S || !count || (max > 0 && !out)) return LSG_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.erase(S->done.begin());
    }
    *count = k;
    return LSG_OK;
}

int lsg_server_drain(lsg_server *S)
{
    if (!S) return LSG_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait(lk, [S] { return S->queue.empty() && S->active == 0; });
    return LSG_OK;
}

int lsg_server_release(lsg_server *S, lsg_result *res)
{
    if (!S || !res) return LSG_ERR_ARG;
    free(res->u);
    res->u = nullptr;
    return LSG_OK;
}

int lsg_server_destroy(lsg_server *S)
{
    if (!S) return LSG_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &r : S->done) free(r.u);
    delete S;
    return LSG_OK;
}

}  // extern "C"
