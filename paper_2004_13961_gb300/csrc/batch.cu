// batch.cu -- batched PCG over many independent problems (uneven sizes).
// FP64: all problems run as one CUDA graph, one branch per problem, each with
// Algorithm 1's loop in a conditional WHILE node on the device, so the kernels
// of different problems overlap and each problem stops at its own tolerance
// with a single launch and a single wait for the whole batch.  If the graph
// cannot be built, every problem runs on its own stream and the host advances
// all runs without blocking on any one of them.  Mixed-
// precision contexts (FP64 refinement around an FP32 inner PCG, whose steps
// need host decisions between refinements) run as concurrent solves, one host
// thread and stream each, a bounded number at a time.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "lsg_internal.cuh"

using namespace lsg;

// Concurrent whole solves (lsg_pcg_solve) on per-thread streams, at most
// kConc at a time; the caller's stream is ordered before and after them.
static int batch_concurrent(int count, lsg_ctx *const *ctxs, const double *const *F, double *const *u, double rtol,
                            int kmax, lsg_info *infos, cudaStream_t s0)
{
    constexpr int kConc = 8;
    int dev = 0;
    LSG_CK(cudaGetDevice(&dev));
    LSG_CK(cudaStreamSynchronize(s0));
    std::vector<int> status(count, LSG_OK);
    std::vector<lsg_info> inf(count);
    std::atomic<int> next{0};
    auto work = [&]() {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (int i; (i = next.fetch_add(1)) < count;) status[i] = LSG_ERR_CUDA;
            return;
        }
        for (int i; (i = next.fetch_add(1)) < count;)
            status[i] = lsg_pcg_solve(ctxs[i], F[i], u[i], rtol, kmax, &inf[i], (lsg_stream_t)s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < std::min(kConc, count); ++t) pool.emplace_back(work);
    for (auto &t : pool) t.join();
    int st = LSG_OK;
    for (int i = 0; i < count; ++i) {
        if (infos) infos[i] = inf[i];
        if (status[i] != LSG_OK && st == LSG_OK) st = status[i];
    }
    return st;
}

extern "C" int lsg_batch_solve(int count, lsg_ctx *const *ctxs, const double *const *F, double *const *u,
                               double rtol, int kmax, lsg_info *infos, lsg_stream_t stream)
{
    if (count < 0 || (count > 0 && (!ctxs || !F || !u)) || !(rtol >= 0.0) || kmax < 0) return LSG_ERR_ARG;
    if (count == 0) return LSG_OK;
    for (int i = 0; i < count; ++i)
        if (!ctxs[i] || !F[i] || !u[i]) return LSG_ERR_ARG;
    cudaStream_t s0 = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) ctxs[i]->stream = s0;  // lsg_destroy orders the release on it
    bool mixed = false;
    for (int i = 0; i < count; ++i) mixed = mixed || ctxs[i]->precision != LSG_FP64;
    if (mixed) {
        const int st = batch_concurrent(count, ctxs, F, u, rtol, kmax, infos, s0);
        for (int i = 0; i < count; ++i) ctxs[i]->stream = s0;  // the solves ran on streams that are gone
        return st;
    }
    {
        // FP64: every problem's solve in one CUDA graph (one branch per problem, each with
        // its iteration loop in a conditional WHILE node), launched once on the caller's
        // stream; host arrays are staged in the contexts' buffers around it
        std::vector<const double *> gF(count);
        std::vector<double *> gx(count);
        std::vector<bool> hu(count, false);
        int st = LSG_OK;
        for (int i = 0; i < count && st == LSG_OK; ++i) {
            lsg_ctx *c = ctxs[i];
            const size_t bytes = sizeof(double) * (size_t)c->g.n;
            gF[i] = F[i];
            if (!is_device_ptr(F[i])) {
                if (cudaMemcpyAsync(c->fs, F[i], bytes, cudaMemcpyHostToDevice, s0) != cudaSuccess) st = LSG_ERR_CUDA;
                gF[i] = c->fs;
            }
            gx[i] = u[i];
            hu[i] = !is_device_ptr(u[i]);
            if (hu[i]) {
                if (cudaMemcpyAsync(c->xs, u[i], bytes, cudaMemcpyHostToDevice, s0) != cudaSuccess) st = LSG_ERR_CUDA;
                gx[i] = c->xs;
            }
        }
        if (st == LSG_OK) {
            PcgGraph G;
            st = pcg_graph_build(G, count, ctxs, gF.data(), gx.data());
            if (st == LSG_OK) {
                std::vector<int> status(count, LSG_OK);
                std::vector<lsg_info> inf(count);
                st = pcg_graph_run(G, ctxs, rtol, kmax, s0, inf.data(), status.data());
                for (int i = 0; i < count; ++i) {
                    if (infos) infos[i] = inf[i];
                    if (hu[i] && cudaMemcpyAsync(u[i], gx[i], sizeof(double) * (size_t)ctxs[i]->g.n,
                                                 cudaMemcpyDeviceToHost, s0) != cudaSuccess)
                        st = LSG_ERR_CUDA;
                }
                if (cudaStreamSynchronize(s0) != cudaSuccess) st = LSG_ERR_CUDA;
                pcg_graph_destroy(G);
                return st;
            }
            pcg_graph_destroy(G);
            cudaGetLastError();
        }
        if (st != LSG_OK && st != LSG_ERR_CUDA) return st;
        // the graph could not be built: the host-driven interleaving below
    }
    std::vector<cudaStream_t> st(count, nullptr);
    std::vector<PcgRun> runs(count);
    std::vector<bool> fin(count, false), hostu(count, false);
    std::vector<const double *> dF(count);
    std::vector<double *> du(count);
    cudaEvent_t fork;
    LSG_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    LSG_CK(cudaEventRecord(fork, s0));
    int status = LSG_OK;
    for (int i = 0; i < count; ++i) {
        runs[i] = PcgRun{};
        LSG_CK(cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking));
        LSG_CK(cudaStreamWaitEvent(st[i], fork, 0));
        lsg_ctx *c = ctxs[i];
        const long long n = c->g.n;
        if (is_device_ptr(F[i])) {
            dF[i] = F[i];
        } else {
            LSG_CK(cudaMemcpyAsync(c->fs, F[i], sizeof(double) * n, cudaMemcpyHostToDevice, st[i]));
            dF[i] = c->fs;
        }
        hostu[i] = !is_device_ptr(u[i]);
        du[i] = u[i];
        if (hostu[i]) {
            du[i] = c->xs;
            LSG_CK(cudaMemcpyAsync(du[i], u[i], sizeof(double) * n, cudaMemcpyHostToDevice, st[i]));
        }
        int s = pcg_start(runs[i], c, dF[i], du[i], rtol, kmax, st[i]);
        if (s != LSG_OK) {
            fin[i] = true;
            runs[i].status = s;
            if (status == LSG_OK) status = s;
        }
    }
    int left = 0;
    for (int i = 0; i < count; ++i) left += fin[i] ? 0 : 1;
    while (left > 0) {
        bool progressed = false;
        for (int i = 0; i < count; ++i) {
            if (fin[i]) continue;
            int ph = runs[i].phase, la = runs[i].launched;
            bool f = false;
            int s = pcg_poll(runs[i], st[i], false, &f);
            if (f || s != LSG_OK) {
                fin[i] = true;
                --left;
                if (s != LSG_OK && status == LSG_OK) status = s;
            }
            if (f || runs[i].phase != ph || runs[i].launched != la) progressed = true;
        }
        if (!progressed) std::this_thread::yield();
    }
    for (int i = 0; i < count; ++i) {
        lsg_ctx *c = ctxs[i];
        if (hostu[i])
            LSG_CK(cudaMemcpyAsync(u[i], du[i], sizeof(double) * c->g.n, cudaMemcpyDeviceToHost, st[i]));
        cudaEvent_t j;
        LSG_CK(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
        LSG_CK(cudaEventRecord(j, st[i]));
        LSG_CK(cudaStreamWaitEvent(s0, j, 0));
        LSG_CK(cudaStreamSynchronize(st[i]));
        cudaEventDestroy(j);
        if (infos) pcg_info(runs[i], &infos[i]);
        pcg_release(runs[i]);
        cudaStreamDestroy(st[i]);
    }
    cudaEventDestroy(fork);
    return status;
}
