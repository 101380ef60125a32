// pcg.cu -- Algorithm 1 (PCG) kept on the device.  Each iteration is a fixed
// sequence of kernels on one stream: z = M^-1 r (two sweeps), rho = r^T z and
// beta, p = z + beta p, w = K p (transforms), alpha = rho / p^T w, then
// x += alpha p, r -= alpha w and r^T r.  Every reduction uses a fixed grid and
// a last-block combine in block order, so results are bitwise reproducible.
// The stop test of Algorithm 1 is evaluated on the device and written to a
// `done` word; every kernel of later iterations returns at once when it is
// set.  The host queues iterations in chunks sized from the residual decrease
// seen so far (next_chunk), so it looks at the device state only a few times
// per solve and queues few iterations past the stop.
#include <math.h>

#include <algorithm>

#include "lsg_internal.cuh"

namespace lsg {

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// Returns true in every thread of the block that finishes last; that block
// then combines the partials (in block order) and resets the counter.
__device__ __forceinline__ bool last_block(unsigned *cnt)
{
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(cnt, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

__device__ __forceinline__ double combine(const double *red, int stride, int which, double *sh)
{
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(red + (size_t)b * stride + which);
    // fixed combine order: thread-strided partials then the block tree
    return block_sum(v, sh);
}

// r = F - Kx; nF2 = F.F; rr = r.r; initial stop test.
__global__ void __launch_bounds__(kRedThreads) k_init(long long n, const double *F, const double *Kx, double *r,
                                                     double *red, unsigned *cnt, PcgState *st)
{
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double f = F[i], ri = f - Kx[i];
        r[i] = ri;
        a += f * f;
        b += ri * ri;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        red[2 * blockIdx.x] = a;
        red[2 * blockIdx.x + 1] = b;
    }
    if (last_block(cnt)) {
        double nF2 = combine(red, 2, 0, sh);
        double rr = combine(red, 2, 1, sh);
        if (threadIdx.x == 0) {
            st->nF2 = nF2;
            st->rr = rr;
            st->k = 0;
            st->rho = 0.0;
            st->done = (rr <= st->eps2 * nF2 || st->kmax <= 0) ? 1 : 0;
            *cnt = 0;
        }
    }
}

// rho = r.z ; beta = rho / rho_old (first pass: beta = 0)
__global__ void __launch_bounds__(kRedThreads) k_rz(long long n, const double *r, const double *z, double *red,
                                                   unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a += r[i] * z[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double rho = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->beta = (st->k == 0) ? 0.0 : rho / st->rho;
            st->rho_old = st->rho;
            st->rho = rho;
            *cnt = 0;
        }
    }
}

// p = z + beta p   (p = z on the first pass)
__global__ void k_pupd(long long n, const double *z, double *p, const PcgState *st)
{
    if (st->done) return;
    const double beta = st->beta;
    const bool first = st->k == 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : z[i] + beta * p[i];
}

// pw = p.w ; alpha = rho / pw  (pw <= 0: stop, not converged)
__global__ void __launch_bounds__(kRedThreads) k_pw(long long n, const double *p, const double *w, double *red,
                                                   unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a += p[i] * w[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double pw = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->pw = pw;
            if (!(pw > 0.0)) {
                st->status = LSG_ERR_NOT_CONVERGED;
                st->done = 1;
            } else {
                st->alpha = st->rho / pw;
            }
            *cnt = 0;
        }
    }
}

// x += alpha p ; r -= alpha w ; rr = r.r ; k += 1 ; stop test of Algorithm 1
__global__ void __launch_bounds__(kRedThreads) k_xr(long long n, double *x, double *r, const double *p,
                                                   const double *w, double *red, unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    const double alpha = st->alpha;
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * w[i];
        r[i] = ri;
        a += ri * ri;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double rr = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->rr = rr;
            st->k += 1;
            if (rr <= st->eps2 * st->nF2 || st->k >= st->kmax) st->done = 1;
            *cnt = 0;
        }
    }
}

// tr = |F - Kx|^2 (true residual), nF2 refreshed
__global__ void __launch_bounds__(kRedThreads) k_true(long long n, const double *F, const double *Kx, double *red,
                                                     unsigned *cnt, PcgState *st)
{
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double f = F[i], d = f - Kx[i];
        a += d * d;
        b += f * f;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        red[2 * blockIdx.x] = a;
        red[2 * blockIdx.x + 1] = b;
    }
    if (last_block(cnt)) {
        double tr = combine(red, 2, 0, sh);
        double nf = combine(red, 2, 1, sh);
        if (threadIdx.x == 0) {
            st->tr = tr;
            st->nF2 = nf;
            *cnt = 0;
        }
    }
}

int next_chunk(ChunkPlan &P, int k, double rr, double target, int cap)
{
    // per-iteration factor of r^T r over the whole run and over the last chunk; the
    // faster of the two (PCG tends to speed up), so that the plan rarely overshoots
    int m = 2;
    if (k > 0 && rr > 0.0 && P.rr0 > 0.0 && target > 0.0) {
        double rate = pow(rr / P.rr0, 1.0 / k);
        if (k > P.k_prev && P.rr_prev > 0.0) {
            const double last = pow(rr / P.rr_prev, 1.0 / (k - P.k_prev));
            if (last < rate) rate = last;
        }
        if (rate > 0.0 && rate < 1.0) {
            const double est = ceil(log(target / rr) / log(rate));
            m = est < 1.0 ? 1 : (est > cap ? cap : (int)est);
        } else {
            m = 4;  // no decrease seen yet
        }
    }
    P.rr_prev = rr;
    P.k_prev = k;
    return m < cap ? m : cap;
}

static int iteration(lsg_ctx *c, double *x, cudaStream_t s)
{
    const long long n = c->g.n;
    const int *done = &c->st->done;
    unsigned *cnt = c->counters + 4;
    LSG_TRY(apply_Minv(c, c->r, c->z, done, s));
    ::lsg::count_launch();
    k_rz<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->r, c->z, c->red, cnt, c->st);
    ::lsg::count_launch();
    k_pupd<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->z, c->p, c->st);
    int slot;
    LSG_TRY(prof_begin(c, PROF_KX, s, &slot));
    LSG_TRY(apply_K(c, c->p, c->wv, done, s));
    LSG_TRY(prof_end(c, slot, s));
    ::lsg::count_launch();
    k_pw<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->p, c->wv, c->red, cnt, c->st);
    ::lsg::count_launch();
    k_xr<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, c->r, c->p, c->wv, c->red, cnt, c->st);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

// Copy the device state (and the device error word) to the pinned mirror and
// mark the point with the run's event.
static int snapshot(PcgRun &R, cudaStream_t s)
{
    lsg_ctx *c = R.c;
    LSG_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaMemcpyAsync(&c->st_host->pad[0], c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaEventRecord(R.ev, s));
    return LSG_OK;
}

int pcg_start(PcgRun &R, lsg_ctx *c, const double *F, double *x, double rtol, int kmax, cudaStream_t s)
{
    R.c = c;
    R.F = F;
    R.x = x;
    R.kmax = kmax;
    R.launched = 0;
    R.chunk = 2;
    R.tag0 = -1;
    R.plan = ChunkPlan{};
    R.phase = 0;
    R.status = LSG_OK;
    if (!R.ev) LSG_CK(cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming));
    const long long n = c->g.n;
    PcgState *h = c->st_host;
    *h = PcgState{};
    h->eps2 = rtol * rtol;
    h->kmax = kmax;
    LSG_CK(cudaMemcpyAsync(c->st, h, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    LSG_CK(cudaMemsetAsync(c->counters + 4, 0, sizeof(unsigned), s));
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(apply_K(c, x, c->wv, nullptr, s));
    ::lsg::count_launch();
    k_init<<<kRedBlocks, kRedThreads, 0, s>>>(n, F, c->wv, c->r, c->red, c->counters + 4, c->st);
    LSG_CK(cudaGetLastError());
    return snapshot(R, s);
}

static int dev_err_status(int e)
{
    switch (e) {
    case DERR_NONE: return LSG_OK;
    case DERR_BREAKDOWN: return LSG_ERR_ILU_BREAKDOWN;
    case DERR_TIMEOUT: return LSG_ERR_TIMEOUT;
    case DERR_NONFINITE: return LSG_ERR_NONFINITE;
    default: return LSG_ERR_CUDA;
    }
}

// Advance a run by one step if its last snapshot has landed.  Non-blocking
// unless `wait` is set.  *finished becomes true once the run is complete.
int pcg_poll(PcgRun &R, cudaStream_t s, bool wait, bool *finished)
{
    *finished = false;
    if (R.phase == 2) {
        *finished = true;
        return R.status;
    }
    if (wait) {
        LSG_CK(cudaEventSynchronize(R.ev));
    } else {
        cudaError_t q = cudaEventQuery(R.ev);
        if (q == cudaErrorNotReady) return LSG_OK;
        LSG_CK(q);
    }
    lsg_ctx *c = R.c;
    PcgState *h = c->st_host;
    int derr = dev_err_status(h->pad[0]);
    if (R.phase == 1 || derr == LSG_ERR_TIMEOUT) {
        if (R.tag0 >= 0) prof_mark_done(c, R.tag0, h->k);
        R.status = h->status;
        if (R.status == LSG_OK && !(h->rr <= h->eps2 * h->nF2)) R.status = LSG_ERR_NOT_CONVERGED;
        if (derr != LSG_OK) R.status = derr;
        R.phase = 2;
        *finished = true;
        return R.status;
    }
    if (h->done || R.launched >= R.kmax) {
        // true residual in FP64, then finish
        LSG_TRY(apply_K(c, R.x, c->wv, nullptr, s));
        ::lsg::count_launch();
        k_true<<<kRedBlocks, kRedThreads, 0, s>>>(c->g.n, R.F, c->wv, c->red, c->counters + 4, c->st);
        LSG_CK(cudaGetLastError());
        R.phase = 1;
        return snapshot(R, s);
    }
    if (R.launched == 0) R.plan.rr0 = h->rr;
    int m = std::min(next_chunk(R.plan, h->k, h->rr, h->eps2 * h->nF2, 32), R.kmax - R.launched);
    for (int it = 0; it < m; ++it) {
        const int tag = prof_tag(c);
        if (R.tag0 < 0) R.tag0 = tag;
        prof_set_tag(c, tag);
        LSG_TRY(iteration(c, R.x, s));
    }
    prof_set_tag(c, -1);
    R.launched += m;
    return snapshot(R, s);
}

void pcg_info(const PcgRun &R, lsg_info *info)
{
    if (!info) return;
    const PcgState *h = R.c->st_host;
    info->iters = h->k;
    info->outer_iters = 0;
    double nF = sqrt(h->nF2);
    info->relres = nF > 0 ? sqrt(h->rr) / nF : sqrt(h->rr);
    info->relres_true = nF > 0 ? sqrt(h->tr) / nF : sqrt(h->tr);
    info->status = R.status;
}

void pcg_release(PcgRun &R)
{
    if (R.ev) cudaEventDestroy(R.ev);
    R.ev = nullptr;
}

// ---------------------------------------------------------------------------
// Algorithm 1 as one CUDA graph.  The loop runs on the device: a conditional WHILE
// node whose body is one iteration (the same kernels as above) ends with a
// one-thread kernel that sets the loop condition from the device-side stop test,
// so nothing is launched past convergence and the host waits once per solve.

__global__ void k_loop_cond(cudaGraphConditionalHandle h, const PcgState *st)
{
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// Appends one solve to the graph being captured on stream s: the state upload from
// the pinned mirror (read when the graph runs), r = F - K x, the WHILE node with one
// iteration in its body (captured on the helper stream bs), the true residual and
// the state download.  *body_launches: kernels per loop pass.
static int capture_pcg(lsg_ctx *c, const double *F, double *x, cudaStream_t s, cudaStream_t bs,
                       long long *body_launches)
{
    const long long n = c->g.n;
    LSG_CK(cudaMemcpyAsync(c->st, c->st_host, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    LSG_CK(cudaMemsetAsync(c->counters + 4, 0, sizeof(unsigned), s));
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(apply_K(c, x, c->wv, nullptr, s));
    ::lsg::count_launch();
    k_init<<<kRedBlocks, kRedThreads, 0, s>>>(n, F, c->wv, c->r, c->red, c->counters + 4, c->st);
    LSG_CK(cudaGetLastError());
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    LSG_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    LSG_CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    ::lsg::count_launch();
    k_loop_cond<<<1, 1, 0, s>>>(h, c->st);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    LSG_CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
    LSG_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    LSG_CK(cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
    const long long l0 = launches_so_far();
    int st = iteration(c, x, bs);
    if (st == LSG_OK) {
        ::lsg::count_launch();
        k_loop_cond<<<1, 1, 0, bs>>>(h, c->st);
        if (cudaGetLastError() != cudaSuccess) st = LSG_ERR_CUDA;
    }
    *body_launches = launches_so_far() - l0;
    cudaGraph_t body = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &body);
    LSG_TRY(st);
    LSG_CK(e);
    LSG_TRY(apply_K(c, x, c->wv, nullptr, s));
    ::lsg::count_launch();
    k_true<<<kRedBlocks, kRedThreads, 0, s>>>(n, F, c->wv, c->red, c->counters + 4, c->st);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaMemcpyAsync(&c->st_host->pad[0], c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return LSG_OK;
}

void PcgGraph::reset()
{
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    nctx = 0;
}

// Captures `count` solves (context i on F[i], x[i]) into one graph, each on its own
// branch forked from the capture stream, and instantiates it.
int pcg_graph_build(PcgGraph &G, int count, lsg_ctx *const *ctxs, const double *const *F, double *const *x)
{
    G.reset();
    if (!G.cap) LSG_CK(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    if (!G.body) LSG_CK(cudaStreamCreateWithFlags(&G.body, cudaStreamNonBlocking));
    if ((int)G.branch.size() < count) {
        const size_t old = G.branch.size();
        G.branch.resize(count, nullptr);
        for (size_t i = old; i < G.branch.size(); ++i)
            LSG_CK(cudaStreamCreateWithFlags(&G.branch[i], cudaStreamNonBlocking));
    }
    if (!G.fork) LSG_CK(cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming));
    if (G.join.size() < (size_t)count) {
        const size_t old = G.join.size();
        G.join.resize(count, nullptr);
        for (size_t i = old; i < G.join.size(); ++i)
            LSG_CK(cudaEventCreateWithFlags(&G.join[i], cudaEventDisableTiming));
    }
    const long long l0 = launches_so_far();
    LSG_CK(cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeRelaxed));
    int st = LSG_OK;
    cudaError_t e = cudaEventRecord(G.fork, G.cap);
    if (e != cudaSuccess) st = LSG_ERR_CUDA;
    G.body_launches.assign(count, 0);
    for (int i = 0; i < count && st == LSG_OK; ++i) {
        cudaStream_t b = count == 1 ? G.cap : G.branch[i];
        if (count > 1 && cudaStreamWaitEvent(b, G.fork, 0) != cudaSuccess) st = LSG_ERR_CUDA;
        if (st == LSG_OK) st = capture_pcg(ctxs[i], F[i], x[i], b, G.body, &G.body_launches[i]);
        if (st == LSG_OK && count > 1 &&
            (cudaEventRecord(G.join[i], b) != cudaSuccess || cudaStreamWaitEvent(G.cap, G.join[i], 0) != cudaSuccess))
            st = LSG_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(G.cap, &graph);
    if (st == LSG_OK && e != cudaSuccess) {
        record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        st = LSG_ERR_CUDA;
    }
    if (st == LSG_OK) {
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        if (e != cudaSuccess) {
            record_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
            G.exec = nullptr;
            st = LSG_ERR_CUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    // kernels count when the graph runs, not when they are captured
    long long body = 0;
    for (long long b : G.body_launches) body += b;
    G.fixed_launches = launches_so_far() - l0 - body;
    count_launches(-(launches_so_far() - l0));
    G.nctx = st == LSG_OK ? count : 0;
    return st;
}

// Runs a built graph on stream s with the given tolerance and iteration limit, and
// waits for it.  infos/status per context.
int pcg_graph_run(PcgGraph &G, lsg_ctx *const *ctxs, double rtol, int kmax, cudaStream_t s, lsg_info *infos,
                  int *status)
{
    for (int i = 0; i < G.nctx; ++i) {
        PcgState *h = ctxs[i]->st_host;
        *h = PcgState{};
        h->eps2 = rtol * rtol;
        h->kmax = kmax;
    }
    LSG_CK(cudaGraphLaunch(G.exec, s));
    LSG_CK(cudaStreamSynchronize(s));
    long long runs = G.fixed_launches;
    int first = LSG_OK;
    for (int i = 0; i < G.nctx; ++i) {
        const PcgState *h = ctxs[i]->st_host;
        int st = h->status;
        if (st == LSG_OK && !(h->rr <= h->eps2 * h->nF2)) st = LSG_ERR_NOT_CONVERGED;
        const int derr = dev_err_status(h->pad[0]);
        if (derr != LSG_OK) st = derr;
        // the body ran once per completed pass, plus the pass that found p^T w <= 0
        runs += G.body_launches[i] * (long long)(h->k + (h->status != LSG_OK ? 1 : 0));
        if (infos) {
            lsg_info &in = infos[i];
            in.iters = h->k;
            in.outer_iters = 0;
            const double nF = sqrt(h->nF2);
            in.relres = nF > 0 ? sqrt(h->rr) / nF : sqrt(h->rr);
            in.relres_true = nF > 0 ? sqrt(h->tr) / nF : sqrt(h->tr);
            in.status = st;
        }
        if (status) status[i] = st;
        if (st != LSG_OK && first == LSG_OK) first = st;
    }
    count_launches(runs);
    return first;
}

void pcg_graph_destroy(PcgGraph &G)
{
    G.reset();
    for (cudaStream_t b : G.branch)
        if (b) cudaStreamDestroy(b);
    G.branch.clear();
    for (cudaEvent_t e : G.join)
        if (e) cudaEventDestroy(e);
    G.join.clear();
    if (G.fork) cudaEventDestroy(G.fork);
    if (G.cap) cudaStreamDestroy(G.cap);
    if (G.body) cudaStreamDestroy(G.body);
    G.fork = nullptr;
    G.cap = G.body = nullptr;
}

// PCG on device-resident F and x (x: initial guess in, iterate out); blocking.
// Contexts set up with LSG_SETUP_PROFILE run the host-driven loop (its per-kernel
// events cannot be recorded inside a graph's loop); the others run the solve as one
// graph, captured once per (F, x) pair and kept with the context.
int pcg_fp64(lsg_ctx *c, const double *F, double *x, double rtol, int kmax, lsg_info *info, cudaStream_t s)
{
    if (!c->prof && !c->no_graph) {
        if (!c->graph) c->graph = new PcgGraph();
        PcgGraph &G = *c->graph;
        int st = LSG_OK;
        if (!G.exec || G.F0 != F || G.x0 != x) {
            st = pcg_graph_build(G, 1, &c, &F, &x);
            G.F0 = F;
            G.x0 = x;
        }
        if (st == LSG_OK) {
            int status = LSG_OK;
            lsg_info tmp;
            st = pcg_graph_run(G, &c, rtol, kmax, s, &tmp, &status);
            if (info) *info = tmp;
            return st == LSG_OK ? status : st;
        }
        // the graph could not be built: use the host-driven loop from now on
        c->no_graph = 1;
        G.reset();
    }
    PcgRun R{};
    int st = pcg_start(R, c, F, x, rtol, kmax, s);
    bool fin = false;
    while (st == LSG_OK && !fin) st = pcg_poll(R, s, true, &fin);
    if (fin) st = R.status;
    pcg_info(R, info);
    if (info) info->status = st;
    pcg_release(R);
    return st;
}

// ---------------------------------------------------------------------------
// Mixed precision (a FP64 refinement loop around an FP32 inner PCG).
//
// Outer loop in FP64: r = F - K u (FP64 transforms), stop when
// ||r|| <= rtol ||F||; otherwise solve K e = r / ||r|| approximately with PCG
// in FP32 (FP32 vectors, FP32 ILU(0) factors, low-precision transforms, FP64
// dot-product accumulation) to a loose relative tolerance, and update
// u += ||r|| e in FP64.  Residual normalisation keeps the FP32 inner problem
// well scaled at every refinement step.

__global__ void k_cast_scale(long long n, const double *r, double scale, float *r32, float *x32)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        r32[i] = (float)(r[i] * scale);
        x32[i] = 0.f;
    }
}

// inner start: nF2 := r.r (reference), rr = r.r, k = 0
__global__ void __launch_bounds__(kRedThreads) k_init32(long long n, const float *r, double *red, unsigned *cnt,
                                                       PcgState *st)
{
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = r[i];
        a += v * v;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double rr = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->nF2 = rr;
            st->rr = rr;
            st->k = 0;
            st->rho = 0.0;
            st->status = LSG_OK;
            st->done = (rr <= st->eps2 * rr || st->kmax <= 0 || rr == 0.0) ? 1 : 0;
            *cnt = 0;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) k_rz32(long long n, const float *r, const float *z, double *red,
                                                     unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a += (double)r[i] * (double)z[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double rho = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->beta = (st->k == 0) ? 0.0 : rho / st->rho;
            st->rho_old = st->rho;
            st->rho = rho;
            *cnt = 0;
        }
    }
}

__global__ void k_pupd32(long long n, const float *z, float *p, const PcgState *st)
{
    if (st->done) return;
    const float beta = (float)st->beta;
    const bool first = st->k == 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : fmaf(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(kRedThreads) k_pw32(long long n, const float *p, const float *w, double *red,
                                                     unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a += (double)p[i] * (double)w[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double pw = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->pw = pw;
            if (!(pw > 0.0)) {
                st->status = LSG_ERR_NOT_CONVERGED;
                st->done = 1;
            } else {
                st->alpha = st->rho / pw;
            }
            *cnt = 0;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) k_xr32(long long n, float *x, float *r, const float *p, const float *w,
                                                     double *red, unsigned *cnt, PcgState *st)
{
    if (st->done) return;
    __shared__ double sh[32];
    const float alpha = (float)st->alpha;
    double a = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fmaf(alpha, p[i], x[i]);
        float ri = fmaf(-alpha, w[i], r[i]);
        r[i] = ri;
        a += (double)ri * (double)ri;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = a;
    if (last_block(cnt)) {
        double rr = combine(red, 1, 0, sh);
        if (threadIdx.x == 0) {
            st->rr = rr;
            st->k += 1;
            if (rr <= st->eps2 * st->nF2 || st->k >= st->kmax) st->done = 1;
            *cnt = 0;
        }
    }
}

__global__ void k_update64(long long n, double *u, const float *e, double scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] += scale * (double)e[i];
}

static int iteration32(lsg_ctx *c, cudaStream_t s)
{
    const long long n = c->g.n;
    const int *done = &c->st->done;
    unsigned *cnt = c->counters + 4;
    LSG_TRY(apply_Minv32(c, c->r32, c->z32, done, s));
    ::lsg::count_launch();
    k_rz32<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->r32, c->z32, c->red, cnt, c->st);
    ::lsg::count_launch();
    k_pupd32<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->z32, c->p32, c->st);
    int slot;
    LSG_TRY(prof_begin(c, PROF_KX_LO, s, &slot));
    LSG_TRY(apply_K_tc(c, c->p32, c->w32, done, s));
    LSG_TRY(prof_end(c, slot, s));
    ::lsg::count_launch();
    k_pw32<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->p32, c->w32, c->red, cnt, c->st);
    ::lsg::count_launch();
    k_xr32<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->e32, c->r32, c->p32, c->w32, c->red, cnt, c->st);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

// r = F - K u in FP64 and its norm; returns rr and nF2 on the host.
static int outer_residual(lsg_ctx *c, const double *F, const double *u, double *rr, double *nF2, cudaStream_t s)
{
    PcgState *h = c->st_host;
    LSG_TRY(apply_K(c, u, c->wv, nullptr, s));
    ::lsg::count_launch();
    k_init<<<kRedBlocks, kRedThreads, 0, s>>>(c->g.n, F, c->wv, c->r, c->red, c->counters + 4, c->st);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaMemcpyAsync(h, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaStreamSynchronize(s));
    *rr = h->rr;
    *nF2 = h->nF2;
    return LSG_OK;
}

int pcg_mixed(lsg_ctx *c, const double *F, double *u, double rtol, int kmax, lsg_info *info, cudaStream_t s)
{
    const long long n = c->g.n;
    PcgState *h = c->st_host;
    // inner relative tolerance: three digits per refinement step; the
    // split-operand tensor-core product is accurate to ~1e-6..1e-5, so the
    // refinement contracts by about the inner tolerance per step
    const double inner_tol = 1e-3;
    const int max_outer = 40;
    *h = PcgState{};
    h->eps2 = rtol * rtol;
    h->kmax = 1;
    LSG_CK(cudaMemcpyAsync(c->st, h, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    LSG_CK(cudaMemsetAsync(c->counters + 4, 0, sizeof(unsigned), s));
    double rr = 0.0, nF2 = 0.0;
    LSG_TRY(outer_residual(c, F, u, &rr, &nF2, s));
    int total = 0, outer = 0, status = LSG_OK;
    double last_inner = 0.0;
    while (!(rr <= rtol * rtol * nF2)) {
        if (outer >= max_outer || total >= kmax) {
            status = LSG_ERR_NOT_CONVERGED;
            break;
        }
        const double rn = sqrt(rr);
        ::lsg::count_launch();
        k_cast_scale<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->r, 1.0 / rn, c->r32, c->e32);
        h->eps2 = inner_tol * inner_tol;
        h->kmax = kmax - total;
        h->done = 0;
        LSG_CK(cudaMemcpyAsync(&c->st->eps2, &h->eps2, sizeof(double), cudaMemcpyHostToDevice, s));
        LSG_CK(cudaMemcpyAsync(&c->st->kmax, &h->kmax, sizeof(int), cudaMemcpyHostToDevice, s));
        ::lsg::count_launch();
        k_init32<<<kRedBlocks, kRedThreads, 0, s>>>(n, c->r32, c->red, c->counters + 4, c->st);
        LSG_CK(cudaGetLastError());
        int launched = 0, tag0 = -1;
        ChunkPlan plan;
        for (;;) {
            LSG_CK(cudaMemcpyAsync(h, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
            LSG_CK(cudaStreamSynchronize(s));
            if (h->done || launched >= kmax - total) break;
            int e = read_dev_error(c, s);
            if (e != LSG_OK) return e;
            if (launched == 0) plan.rr0 = h->rr;
            int m = std::min(next_chunk(plan, h->k, h->rr, h->eps2 * h->nF2, 32), kmax - total - launched);
            for (int it = 0; it < m; ++it) {
                const int tag = prof_tag(c);
                if (tag0 < 0) tag0 = tag;
                prof_set_tag(c, tag);
                LSG_TRY(iteration32(c, s));
            }
            prof_set_tag(c, -1);
            launched += m;
        }
        if (tag0 >= 0) prof_mark_done(c, tag0, h->k);
        total += h->k;
        last_inner = h->nF2 > 0 ? sqrt(h->rr / h->nF2) : 0.0;
        int e = read_dev_error(c, s);
        if (e != LSG_OK) return e;
        if (h->k == 0) {
            status = LSG_ERR_NOT_CONVERGED;
            break;
        }
        ::lsg::count_launch();
        k_update64<<<kRedBlocks, kRedThreads, 0, s>>>(n, u, c->e32, rn);
        double prev = rr;
        LSG_TRY(outer_residual(c, F, u, &rr, &nF2, s));
        ++outer;
        if (!(rr < 0.99 * prev) && !(rr <= rtol * rtol * nF2)) {
            status = LSG_ERR_NOT_CONVERGED;  // refinement stagnated
            break;
        }
    }
    if (info) {
        info->iters = total;
        info->outer_iters = outer;
        info->relres = last_inner;
        info->relres_true = nF2 > 0 ? sqrt(rr / nF2) : sqrt(rr);
        info->status = status;
    }
    return status;
}

}  // namespace lsg
