// api.cu -- the extern "C" entry points declared in include/lsg.h: argument
// checks, staging of host arrays, context lifetime, exports.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "lsg_internal.cuh"

namespace lsg {

static thread_local char g_last_error[512] = "";
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int dalloc(lsg_ctx *c, void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) return LSG_OK;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LSG_ERR_NOMEM;
    }
    c->bytes += bytes;
    return LSG_OK;
}

int read_dev_error(lsg_ctx *c, cudaStream_t s)
{
    int e = 0;
    LSG_CK(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaStreamSynchronize(s));
    switch (e) {
    case DERR_NONE: return LSG_OK;
    case DERR_BREAKDOWN: return LSG_ERR_ILU_BREAKDOWN;
    case DERR_TIMEOUT: return LSG_ERR_TIMEOUT;
    case DERR_NONFINITE: return LSG_ERR_NONFINITE;
    default: return LSG_ERR_CUDA;
    }
}

// A compute call starts with a clear device error word, so that a context stays
// usable after a call that reported a timeout; an ILU(0) breakdown found at
// setup stays recorded (the factors are not valid).
int clear_dev_error(lsg_ctx *c, cudaStream_t s)
{
    if (c->setup_status != LSG_OK) return LSG_OK;
    LSG_CK(cudaMemsetAsync(c->err, 0, sizeof(int), s));
    return LSG_OK;
}

struct Sizes {
    size_t tab, grid, series, band, Lv, Uv, Mkeep, ws, vec, lines;
};

static Sizes sizes_for(const Geom &g, int precision, unsigned flags)
{
    Sizes z{};
    size_t T1 = g.T + 1, ns = 1;
    for (int i = 0; i < g.d; ++i) ns *= T1;
    size_t vsz = precision == LSG_FP64 ? 8 : 4;
    z.tab = 4 * (size_t)g.QhP * g.KP * 8;
    z.grid = (size_t)g.nq * 8;
    z.series = ns * 8;
    z.band = T1 * g.n1 * g.W1 * 8;
    const bool cst = (flags & LSG_SETUP_CONST_PRECOND) != 0;  // no factors: M_0 is solved directly
    z.Lv = cst ? 0 : (size_t)g.n * g.SL * vsz;
    z.Uv = cst ? 0 : (size_t)g.n * g.SU * vsz;
    z.Mkeep = (flags & LSG_SETUP_KEEP_M) ? (size_t)g.n * g.S * 8 : 0;
    z.ws = workspace_elems(g) * 8;
    z.vec = (size_t)g.n * 8;
    z.lines = (size_t)g.nlines * 4;
    return z;
}

static size_t footprint(const Geom &g, int precision, unsigned flags)
{
    Sizes z = sizes_for(g, precision, flags);
    size_t b = 2 * (size_t)g.Q * 8 + z.tab + 3 * z.grid + 2 * z.series + 2 * z.band + z.Lv + z.Uv +
               z.Mkeep + z.ws + 7 * z.vec + (size_t)g.n * 4 * 2 + 2 * z.lines + 64 + kRedBlocks * 16 +
               sizeof(PcgState);
    if (precision != LSG_FP64) b += 6 * (size_t)g.n * 4 + 2 * (size_t)g.nq * 4 + 2 * z.vec + tc_ws_bytes(g, precision);
    b += tc_table_bytes(g, precision);
    // transient setup buffers: sample staging (2 grids) and the precontracted arrays
    size_t T1 = g.T + 1;
    size_t nK = g.d == 3 ? T1 * T1 : T1;
    b += 2 * z.grid + 2 * nK * g.n1 * g.W1 * 8 + (size_t)g.levels * 4;
    return b;
}

// Structural nonzeros of M: the pattern is a union of product sets (one per
// Kronecker term), so count it by inclusion-exclusion over the terms, with the
// in-grid count of a product set factorising over the axes.  On one axis a term
// is a stiffness band (its own direction) or a mass band of the term's degree
// there; the offsets counted are those every term of the subset allows.
static bool band_ok(int o, int kind, int T)  // kind 1: stiffness band, 2: mass band
{
    const int a = o < 0 ? -o : o;
    if (kind == 1) return a <= T;
    return a <= T + 2 && (T > 0 || (a % 2) == 0);
}
long long structural_nnz(const Geom &g)
{
    const int nt = g.d + (g.has_b ? 1 : 0);  // terms: d stiffness terms, then the mass term
    long long total = 0;
    for (int mask = 1; mask < (1 << nt); ++mask) {
        long long prod = 1;
        for (int ax = 0; ax < g.d; ++ax) {
            long long cnt = 0;
            for (int o = -g.w; o <= g.w; ++o) {
                bool in = true;
                for (int t = 0; t < nt && in; ++t) {
                    if (!(mask & (1 << t))) continue;
                    if (t < g.d) in = band_ok(o, t == ax ? 1 : 2, g.ta[t][ax]);
                    else in = band_ok(o, 2, g.tb[ax]);
                }
                if (in) cnt += std::max(0, g.n1 - (o < 0 ? -o : o));
            }
            prod *= cnt;
        }
        total += (__builtin_popcount(mask) & 1) ? prod : -prod;
    }
    return total;
}

static int check_sizes(int d, int N, int T, int Q)
{
    if (d < 1 || d > 3 || N < 3 || T < 0 || Q < N + 1) return LSG_ERR_ARG;
    if (N > 8193 || T > 64) return LSG_ERR_ARG;
    long long n = 1;
    for (int i = 0; i < d; ++i) n *= (N - 1);
    if (n > (1ll << 31) - 1) return LSG_ERR_ARG;
    return LSG_OK;
}

// Pinned host mirrors of the PCG state, reused across contexts: cudaMallocHost and
// cudaFreeHost are slow and may synchronise the device, which would serialise the
// contexts that a server sets up and tears down while others compute.
static std::mutex g_pin_mu;
static std::vector<PcgState *> g_pin_free;

static PcgState *pinned_state()
{
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free.empty()) {
            PcgState *p = g_pin_free.back();
            g_pin_free.pop_back();
            return p;
        }
    }
    // one allocation for a slab of states, handed out one by one
    constexpr int kSlab = 64;
    PcgState *slab = nullptr;
    if (cudaMallocHost((void **)&slab, sizeof(PcgState) * kSlab) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (int i = 1; i < kSlab; ++i) g_pin_free.push_back(slab + i);
    return slab;
}

static void release_pinned_state(PcgState *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

// Frees a context's device memory in the order of stream `s` (no device-wide
// synchronisation), waits for that stream only, then returns the pinned state.
static void free_ctx(lsg_ctx *c, cudaStream_t s)
{
    if (!c) return;
    void *ptrs[] = {c->gx, c->gw, c->tab, c->Wa, c->Wb, c->Wg, c->ahat, c->bhat, c->bandS, c->bandM,
                    c->Lv, c->Uv, c->Mkeep, c->order, c->rowflag, c->prog, c->counters, c->err, c->ws, c->ws32,
                    c->r, c->z, c->p, c->wv, c->xs, c->fs, c->ys, c->red, c->st, c->r32, c->z32, c->p32, c->w32,
                    c->e32, c->e64, c->u64, c->y32, c->Wa32, c->Wb32, c->tct,
                    c->Way, c->Waz, c->Wa32y, c->Wa32z, c->ahaty, c->ahatz, c->ctab, c->clam, c->cdinv};
    const int np = (int)(sizeof ptrs / sizeof ptrs[0]);
    for (int i = 0; i < np; ++i) {
        bool dup = false;  // per-direction arrays may alias the first direction's
        for (int k = 0; k < i && !dup; ++k) dup = ptrs[k] == ptrs[i];
        if (ptrs[i] && !dup) cudaFreeAsync(ptrs[i], s);
    }
    cudaStreamSynchronize(s);
    cudaGetLastError();
    release_pinned_state(c->st_host);
    prof_destroy(c);
    if (c->graph) {
        pcg_graph_destroy(*c->graph);
        delete c->graph;
    }
    delete c;
}

// Stage an input array: device pointers pass through, host arrays are copied
// into `stage` (which must hold `count` doubles).
static int stage_in(const double *p, long long count, double *stage, const double **out, cudaStream_t s)
{
    if (is_device_ptr(p)) {
        *out = p;
        return LSG_OK;
    }
    LSG_CK(cudaMemcpyAsync(stage, p, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice, s));
    *out = stage;
    return LSG_OK;
}

template <typename V>
__global__ void k_unsplit(long long n, int S, int Sc, int SL, int SU, const V *Lv, const V *Uv, double *out)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n * S) return;
    long long r = idx / S;
    int s = (int)(idx % S);
    out[idx] = s < Sc ? (double)Lv[r * SL + s] : (double)Uv[r * SU + (s - Sc)];
}

}  // namespace lsg

using namespace lsg;

extern "C" {

int lsg_version(void) { return 100; }

const char *lsg_status_string(int st)
{
    switch (st) {
    case LSG_OK: return "ok";
    case LSG_ERR_ARG: return "invalid argument";
    case LSG_ERR_NOMEM: return "out of memory";
    case LSG_ERR_CUDA: return "CUDA error";
    case LSG_ERR_ILU_BREAKDOWN: return "ILU(0) breakdown (non-positive pivot)";
    case LSG_ERR_NOT_CONVERGED: return "PCG did not converge";
    case LSG_ERR_TIMEOUT: return "device wait budget expired";
    case LSG_ERR_NONFINITE: return "non-finite coefficient samples";
    default: return "unknown status";
    }
}

const char *lsg_last_error(void) { return g_last_error; }

long long lsg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int lsg_gauss(int Q, double *x, double *w)
{
    if (Q < 1 || !x || !w) return LSG_ERR_ARG;
    double *dx = nullptr, *dw = nullptr;
    LSG_CK(cudaMalloc((void **)&dx, sizeof(double) * Q));
    if (cudaMalloc((void **)&dw, sizeof(double) * Q) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dx);
        return LSG_ERR_NOMEM;
    }
    int st = gauss_rule(Q, dx, dw, 0);
    if (st == LSG_OK) {
        cudaError_t e1 = cudaMemcpy(x, dx, sizeof(double) * Q, cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaMemcpy(w, dw, sizeof(double) * Q, cudaMemcpyDeviceToHost);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = LSG_ERR_CUDA;
    }
    cudaFree(dx);
    cudaFree(dw);
    return st;
}

size_t lsg_footprint_bytes(int d, int N, int T, int Q, int precision)
{
    if (Q <= 0) Q = N + 2;
    if (check_sizes(d, N, T, Q) != LSG_OK) return 0;
    return footprint(make_geom(d, N, T, Q), precision, 0);
}

// Setup for one diffusion coefficient per direction (a[j] multiplies the j-th
// gradient term; a[j] == a[0] for the scalar coefficient) with truncation degrees
// per coefficient and direction.
static int setup_impl(lsg_ctx **out, int d, int N, const int ta[3][3], const int tb[3], int Q,
                      const double *const *a, const double *b, int precision, unsigned flags, cudaStream_t s)
{
    if (!out || !b) return LSG_ERR_ARG;
    *out = nullptr;
    if (d < 1 || d > 3) return LSG_ERR_ARG;
    for (int j = 0; j < d; ++j) {
        if (!a[j]) return LSG_ERR_ARG;
        if (tb[j] < 0 || tb[j] > 64) return LSG_ERR_ARG;
        for (int i = 0; i < d; ++i)
            if (ta[j][i] < 0 || ta[j][i] > 64) return LSG_ERR_ARG;
    }
    if (Q <= 0) Q = N + 2;
    const Geom g0 = make_geom_dir(d, N, ta, tb, Q);
    LSG_TRY(check_sizes(d, N, g0.T, Q));
    if (g0.w > 66) return LSG_ERR_ARG;
    if (precision < LSG_FP64 || precision > LSG_MIXED_BF16) return LSG_ERR_ARG;
    if ((flags & LSG_SETUP_CONST_PRECOND) && precision != LSG_FP64) return LSG_ERR_ARG;
    lsg_ctx *c = new lsg_ctx{};
    c->precond = (flags & LSG_SETUP_CONST_PRECOND) ? 1 : 0;
    c->stream = s;
    c->g = g0;
    c->precision = precision;
    c->flags = flags;
    c->wait_budget = kSpinBudgetCycles;
    for (int i = 0; i < 3; ++i) c->xf_fwd[i] = c->xf_bwd[i] = -1;
    if (flags & LSG_SETUP_PROFILE) prof_create(c);
    LSG_CK(cudaGetDevice(&c->device));
    {
        // keep freed context memory in the stream-ordered pool for the next setup
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
            unsigned long long thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    const Geom &g = c->g;
    Sizes z = sizes_for(g, precision, flags);
    int st = LSG_OK;
#define ALLOC(ptr, bytes)                                                      \
    do {                                                                       \
        if (st == LSG_OK) st = dalloc(c, (void **)&(ptr), (bytes), s);         \
    } while (0)
    ALLOC(c->gx, sizeof(double) * Q);
    ALLOC(c->gw, sizeof(double) * Q);
    ALLOC(c->tab, z.tab);
    ALLOC(c->Wa, z.grid);
    ALLOC(c->Wb, z.grid);
    ALLOC(c->Wg, z.grid);
    ALLOC(c->ahat, z.series);
    ALLOC(c->bhat, z.series);
    // the other directions' coefficients: separate arrays only where the samples (or,
    // for the series, the degrees) differ from a direction already held
    auto same_deg = [&](int j, int k) {
        for (int i = 0; i < 3; ++i)
            if (g.ta[j][i] != g.ta[k][i]) return false;
        return true;
    };
    c->Way = c->Waz = c->Wa;
    c->ahaty = c->ahatz = c->ahat;
    if (d >= 2) {
        c->own_ay = a[1] != a[0];
        if (c->own_ay) ALLOC(c->Way, z.grid);
        if (!(a[1] == a[0] && same_deg(1, 0))) ALLOC(c->ahaty, z.series);
    }
    if (d == 3) {
        if (a[2] == a[0]) c->Waz = c->Wa;
        else if (a[2] == a[1]) c->Waz = c->Way;
        else {
            c->own_az = 1;
            ALLOC(c->Waz, z.grid);
        }
        if (a[2] == a[0] && same_deg(2, 0)) c->ahatz = c->ahat;
        else if (a[2] == a[1] && same_deg(2, 1)) c->ahatz = c->ahaty;
        else ALLOC(c->ahatz, z.series);
    }
    ALLOC(c->bandS, z.band);
    ALLOC(c->bandM, z.band);
    ALLOC(c->Lv, z.Lv);
    ALLOC(c->Uv, z.Uv);
    if (c->precond == 1) {
        ALLOC(c->ctab, sizeof(double) * 4 * (size_t)g.KP * g.KP);
        ALLOC(c->clam, sizeof(double) * (size_t)g.n1);
        ALLOC(c->cdinv, sizeof(double) * (size_t)g.n);
    }
    if (z.Mkeep) ALLOC(c->Mkeep, z.Mkeep);
    ALLOC(c->order, sizeof(int) * (size_t)g.n);
    ALLOC(c->rowflag, sizeof(unsigned) * (size_t)g.n);
    ALLOC(c->prog, 2 * z.lines);
    ALLOC(c->counters, sizeof(unsigned) * 16);
    ALLOC(c->err, sizeof(int) * 4);
    ALLOC(c->ws, z.ws);
    ALLOC(c->r, z.vec);
    ALLOC(c->z, z.vec);
    ALLOC(c->p, z.vec);
    ALLOC(c->wv, z.vec);
    ALLOC(c->xs, z.vec);
    ALLOC(c->fs, std::max(z.vec, z.grid));
    ALLOC(c->ys, z.vec);
    ALLOC(c->red, sizeof(double) * 2 * kRedBlocks);
    ALLOC(c->st, sizeof(PcgState));
    if (precision != LSG_FP64) {
        ALLOC(c->r32, (size_t)g.n * 4);
        ALLOC(c->z32, (size_t)g.n * 4);
        ALLOC(c->p32, (size_t)g.n * 4);
        ALLOC(c->w32, (size_t)g.n * 4);
        ALLOC(c->e32, (size_t)g.n * 4);
        ALLOC(c->y32, (size_t)g.n * 4);
        ALLOC(c->Wa32, (size_t)g.nq * 4);
        ALLOC(c->Wb32, (size_t)g.nq * 4);
        c->Wa32y = c->Wa32z = c->Wa32;
        if (c->own_ay) ALLOC(c->Wa32y, (size_t)g.nq * 4);
        if (c->own_az) ALLOC(c->Wa32z, (size_t)g.nq * 4);
        else if (d == 3 && c->Waz == c->Way) c->Wa32z = c->Wa32y;
        ALLOC(c->e64, z.vec);
        ALLOC(c->u64, z.vec);
        ALLOC(c->ws32, tc_ws_bytes(g, precision));
        // padding slots of the split fields are never written: they must read as zero
        if (st == LSG_OK && cudaMemsetAsync(c->ws32, 0, tc_ws_bytes(g, precision), s) != cudaSuccess) {
            record_cuda_error(cudaGetLastError(), "clearing the split-field workspace", __FILE__, __LINE__);
            st = LSG_ERR_CUDA;
        }
        ALLOC(c->tct, tc_table_bytes(g, precision));
    }
    // host samples are staged in temporary device arrays (one per distinct array)
    double *stage[4] = {nullptr, nullptr, nullptr, nullptr};
    const double *dev_in[4] = {a[0], d >= 2 ? a[1] : a[0], d == 3 ? a[2] : a[0], b};
    const double *host_in[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k) {
        if (is_device_ptr(dev_in[k])) continue;
        int same = -1;
        for (int m = 0; m < k && same < 0; ++m)
            if (host_in[m] == dev_in[k]) same = m;
        host_in[k] = dev_in[k];
        if (same >= 0) {
            stage[k] = nullptr;
            dev_in[k] = stage[same];
            continue;
        }
        ALLOC(stage[k], z.grid);
        dev_in[k] = stage[k];
    }
#undef ALLOC
    if (st == LSG_OK && !(c->st_host = pinned_state())) st = LSG_ERR_NOMEM;
    auto release_stage = [&]() {
        for (int k = 0; k < 4; ++k)
            if (stage[k]) cudaFreeAsync(stage[k], s);
        for (int k = 0; k < 4; ++k) stage[k] = nullptr;
    };
    if (st != LSG_OK) {
        release_stage();
        free_ctx(c, s);
        return st;
    }
    auto fail = [&](int code) {
        release_stage();
        free_ctx(c, s);
        return code;
    };
    for (int k = 0; k < 4; ++k)
        if (stage[k] && cudaMemcpyAsync(stage[k], host_in[k], z.grid, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(LSG_ERR_CUDA);
    const double *da[3] = {dev_in[0], dev_in[1], dev_in[2]}, *db = dev_in[3];
    if (cudaMemsetAsync(c->err, 0, sizeof(int) * 4, s) != cudaSuccess) return fail(LSG_ERR_CUDA);
    st = build_tables(c, da, db, s);
    if (st != LSG_OK) return fail(st);
    if (!tile_table_lookup(c) && (flags & LSG_SETUP_AUTOTUNE)) {
        st = autotune_transforms(c, 5, s);
        if (st != LSG_OK) return fail(st);
    }
    st = build_tc_tables(c, s);
    if (st != LSG_OK) return fail(st);
    int derr = read_dev_error(c, s);
    if (derr != LSG_OK) return fail(derr);
    st = c->precond == 1 ? build_const_preconditioner(c, s) : build_preconditioner(c, s);
    if (st != LSG_OK) return fail(st);
    release_stage();
    derr = read_dev_error(c, s);
    if (derr == LSG_ERR_TIMEOUT || derr == LSG_ERR_CUDA) return fail(derr);
    c->setup_status = derr;
    *out = c;
    return derr;  // LSG_OK or LSG_ERR_ILU_BREAKDOWN (context kept for inspection)
}

int lsg_setup_ex(lsg_ctx **out, int d, int N, int T, int Q, const double *a, const double *b, int precision,
                 unsigned flags, lsg_stream_t stream)
{
    if (!a || T < 0 || T > 64) return LSG_ERR_ARG;
    int ta[3][3], tb[3];
    for (int j = 0; j < 3; ++j) {
        tb[j] = T;
        for (int i = 0; i < 3; ++i) ta[j][i] = T;
    }
    const double *ad[3] = {a, a, a};
    return setup_impl(out, d, N, ta, tb, Q, ad, b, precision, flags, (cudaStream_t)stream);
}

int lsg_setup_problem(lsg_ctx **out, const lsg_problem *p, lsg_stream_t stream)
{
    if (!p || p->d < 1 || p->d > 3) return LSG_ERR_ARG;
    int ta[3][3], tb[3];
    const double *ad[3];
    for (int j = 0; j < 3; ++j) {
        tb[j] = p->tb[j];
        ad[j] = (j < p->d && p->a[j]) ? p->a[j] : p->a[0];
        for (int i = 0; i < 3; ++i) ta[j][i] = p->ta[j][i];
    }
    return setup_impl(out, p->d, p->N, ta, tb, p->Q, ad, p->b, p->precision, p->flags, (cudaStream_t)stream);
}

int lsg_setup(lsg_ctx **out, int d, int N, int T, int Q, const double *a, const double *b, int precision,
              lsg_stream_t stream)
{
    return lsg_setup_ex(out, d, N, T, Q, a, b, precision, 0u, stream);
}

int lsg_destroy(lsg_ctx *c)
{
    if (!c) return LSG_ERR_ARG;
    free_ctx(c, c->stream);
    return LSG_OK;
}

int lsg_load_vector(lsg_ctx *c, const double *f, double *F, lsg_stream_t stream)
{
    if (!c || !f || !F) return LSG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *df;
    c->stream = s;  // lsg_destroy orders the release after the last call's stream
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(stage_in(f, c->g.nq, c->fs, &df, s));
    bool hF = !is_device_ptr(F);
    double *dF = hF ? c->ys : F;
    LSG_TRY(load_vector(c, df, dF, s));
    if (hF) {
        LSG_CK(cudaMemcpyAsync(F, dF, sizeof(double) * (size_t)c->g.n, cudaMemcpyDeviceToHost, s));
        LSG_CK(cudaStreamSynchronize(s));
    }
    return LSG_OK;
}

int lsg_apply_A_lowp(lsg_ctx *c, const float *x, float *y, lsg_stream_t stream)
{
    if (!c || !x || !y || x == y || c->precision == LSG_FP64) return LSG_ERR_ARG;
    if (!is_device_ptr(x) || !is_device_ptr(y)) return LSG_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    LSG_TRY(clear_dev_error(c, (cudaStream_t)stream));
    LSG_TRY(apply_K_tc(c, x, y, nullptr, (cudaStream_t)stream));
    return read_dev_error(c, (cudaStream_t)stream);
}

int lsg_apply_A(lsg_ctx *c, const double *x, double *y, lsg_stream_t stream)
{
    if (!c || !x || !y || x == y) return LSG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *dx;
    c->stream = s;  // lsg_destroy orders the release after the last call's stream
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(stage_in(x, c->g.n, c->xs, &dx, s));
    bool hy = !is_device_ptr(y);
    double *dy = hy ? c->ys : y;
    LSG_TRY(apply_K(c, dx, dy, nullptr, s));
    if (hy) {
        LSG_CK(cudaMemcpyAsync(y, dy, sizeof(double) * (size_t)c->g.n, cudaMemcpyDeviceToHost, s));
        LSG_CK(cudaStreamSynchronize(s));
    }
    return LSG_OK;
}

int lsg_apply_Minv(lsg_ctx *c, const double *r, double *z, lsg_stream_t stream)
{
    if (!c || !r || !z || r == z) return LSG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *dr;
    c->stream = s;  // lsg_destroy orders the release after the last call's stream
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(stage_in(r, c->g.n, c->xs, &dr, s));
    bool hz = !is_device_ptr(z);
    double *dz = hz ? c->wv : z;
    LSG_TRY(apply_Minv(c, dr, dz, nullptr, s));
    if (hz) {
        LSG_CK(cudaMemcpyAsync(z, dz, sizeof(double) * (size_t)c->g.n, cudaMemcpyDeviceToHost, s));
        LSG_CK(cudaStreamSynchronize(s));
        return read_dev_error(c, s);
    }
    return LSG_OK;
}

int lsg_pcg_solve(lsg_ctx *c, const double *F, double *u, double rtol, int kmax, lsg_info *info,
                  lsg_stream_t stream)
{
    if (!c || !F || !u || !(rtol >= 0.0) || kmax < 0) return LSG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *dF;
    c->stream = s;  // lsg_destroy orders the release after the last call's stream
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(stage_in(F, c->g.n, c->fs, &dF, s));
    bool hu = !is_device_ptr(u);
    double *du = u;
    if (hu) {
        du = c->xs;
        LSG_CK(cudaMemcpyAsync(du, u, sizeof(double) * (size_t)c->g.n, cudaMemcpyHostToDevice, s));
    }
    prof_reset(c);
    int st = (c->precision == LSG_FP64) ? pcg_fp64(c, dF, du, rtol, kmax, info, s)
                                        : pcg_mixed(c, dF, du, rtol, kmax, info, s);
    if (st == LSG_OK || st == LSG_ERR_NOT_CONVERGED) {
        int pst = prof_collect(c);
        if (pst != LSG_OK) st = pst;
    }
    if (hu) {
        LSG_CK(cudaMemcpyAsync(u, du, sizeof(double) * (size_t)c->g.n, cudaMemcpyDeviceToHost, s));
        LSG_CK(cudaStreamSynchronize(s));
    }
    return st;
}

int lsg_eval(lsg_ctx *c, const double *u, double *vals, lsg_stream_t stream)
{
    if (!c || !u || !vals) return LSG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *du;
    c->stream = s;  // lsg_destroy orders the release after the last call's stream
    LSG_TRY(clear_dev_error(c, s));
    LSG_TRY(stage_in(u, c->g.n, c->xs, &du, s));
    bool hv = !is_device_ptr(vals);
    double *dv = hv ? c->fs : vals;
    LSG_TRY(eval_grid(c, du, dv, s));
    if (hv) {
        LSG_CK(cudaMemcpyAsync(vals, dv, sizeof(double) * (size_t)c->g.nq, cudaMemcpyDeviceToHost, s));
        LSG_CK(cudaStreamSynchronize(s));
    }
    return LSG_OK;
}

long long lsg_export_count(lsg_ctx *c, int item)
{
    if (!c) return 0;
    const Geom &g = c->g;
    long long ns = 1;
    for (int i = 0; i < g.d; ++i) ns *= (g.T + 1);
    switch (item) {
    case LSG_EXPORT_GAUSS_X:
    case LSG_EXPORT_GAUSS_W: return g.Q;
    case LSG_EXPORT_AHAT:
    case LSG_EXPORT_AHAT_Y:
    case LSG_EXPORT_AHAT_Z:
    case LSG_EXPORT_BHAT: return ns;
    case LSG_EXPORT_BAND_S:
    case LSG_EXPORT_BAND_M: return (long long)(g.T + 1) * g.n1 * g.W1;
    case LSG_EXPORT_M: return c->Mkeep ? g.n * g.S : 0;
    case LSG_EXPORT_LU: return c->Lv ? g.n * g.S : 0;
    case LSG_EXPORT_CONST_EIG: return c->clam ? g.n1 : 0;
    default: return 0;
    }
}

int lsg_export(lsg_ctx *c, int item, double *out)
{
    if (!c || !out) return LSG_ERR_ARG;
    long long cnt = lsg_export_count(c, item);
    if (cnt <= 0) return LSG_ERR_ARG;
    const double *src = nullptr;
    switch (item) {
    case LSG_EXPORT_GAUSS_X: src = c->gx; break;
    case LSG_EXPORT_GAUSS_W: src = c->gw; break;
    case LSG_EXPORT_AHAT: src = c->ahat; break;
    case LSG_EXPORT_AHAT_Y: src = c->ahaty; break;
    case LSG_EXPORT_AHAT_Z: src = c->ahatz; break;
    case LSG_EXPORT_CONST_EIG: src = c->clam; break;
    case LSG_EXPORT_BHAT: src = c->bhat; break;
    case LSG_EXPORT_BAND_S: src = c->bandS; break;
    case LSG_EXPORT_BAND_M: src = c->bandM; break;
    case LSG_EXPORT_M: src = c->Mkeep; break;
    default: break;
    }
    LSG_CK(cudaDeviceSynchronize());
    if (item == LSG_EXPORT_LU) {
        double *tmp = nullptr;
        LSG_CK(cudaMalloc((void **)&tmp, sizeof(double) * (size_t)cnt));
        const Geom &g = c->g;
        unsigned blocks = (unsigned)((cnt + 255) / 256);
        if (c->precision == LSG_FP64)
            k_unsplit<double><<<blocks, 256>>>(g.n, g.S, g.Sc, g.SL, g.SU, (const double *)c->Lv, (const double *)c->Uv, tmp);
        else
            k_unsplit<float><<<blocks, 256>>>(g.n, g.S, g.Sc, g.SL, g.SU, (const float *)c->Lv, (const float *)c->Uv, tmp);
        cudaError_t e = cudaMemcpy(out, tmp, sizeof(double) * (size_t)cnt, cudaMemcpyDeviceToHost);
        cudaFree(tmp);
        LSG_CK(e);
        return LSG_OK;
    }
    LSG_CK(cudaMemcpy(out, src, sizeof(double) * (size_t)cnt, cudaMemcpyDeviceToHost));
    return LSG_OK;
}

long long lsg_query(lsg_ctx *c, int item)
{
    if (!c) return -1;
    const Geom &g = c->g;
    switch (item) {
    case LSG_Q_UNKNOWNS: return g.n;
    case LSG_Q_GRID: return g.nq;
    case LSG_Q_HALF_WIDTH: return g.w;
    case LSG_Q_SLOTS: return g.S;
    case LSG_Q_LEVELS: return g.levels;
    case LSG_Q_DEVICE_BYTES: return (long long)c->bytes;
    case LSG_Q_NNZ: return structural_nnz(g);
    case LSG_Q_PRECISION: return c->precision;
    case LSG_Q_ASSEMBLE_US: return (long long)(c->t_assemble_ms * 1000.0f);
    case LSG_Q_ILU_US: return (long long)(c->t_ilu_ms * 1000.0f);
    case LSG_Q_SWEEP_L_US: return prof_query(c, PROF_SWEEP_L, false);
    case LSG_Q_SWEEP_L_CALLS: return prof_query(c, PROF_SWEEP_L, true);
    case LSG_Q_SWEEP_U_US: return prof_query(c, PROF_SWEEP_U, false);
    case LSG_Q_SWEEP_U_CALLS: return prof_query(c, PROF_SWEEP_U, true);
    case LSG_Q_KX_US: return prof_query(c, PROF_KX, false);
    case LSG_Q_KX_CALLS: return prof_query(c, PROF_KX, true);
    case LSG_Q_KX_LO_US: return prof_query(c, PROF_KX_LO, false);
    case LSG_Q_KX_LO_CALLS: return prof_query(c, PROF_KX_LO, true);
    case LSG_Q_CONST_US: return prof_query(c, PROF_CONST, false);
    case LSG_Q_CONST_CALLS: return prof_query(c, PROF_CONST, true);
    case LSG_Q_PRECOND_KIND: return c->precond;
    default: return -1;
    }
}

int lsg_autotune_transforms(lsg_ctx *c, int reps, int *choice)
{
    if (!c) return LSG_ERR_ARG;
    LSG_TRY(autotune_transforms(c, reps, c->stream));
    if (c->graph) c->graph->reset();  // a captured solve holds the old launches
    if (choice)
        for (int i = 0; i < 3; ++i) choice[i] = c->xf_fwd[i], choice[3 + i] = c->xf_bwd[i];
    return LSG_OK;
}

int lsg_transform_tiles(lsg_ctx *c, int *choice)
{
    if (!c || !choice) return LSG_ERR_ARG;
    for (int i = 0; i < 3; ++i) choice[i] = c->xf_fwd[i], choice[3 + i] = c->xf_bwd[i];
    return LSG_OK;
}

int lsg_set_transform_tiles(lsg_ctx *c, const int *choice)
{
    if (!c || !choice) return LSG_ERR_ARG;
    for (int i = 0; i < 6; ++i)
        if (choice[i] < -1 || choice[i] > 4) return LSG_ERR_ARG;
    for (int i = 0; i < 3; ++i) c->xf_fwd[i] = (signed char)choice[i], c->xf_bwd[i] = (signed char)choice[3 + i];
    if (c->graph) c->graph->reset();  // a captured solve holds the old launches
    return LSG_OK;
}

int lsg_set_wait_budget(lsg_ctx *c, long long cycles)
{
    if (!c || cycles < 0) return LSG_ERR_ARG;
    c->wait_budget = cycles == 0 ? kSpinBudgetCycles : cycles;
    return LSG_OK;
}

}  // extern "C"
