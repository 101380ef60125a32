// lsg_internal.cuh -- context layout, geometry and small device helpers shared by
// the CUDA sources of the solver library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lsg.h"

namespace lsg {

// ---------------------------------------------------------------------------
// error handling
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define LSG_CK(call)                                                          \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            ::lsg::record_cuda_error(e_, #call, __FILE__, __LINE__);          \
            return LSG_ERR_CUDA;                                              \
        }                                                                     \
    } while (0)

#define LSG_TRY(expr)                                                         \
    do {                                                                      \
        int s_ = (expr);                                                      \
        if (s_ != LSG_OK) return s_;                                          \
    } while (0)

// device error word values (first error wins)
enum DevErr : int { DERR_NONE = 0, DERR_BREAKDOWN = 1, DERR_TIMEOUT = 2, DERR_NONFINITE = 3 };

// wait budget of every device-side spin, in SM clock cycles (clock64 is local to
// the SM and cheap to read; ~4 s at 2 GHz)
constexpr long long kSpinBudgetCycles = 8000000000ll;

// ---------------------------------------------------------------------------
// geometry of one problem
struct Geom {
    int d, N, n1, Q, Qh, T, w, W1;
    int S, Sc;            // stencil slots (2w+1)^d and the centre slot
    int SL, SU;           // padded row lengths of the strictly-lower / diag+upper stencil halves
    int ne, no;           // even / odd basis counts ceil(n1/2), floor(n1/2)
    int KP, QhP;          // padded table dims (columns: half basis count, rows: half node count)
    long long n, nq;      // unknowns n1^d, grid points Q^d
    long long nlines;     // n1^(d-1)
    int levels;           // wavefront levels (n1-1) * sum_{a<d} (w+1)^a + 1
    int has_b;            // reaction term present (pattern includes the mass term)
    // truncation degrees: ta[j][i] of the series of a_j (the coefficient of the j-th
    // gradient term) in direction i, tb[i] of b's; T is the largest, w the half-width
    // of the offset box that holds every band of the pattern
    int ta[3][3], tb[3];
};

Geom make_geom(int d, int N, int T, int Q);
Geom make_geom_dir(int d, int N, const int ta[3][3], const int tb[3], int Q);

// pinned + device scalars of one PCG run (device-resident Algorithm 1 state)
struct PcgState {
    double rho, rho_old, alpha, beta, pw, rr, nF2, eps2, tr;  // tr: true residual^2 scratch
    int k, kmax, done, status;
    int pad[4];
};

// A PCG solve (or several, one branch each) captured as one CUDA graph with the
// iteration loop in a conditional WHILE node (pcg.cu).
struct PcgGraph {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr, body = nullptr;  // capture streams
    std::vector<cudaStream_t> branch;            // one per solve (several solves)
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<long long> body_launches;        // kernels per loop pass of each solve
    long long fixed_launches = 0;                // kernels outside the loops
    int nctx = 0;
    const double *F0 = nullptr;                  // single solve: the vectors it was captured on
    double *x0 = nullptr;
    void reset();
};

// stages timed by the optional per-context profiler (LSG_SETUP_PROFILE)
enum ProfStage : int { PROF_SWEEP_L = 0, PROF_SWEEP_U = 1, PROF_KX = 2, PROF_KX_LO = 3, PROF_CONST = 4, PROF_STAGES = 5 };
struct Prof;

// reduction scratch: fixed grid so that sums are deterministic
constexpr int kRedBlocks = 296;   // 2 x 148..152 SMs, fixed for determinism
constexpr int kRedThreads = 256;

}  // namespace lsg

struct lsg_ctx {
    lsg::Geom g;
    int precision;
    int device;
    unsigned flags;
    size_t bytes;

    // Gauss rule and folded transform tables (FP64)
    double *gx, *gw;           // Q nodes / weights
    double *tab;               // 4 blocks of QhP*KP: phiE, phiO, dphiE, dphiO
    double *Wa, *Wb, *Wg;      // w(x)w(y)w(z) * a, * b, and the weights alone (Q^d)
    double *Way, *Waz;         // W * a_y, W * a_z (aliases of Wa for one diffusion coefficient)
    float *Wa32, *Wb32;        // FP32 copies (mixed)
    float *Wa32y, *Wa32z;
    int own_ay, own_az;        // Way / Waz (and their FP32 copies, series) are separate arrays
    void *tct;                 // mixed: unfolded TF32/BF16 tables for the tensor-core contractions
    int tcMpF, tcKpF, tcMpB, tcKpB;  // their padded shapes (forward [MpF][KpF], backward [MpB][KpB])
    double *ahat, *bhat;       // (T+1)^d, zero beyond each direction's degree
    double *ahaty, *ahatz;     // series of a_y, a_z (aliases of ahat for one coefficient and degree)
    double *bandS, *bandM;     // (T+1) x n1 x W1

    // ILU(0) factors in split stencil storage: Lv [n][SL] strictly lower slots,
    // Uv [n][SU] diagonal then strictly upper slots (double, or float when mixed)
    void *Lv, *Uv;
    double *Mkeep;             // optional copy of M ([n][S])
    int *order;                // rows in wavefront-level order
    unsigned *rowflag;         // ILU row completion flags
    unsigned *prog;            // sweep progress per line (2 x nlines: forward, backward)
    unsigned *counters;        // claim counters (ILU, sweep L, sweep U, reductions)
    int *err;                  // device error word

    // matrix-free product workspace
    double *ws;
    size_t ws_elems;
    float *ws32;            // mixed contexts: the split fields of the tensor-core product (tc_ws_bytes)

    // PCG vectors and reductions
    double *r, *z, *p, *wv, *xs, *fs, *ys;   // xs/fs/ys: staging for host arguments
    double *red;               // kRedBlocks partials
    lsg::PcgState *st;         // device state
    lsg::PcgState *st_host;    // pinned mirror
    // mixed precision inner vectors
    float *r32, *z32, *p32, *w32, *e32, *y32;
    double *e64, *u64;

    // budget (SM clock cycles) of the triangular sweeps' dependency waits (lsg_set_wait_budget)
    long long wait_budget;
    cudaStream_t stream;       // stream of the last call (setup or compute): lsg_destroy frees on it
    int setup_status;          // LSG_OK, or LSG_ERR_ILU_BREAKDOWN (kept in the device error word)

    // setup stage times (milliseconds, CUDA events): tables, assembly, ILU(0)
    float t_tables_ms, t_assemble_ms, t_ilu_ms;
    lsg::Prof *prof;           // solve-stage event timing (null unless LSG_SETUP_PROFILE)
    signed char xf_fwd[3], xf_bwd[3];  // tile variant of each FP64 contraction of K x (-1: default)
    // constant-coefficient preconditioner of PCG-I (LSG_SETUP_CONST_PRECOND) instead of ILU(0)
    int precond;               // 0: ILU(0) of M, 1: M_0 solved by fast diagonalisation
    double *ctab;              // parity blocks of E^T (2 x KP^2) then of E (2 x KP^2)
    double *clam;              // generalised eigenvalues, n1 (index 2k + parity)
    double *cdinv;             // 1 / D, n
    lsg::PcgGraph *graph;      // the captured FP64 solve (pcg_fp64), built on first use
    int no_graph;              // capture failed once: solves use the host-driven loop
};

namespace lsg {

// allocation helpers (device memory accounted in ctx->bytes)
int dalloc(lsg_ctx *c, void **p, size_t bytes, cudaStream_t s);
bool is_device_ptr(const void *p);

// kernels / drivers implemented in the .cu files
int build_tables(lsg_ctx *c, const double *const *a_dev, const double *b_dev, cudaStream_t s);
int build_preconditioner(lsg_ctx *c, cudaStream_t s);
int apply_K(lsg_ctx *c, const double *x, double *y, const int *done, cudaStream_t s);
int apply_K_tc(lsg_ctx *c, const float *x, float *y, const int *done, cudaStream_t s);
int build_tc_tables(lsg_ctx *c, cudaStream_t s);
size_t tc_table_bytes(const Geom &g, int precision);
// the mixed form's split-field workspace (cleared once at set-up)
size_t tc_ws_bytes(const Geom &g, int precision);
int load_vector(lsg_ctx *c, const double *f, double *F, cudaStream_t s);
int eval_grid(lsg_ctx *c, const double *u, double *vals, cudaStream_t s);
int apply_Minv(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s);
int build_const_preconditioner(lsg_ctx *c, cudaStream_t s);
int apply_const_precond(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s);
int apply_Minv32(lsg_ctx *c, const float *r, float *z, const int *done, cudaStream_t s);
int pcg_fp64(lsg_ctx *c, const double *F, double *u, double rtol, int kmax, lsg_info *info,
             cudaStream_t s);

// How many iterations to queue before the host looks at the device state again:
// from the residual decrease observed so far, just enough to reach the stop test,
// so that few iterations are launched after convergence (they would return at once).
struct ChunkPlan {
    double rr0 = 0.0, rr_prev = 0.0;
    int k_prev = 0;
};
int next_chunk(ChunkPlan &P, int k, double rr, double target, int cap);

// non-blocking PCG run (Algorithm 1) used by the batched and serving forms
struct PcgRun {
    lsg_ctx *c;
    const double *F;
    double *x;
    int kmax, launched, chunk, phase, status;
    int tag0;                  // profiler tag of the run's first iteration
    ChunkPlan plan;
    cudaEvent_t ev;
};
int pcg_start(PcgRun &R, lsg_ctx *c, const double *F, double *x, double rtol, int kmax, cudaStream_t s);
int pcg_poll(PcgRun &R, cudaStream_t s, bool wait, bool *finished);
void pcg_info(const PcgRun &R, lsg_info *info);
void pcg_release(PcgRun &R);
int pcg_mixed(lsg_ctx *c, const double *F, double *u, double rtol, int kmax, lsg_info *info,
              cudaStream_t s);
int pcg_graph_build(PcgGraph &G, int count, lsg_ctx *const *ctxs, const double *const *F, double *const *x);
int pcg_graph_run(PcgGraph &G, lsg_ctx *const *ctxs, double rtol, int kmax, cudaStream_t s, lsg_info *infos,
                  int *status);
void pcg_graph_destroy(PcgGraph &G);
int read_dev_error(lsg_ctx *c, cudaStream_t s);
int clear_dev_error(lsg_ctx *c, cudaStream_t s);
int check_finite(lsg_ctx *c, const double *v, long long n, cudaStream_t s);
size_t workspace_elems(const Geom &g);
bool tile_table_lookup(lsg_ctx *c);
int autotune_transforms(lsg_ctx *c, int reps, cudaStream_t s);
int gauss_rule(int Q, double *x, double *w, cudaStream_t s);
long long structural_nnz(const Geom &g);

// host-side count of kernel launches issued by the library (all contexts)
void count_launch();
void count_launches(long long k);  // adjusts the count (kernels run inside CUDA graphs)
long long launches_so_far();

// optional stage timing (no-ops when the context was set up without LSG_SETUP_PROFILE)
void prof_create(lsg_ctx *c);
void prof_destroy(lsg_ctx *c);
void prof_reset(lsg_ctx *c);
int prof_begin(lsg_ctx *c, int stage, cudaStream_t s, int *slot);
int prof_end(lsg_ctx *c, int slot, cudaStream_t s);
int prof_collect(lsg_ctx *c);
// iteration tags: records made while tag q is set count only once prof_mark_done
// has marked q as an iteration that did its work (kernels of iterations queued
// after the stop test return at once and are not timed)
int prof_tag(lsg_ctx *c);
void prof_set_tag(lsg_ctx *c, int tag);
void prof_mark_done(lsg_ctx *c, int first_tag, int count);
long long prof_query(const lsg_ctx *c, int stage, bool calls);

// ---------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lsg
