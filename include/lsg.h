/*
 * lsg.h -- C ABI of the GB300 (sm_103a) preconditioned Legendre-Galerkin solver.
 *
 * Problem (Diao, Hu & Ma, arXiv 2004.13961, Sec. 3, `NSproblem`):
 *     -div(a(x) grad u) + b(x) u = f  on (-1,1)^d,  u = 0 on the boundary, d = 1, 2, 3,
 * with a = beta (diffusion) and b = alpha (reaction) in the paper's notation.
 * Galerkin basis phi_k = L_k - L_{k+2}, k = 0..N-2, tensor products in 2D/3D
 * (Sec. 3); the discrete system is K u_hat = F with K = A + B
 * (Sec. 3, `algebraicsystem`), where A and B are applied matrix-free by
 * Legendre-Gauss quadrature (Sec. 4.3, "fast matrix-vector multiplications").
 * The preconditioner M replaces a and b by their Legendre series truncated to
 * degree T in each direction (Sec. 4.1, `1DM`, `2DM`, `3DM`) and is applied
 * through its ILU(0) factors (Sec. 4.2, Algorithms 2-4) inside PCG
 * (Sec. 4, Algorithm 1).
 *
 * Layout contract (Sec. 3, unknown ordering):
 *   - coefficient vectors (u_hat, F, x, y, r, z) hold n = (N-1)^d FP64 values,
 *     first index fastest: u_hat[k + (N-1) j + (N-1)^2 l] multiplies
 *     phi_k(x) phi_j(y) phi_l(z);
 *   - grid arrays (samples of a, b, f; lsg_eval output) hold Q^d FP64 values at
 *     the tensor Legendre-Gauss grid, nodes ascending (lsg_gauss), x fastest.
 *
 * Pointers: every array argument may be a host pointer or a device pointer of
 * the current CUDA device (detected with cudaPointerGetAttributes); host
 * arrays are staged through context-owned device buffers.  The caller owns
 * every array it passes; the library never keeps a pointer to one after the
 * call returns.  A context owns all device memory it allocates.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 * are stream-ordered; only lsg_setup, lsg_pcg_solve, lsg_export and the batch
 * and server calls synchronise.  A context is not thread-safe: serialise calls
 * that use the same context.
 *
 * Errors: every call returns an lsg_status (0 = OK, < 0 = error); no call
 * aborts or traps.  Device-side failures (ILU breakdown, an expired wait
 * budget) are reported through a device error word read back by the
 * synchronising calls.
 */
#ifndef LSG_H
#define LSG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsg_ctx lsg_ctx;
typedef struct lsg_server lsg_server;
typedef void *lsg_stream_t; /* cudaStream_t */

enum lsg_status {
    LSG_OK = 0,
    LSG_ERR_ARG = -1,             /* invalid argument (sizes, null pointer, aliasing) */
    LSG_ERR_NOMEM = -2,           /* a device or host allocation failed / over budget */
    LSG_ERR_CUDA = -3,            /* a CUDA runtime error (see lsg_last_error) */
    LSG_ERR_ILU_BREAKDOWN = -4,   /* ILU(0) pivot U_ii <= 1e-14 |M_ii| (Alg. 2 "assuming they exist") */
    LSG_ERR_NOT_CONVERGED = -5,   /* k_max reached, or p^T w <= 0 in Algorithm 1 */
    LSG_ERR_TIMEOUT = -6,         /* a device-side dependency wait exceeded its budget */
    LSG_ERR_NONFINITE = -7        /* NaN or Inf in the coefficient samples */
};

enum lsg_precision {
    LSG_FP64 = 0,        /* every stage in FP64 */
    LSG_MIXED_TF32 = 1,  /* inner PCG: TF32 tensor-core transforms, FP32 ILU; FP64 refinement */
    LSG_MIXED_BF16 = 2   /* inner PCG: BF16 tensor-core transforms, FP32 ILU; FP64 refinement */
};

/* lsg_setup_ex flags */
#define LSG_SETUP_KEEP_M 1u /* keep an unfactored copy of M for lsg_export(LSG_EXPORT_M) */
#define LSG_SETUP_PROFILE 2u /* time every triangular-sweep kernel and every K x product that
                                lsg_pcg_solve launches, with CUDA events recorded on the solve's
                                stream (no extra synchronisation); read with the LSG_Q_SWEEP_* and
                                LSG_Q_KX_* queries after the solve returns */
#define LSG_SETUP_CONST_PRECOND 8u /* PCG-I, the paper's comparison method (Sec. 5): precondition with
                                      M_0, the operator with every coefficient replaced by the constant
                                      term of its Legendre series (all truncation degrees 0), solved
                                      directly in each iteration by fast diagonalisation (generalised
                                      eigenvectors of the 1D mass and stiffness matrices, computed on the
                                      device) instead of ILU(0) of M; FP64 contexts only */
#define LSG_SETUP_AUTOTUNE 4u /* when the committed tile table has no entry for (d, N, Q), time the
                                 tile variants of the FP64 contractions of K x at setup and keep
                                 the fastest (lsg_autotune_transforms) */
#define LSG_SETUP_SHARED_GPU 16u /* the context is set up while other work runs on the same GPU
                                    (many problems at once, as the batched and served forms): the
                                    ILU(0) factorisation of a 2D M runs on a grid sized by its
                                    wavefront instead of one that fills the GPU, so that several
                                    factorisations overlap; the factors are the same (bitwise) */

/* lsg_export items (host output; sizes from lsg_export_count) */
enum lsg_export_item {
    LSG_EXPORT_GAUSS_X = 0,   /* Q nodes, ascending */
    LSG_EXPORT_GAUSS_W = 1,   /* Q weights */
    LSG_EXPORT_AHAT = 2,      /* (T+1)^d truncated Legendre coefficients of a, x degree fastest */
    LSG_EXPORT_BHAT = 3,      /* (T+1)^d truncated Legendre coefficients of b */
    LSG_EXPORT_BAND_S = 4,    /* (T+1) x (N-1) x (2w+1): S^(t)[i][i+o] = (L_t phi'_i, phi'_{i+o}), o = -w..w */
    LSG_EXPORT_BAND_M = 5,    /* (T+1) x (N-1) x (2w+1): M^(t)[i][i+o] = (L_t phi_i, phi_{i+o}) */
    LSG_EXPORT_M = 6,         /* n x S stencil of M (needs LSG_SETUP_KEEP_M) */
    LSG_EXPORT_LU = 7,        /* n x S stencil of the ILU(0) factors (L strictly lower, U upper) */
    LSG_EXPORT_AHAT_Y = 8,    /* truncated series of the y-direction diffusion coefficient (lsg_setup_problem) */
    LSG_EXPORT_AHAT_Z = 9,    /* truncated series of the z-direction diffusion coefficient */
    LSG_EXPORT_CONST_EIG = 10 /* LSG_SETUP_CONST_PRECOND: the N-1 generalised eigenvalues of the 1D
                                 mass and stiffness matrices, index 2k + parity */
};

/* lsg_query items */
enum lsg_query_item {
    LSG_Q_UNKNOWNS = 0,     /* n = (N-1)^d */
    LSG_Q_GRID = 1,         /* Q^d */
    LSG_Q_HALF_WIDTH = 2,   /* w = T + 2, stencil half-width per direction */
    LSG_Q_SLOTS = 3,        /* S = (2w+1)^d stencil slots per row, lexicographic (dx fastest) */
    LSG_Q_LEVELS = 4,       /* wavefront levels of the natural ordering */
    LSG_Q_DEVICE_BYTES = 5, /* device bytes held by the context */
    LSG_Q_NNZ = 6,          /* structural nonzeros of M */
    LSG_Q_PRECISION = 7,
    LSG_Q_ASSEMBLE_US = 8,  /* setup: M assembly and ordering time, microseconds (CUDA events) */
    LSG_Q_ILU_US = 9,       /* setup: ILU(0) factorisation time, microseconds (CUDA events) */
    /* last lsg_pcg_solve of a context set up with LSG_SETUP_PROFILE (-1 without it): summed
       kernel time in microseconds and launch count of each stage */
    LSG_Q_SWEEP_L_US = 10,    /* forward sweeps L y = r (Algorithm 3) */
    LSG_Q_SWEEP_L_CALLS = 11,
    LSG_Q_SWEEP_U_US = 12,    /* backward sweeps U z = y (Algorithm 4) */
    LSG_Q_SWEEP_U_CALLS = 13,
    LSG_Q_KX_US = 14,         /* FP64 matrix-free products inside the PCG loop */
    LSG_Q_KX_CALLS = 15,
    LSG_Q_KX_LO_US = 16,      /* low-precision products of the mixed form's inner PCG */
    LSG_Q_KX_LO_CALLS = 17,
    LSG_Q_CONST_US = 18,      /* constant-coefficient preconditioner solves (LSG_SETUP_CONST_PRECOND) */
    LSG_Q_CONST_CALLS = 19,
    LSG_Q_PRECOND_KIND = 20   /* 0: ILU(0) of M, 1: the constant-coefficient preconditioner */
};

typedef struct {
    int iters;            /* PCG loop passes k of Algorithm 1 (summed over refinements in mixed) */
    int outer_iters;      /* FP64 refinement steps (mixed precision; 0 for FP64) */
    double relres;        /* recursive sqrt(r^T r)/||F||_2 at exit (innermost) */
    double relres_true;   /* true ||F - K u||_2 / ||F||_2, computed in FP64 */
    int status;           /* lsg_status of the solve */
} lsg_info;

/* Library version (major*10000 + minor*100 + patch). */
int lsg_version(void);
/* Static string for a status code. */
const char *lsg_status_string(int status);
/* Last CUDA error text recorded by this thread (empty if none). */
const char *lsg_last_error(void);

/* Instrumentation, no counterpart in the paper: the number of CUDA kernels this
 * library has launched so far in this process (all contexts, all threads). */
long long lsg_kernel_launches(void);

/* Legendre-Gauss nodes (roots of L_Q, Sec. 2.2, ascending) and weights,
 * computed on the device by Newton iteration on the three-term recurrence
 * (Sec. 2.1).  x, w: host arrays of Q doubles.  Q >= 1. */
int lsg_gauss(int Q, double *x, double *w);

/* The same Gauss rule as lsg_gauss, for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a property of the library, not
 * of the method.  lsg_gauss allocates two device buffers on every call; code that
 * runs while the device's memory is fully reserved by another component, or
 * under a policy that forbids allocator calls once a job has started, cannot use
 * it.  This variant keeps that scratch in a fixed device array inside the library
 * (room for Q <= 16384; 256 KiB held on every device that loads the library until
 * the process exits) and calls no allocator.  Q > 16384 returns LSG_ERR_ARG with
 * an explanation in lsg_last_error.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.  Every
 * call shares the one array and synchronises the device's default stream, so
 * calls that overlap on the GPU (from several host threads) race on it.
 * x, w: host arrays of Q doubles. */
int lsg_gauss_noalloc(int Q, double *x, double *w);

/* Device bytes lsg_setup_ex would allocate for these sizes (admission model). */
size_t lsg_footprint_bytes(int d, int N, int T, int Q, int precision);

/* Build a context: Gauss tables, weighted coefficient samples, the truncated
 * series a_hat, b_hat (Sec. 4.1, the Q-point discrete Legendre transform of the
 * samples truncated to tensor degree <= T), the band matrices and M
 * (Sec. 4.2, Kronecker form), and the ILU(0) factors of M in natural order
 * (Algorithm 2).
 *   d in {1,2,3}; N >= 3 (N-1 unknowns per direction); T >= 0; Q >= N+1
 *   (Q <= 0 selects Q = N+2); a, b: Q^d samples (a > 0, b >= 0 expected).
 * Returns LSG_ERR_NONFINITE for NaN/Inf samples, LSG_ERR_ILU_BREAKDOWN when a
 * pivot vanishes (the context is still returned so it can be inspected and
 * destroyed), LSG_ERR_NOMEM when memory is short (no context is returned).
 * Synchronises `stream`. */
int lsg_setup(lsg_ctx **out, int d, int N, int T, int Q, const double *a, const double *b,
              int precision, lsg_stream_t stream);
int lsg_setup_ex(lsg_ctx **out, int d, int N, int T, int Q, const double *a, const double *b,
                 int precision, unsigned flags, lsg_stream_t stream);

/* The general problem: a diffusion coefficient per direction and truncation
 * degrees per coefficient and direction,
 *     -sum_j d/dx_j (a_j(x) du/dx_j) + b(x) u = f,
 * the form of Sec. 5 Example 4 (`problem2`, `problem3`: beta_1(x), beta_2(y),
 * beta_3(z)); a_j = a for all j is the problem of lsg_setup.  The preconditioner
 * replaces each a_j by its Legendre series truncated to degree ta[j][i] in
 * direction i and b by its series of degrees tb[i] (Sec. 4.1 with separate t_1 for
 * the diffusion and t_2 for the reaction coefficient; Example 4's t_1j); its
 * structural pattern is the union of the Kronecker terms' bands for those degrees
 * (stiffness band of degree ta[j][j] in direction j, mass bands of degree ta[j][i]
 * in the others; mass bands of degrees tb[i] for b when b is not identically 0).
 * Sizes as in lsg_setup; degrees 0..64; a[j] for j >= d ignored (NULL there,
 * or a[j] == a[0], means the same samples). */
typedef struct {
    int d, N, Q;          /* Q <= 0 selects Q = N+2 */
    const double *a[3];   /* Q^d samples of a_1..a_d (host or device, copied) */
    const double *b;      /* Q^d samples of b */
    int ta[3][3];         /* ta[j][i]: degree of a_j's series in direction i */
    int tb[3];            /* tb[i]: degree of b's series in direction i */
    int precision;        /* lsg_precision */
    unsigned flags;       /* LSG_SETUP_* */
} lsg_problem;
/* Build a context for the general problem (otherwise as lsg_setup_ex). */
int lsg_setup_problem(lsg_ctx **out, const lsg_problem *p, lsg_stream_t stream);

/* F_k = (f, Psi_k) by Q-point quadrature of the samples f (Q^d, Sec. 3). */
int lsg_load_vector(lsg_ctx *ctx, const double *f, double *F, lsg_stream_t stream);

/* y = K x = (A + B) x in FP64, matrix-free (Sec. 4.3: Legendre coefficients,
 * transforms to the Gauss grid, pointwise products with a and b, transposed
 * transforms).  x, y: n doubles; y must not alias x. */
int lsg_apply_A(lsg_ctx *ctx, const double *x, double *y, lsg_stream_t stream);

/* y = K x with the mixed form's low-precision transforms (Sec. 4.3, as
 * lsg_apply_A): each contraction is a tensor-core GEMM with TF32
 * (LSG_MIXED_TF32) or BF16 (LSG_MIXED_BF16) operands and FP32 accumulation;
 * the pointwise products use FP32 copies of the weighted coefficients.
 * x, y: n floats on the device; y must not alias x.  LSG_ERR_ARG for FP64
 * contexts. */
int lsg_apply_A_lowp(lsg_ctx *ctx, const float *x, float *y, lsg_stream_t stream);

/* z = U^{-1} L^{-1} r: the one-step ILU(0) preconditioner solve (Sec. 4.2,
 * Algorithms 3 and 4).  r, z: n doubles; z must not alias r.  Mixed-precision
 * contexts hold FP32 factors; this call sweeps them with FP64 accumulation
 * (their inner PCG sweeps FP32 vectors in FP32). */
int lsg_apply_Minv(lsg_ctx *ctx, const double *r, double *z, lsg_stream_t stream);

/* PCG (Algorithm 1) on K u = F with the ILU(0) preconditioner.
 * u: on entry the initial guess x0, on exit the iterate.  Stops when
 * sqrt(r^T r) <= rtol ||F||_2 (recursive residual) or after kmax passes.
 * Mixed-precision contexts run FP64 iterative refinement: r = F - K u in FP64,
 * an inner PCG in the low precision on r, u += e, until the true FP64
 * relative residual is <= rtol.  info may be NULL.  Synchronises `stream`. */
int lsg_pcg_solve(lsg_ctx *ctx, const double *F, double *u, double rtol, int kmax,
                  lsg_info *info, lsg_stream_t stream);

/* u_N at the Q^d grid (forward transform with the phi tables), for checks. */
int lsg_eval(lsg_ctx *ctx, const double *u, double *vals, lsg_stream_t stream);

/* Number of doubles lsg_export writes for an item (0 if unavailable). */
long long lsg_export_count(lsg_ctx *ctx, int item);
/* Copy an inspection item to the host array `out` (synchronises). */
int lsg_export(lsg_ctx *ctx, int item, double *out);
/* Integer properties of a context (-1 for an unknown item). */
long long lsg_query(lsg_ctx *ctx, int item);
/* Free a context and all its device memory.  The release is ordered on the
 * stream of the context's last call (lsg_setup or a compute call) and waits for
 * that stream only, not for the whole device, so that contexts on other streams
 * keep running; work the caller queued with this context on other streams must
 * be complete (or ordered before that stream) when it calls lsg_destroy. */
int lsg_destroy(lsg_ctx *ctx);

/* Autotuner of the FP64 K x transforms (Sec. 4.3 steps 2-3 as dense contractions,
 * one per direction forward and one backward).  Each contraction has five tile
 * shapes (output rows x batch columns per CTA: 16x16, 16x32, 32x32, 32x64, 64x32,
 * numbered 0-4); for each contraction in turn this times K x with every shape on
 * the context's last stream (the others at their current choice), keeps the
 * fastest, and sweeps twice.  The choice is kept by the context and, for later
 * contexts of the same (d, N, Q), by the process.  Contexts whose size is in the
 * library's committed table (tuned on a GB300) start with that choice.
 * choice (may be NULL): 6 ints, forward contractions 1..3 then backward 1..3
 * (-1: the default shape; entries past d unused).  reps: timed K x per variant
 * (< 1: 5).  Synchronises. */
int lsg_autotune_transforms(lsg_ctx *ctx, int reps, int *choice);
/* The tile choice a context uses (6 ints, as lsg_autotune_transforms). */
int lsg_transform_tiles(lsg_ctx *ctx, int *choice);
/* Set the tile choice of a context (6 ints in -1..4, as lsg_autotune_transforms). */
int lsg_set_transform_tiles(lsg_ctx *ctx, const int *choice);

/* Budget of the device-side dependency waits in this context's triangular sweeps
 * (Algorithms 3 and 4), in SM clock cycles; 0 restores the default (8e9 cycles,
 * about 4 s).  The paper has no counterpart: a sweep CTA that waits longer than
 * this for a value another CTA produces gives up, records LSG_ERR_TIMEOUT in the
 * context's device error word (reported by the synchronising calls, e.g.
 * lsg_pcg_solve) and exits after its own bulk copies have landed.  Every compute
 * call starts with a clear error word, so the context stays usable afterwards.
 * A budget of a few thousand cycles makes the waits expire on purpose, which is
 * how the failure path is tested.  cycles < 0: LSG_ERR_ARG. */
int lsg_set_wait_budget(lsg_ctx *ctx, long long cycles);

/* Batched PCG over `count` independent contexts (uneven sizes allowed):
 * the iterations of all problems are interleaved on the device, each problem
 * stopping at its own tolerance.  F[i], u[i] as in lsg_pcg_solve; infos may
 * be NULL.  When any context is mixed-precision, the problems run as
 * concurrent lsg_pcg_solve calls (a few host threads, one stream each).
 * Returns the first non-OK status.  Synchronises `stream`. */
int lsg_batch_solve(int count, lsg_ctx *const *ctxs, const double *const *F, double *const *u,
                    double rtol, int kmax, lsg_info *infos, lsg_stream_t stream);

/* ---- serving: continuous batching of solve requests ---------------------- */
typedef struct {
    long long id;        /* caller's request id */
    int d, N, T, Q;      /* problem sizes (Q <= 0: N+2) */
    int precision;       /* lsg_precision */
    double rtol;         /* target relative residual */
    int kmax;
    const double *a, *b; /* Q^d host samples (copied at submit) */
    const double *f;     /* Q^d host samples of the right-hand side (copied) */
} lsg_request;

typedef struct {
    long long id;
    lsg_info info;
    double latency_ms;    /* submit -> solution in host memory */
    double *u;            /* n doubles, owned by the server until lsg_server_release */
    long long n;
} lsg_result;

/* Create a server with an HBM budget (bytes) for admitted requests and up to
 * max_inflight concurrently running solves (each on its own stream).  Admission:
 * among the queued requests whose footprint (lsg_footprint_bytes) fits the free
 * budget, the smallest first (the earliest on ties), so short solves are not held
 * behind large ones; but once the oldest queued request has waited longer than
 * the aging bound (default 2000 ms), it alone may be admitted next, so that large
 * requests are not starved by a steady stream of small ones. */
int lsg_server_create(lsg_server **srv, size_t hbm_budget, int max_inflight);
/* Set the aging bound of a server in milliseconds (> 0). */
int lsg_server_set_aging(lsg_server *srv, double ms);
/* Queue a request; returns LSG_ERR_NOMEM if it can never fit the budget. */
int lsg_server_submit(lsg_server *srv, const lsg_request *req);
/* Collect up to `max` finished results; *count receives how many. */
int lsg_server_poll(lsg_server *srv, lsg_result *out, int max, int *count);
/* Block until every queued request has finished. */
int lsg_server_drain(lsg_server *srv);
/* Free the solution buffer of a polled result. */
int lsg_server_release(lsg_server *srv, lsg_result *res);
int lsg_server_destroy(lsg_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* LSG_H */
