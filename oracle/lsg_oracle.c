/*
 * lsg_oracle.c -- plain, slow, FP64 CPU reference for the preconditioned
 * Legendre-Galerkin solve of Diao, Hu & Ma, "Preconditioned Legendre spectral
 * Galerkin methods for the non-separable elliptic equation" (arXiv 2004.13961).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header, table or helper with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Every function follows one passage of the paper and says which.  Where the
 * paper is silent or ambiguous the reading used is stated at the function.
 *
 * Layout conventions (paper Sec. 3, unknown ordering): multi-dimensional
 * arrays are stored with the first (x) index fastest, then y, then z.  The
 * coefficient vector u_hat has n1 = N-1 entries per direction; samples and
 * values live on the Q-point tensor Legendre-Gauss grid with nodes ascending.
 *
 * Parity status: every function here is pinned by a test in
 * tests/test_oracle_pins.py or, for the per-direction form (the *_dir
 * functions: one diffusion coefficient per direction as in Sec. 5 Example 4,
 * truncation degrees per coefficient and direction as in Sec. 4.1's t_1, t_2),
 * tests/test_oracle_pins_dir.py (closed forms, library routines, brute force,
 * invariants); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOMEM (-2)
#define OR_ERR_BREAKDOWN (-4)
#define OR_ERR_NOT_CONVERGED (-5)

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: three-term recurrence L0=1, L1=x, (n+1)L_{n+1}=(2n+1)xL_n-nL_{n-1} */
void or_legendre_all(int nmax, double x, double *L)
{
    L[0] = 1.0;
    if (nmax >= 1) L[1] = x;
    for (int n = 1; n < nmax; ++n)
        L[n + 1] = ((2.0 * n + 1.0) * x * L[n] - (double)n * L[n - 1]) / (n + 1.0);
}

/* Sec. 2.1, derivative recurrence (2n+1)L_n = L'_{n+1} - L'_{n-1}:
 * L'_0 = 0, L'_1 = 1, L'_{n+1} = L'_{n-1} + (2n+1) L_n.  Used only by the dense
 * matrix (a different route to phi'_k than the closed form -(2k+3)L_{k+1}). */
void or_legendre_deriv_all(int nmax, double x, double *dL)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)(nmax + 1));
    or_legendre_all(nmax, x, L);
    dL[0] = 0.0;
    if (nmax >= 1) dL[1] = 1.0;
    for (int n = 1; n < nmax; ++n) dL[n + 1] = dL[n - 1] + (2.0 * n + 1.0) * L[n];
    free(L);
}

/* Sec. 2.2: the Legendre-Gauss nodes are the roots of L_Q (Q points).  Newton
 * iteration on L_Q evaluated by the recurrence, Chebyshev-like start
 * x_i = -cos(pi (4i+3)/(4Q+2)), weights w_i = 2 / ((1-x_i^2) L'_Q(x_i)^2).
 * Nodes ascending; the pair (x_i, x_{Q-1-i}) is made exactly antisymmetric. */
int or_gauss(int Q, double *x, double *w)
{
    if (Q < 1) return OR_ERR_ARG;
    double *L = (double *)malloc(sizeof(double) * (size_t)(Q + 1));
    for (int i = 0; i < Q; ++i) {
        double xi = -cos(M_PI * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
        double dLQ = 1.0;
        for (int it = 0; it < 100; ++it) {
            or_legendre_all(Q, xi, L);
            /* L'_Q(x) = Q (x L_Q - L_{Q-1}) / (x^2 - 1) */
            dLQ = Q * (xi * L[Q] - L[Q - 1]) / (xi * xi - 1.0);
            double dx = L[Q] / dLQ;
            xi -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        or_legendre_all(Q, xi, L);
        dLQ = Q * (xi * L[Q] - L[Q - 1]) / (xi * xi - 1.0);
        x[i] = xi;
        w[i] = 2.0 / ((1.0 - xi * xi) * dLQ * dLQ);
    }
    for (int i = 0; i < Q / 2; ++i) {
        int j = Q - 1 - i;
        double xs = 0.5 * (x[j] - x[i]);
        double ws = 0.5 * (w[i] + w[j]);
        x[i] = -xs; x[j] = xs; w[i] = ws; w[j] = ws;
    }
    if (Q % 2 == 1) x[Q / 2] = 0.0;
    free(L);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Tensor helper: out = Mat applied along one axis of a (<=3)-d array.
 * din[0] is the fastest dimension.  Mat is P x A row-major, din[axis] == A. */
static double *apply_axis(const double *in, const int din[3], int axis,
                          const double *Mat, int P, int A, int dout[3])
{
    dout[0] = din[0]; dout[1] = din[1]; dout[2] = din[2];
    dout[axis] = P;
    size_t tot = (size_t)dout[0] * dout[1] * dout[2];
    double *out = (double *)malloc(sizeof(double) * tot);
    long long istride = (axis == 0) ? 1 : (axis == 1) ? din[0] : (long long)din[0] * din[1];
#pragma omp parallel for collapse(2) schedule(static)
    for (int i2 = 0; i2 < dout[2]; ++i2)
        for (int i1 = 0; i1 < dout[1]; ++i1)
            for (int i0 = 0; i0 < dout[0]; ++i0) {
                int c[3] = {i0, i1, i2};
                int p = c[axis];
                c[axis] = 0;
                long long base = ((long long)c[2] * din[1] + c[1]) * din[0] + c[0];
                double s = 0.0;
                for (int a = 0; a < A; ++a) s += Mat[(size_t)p * A + a] * in[base + a * istride];
                out[((size_t)i2 * dout[1] + i1) * dout[0] + i0] = s;
            }
    return out;
}

/* Step 1 of the fast matvec (Sec. 4.3): phi-coefficients -> Legendre
 * coefficients along one axis.  phi_k = L_k - L_{k+2}, so the plain field has
 * c_k = u_k - u_{k-2}; by the derivative recurrence phi'_k = -(2k+3) L_{k+1},
 * so the derivative field has c_{k+1} = -(2k+3) u_k.  Output length N+1. */
static double *phi_to_leg_axis(const double *in, const int din[3], int axis, int deriv,
                               int N, int dout[3])
{
    int n1 = N - 1;
    dout[0] = din[0]; dout[1] = din[1]; dout[2] = din[2];
    dout[axis] = N + 1;
    size_t tot = (size_t)dout[0] * dout[1] * dout[2];
    double *out = (double *)calloc(tot, sizeof(double));
    long long istride = (axis == 0) ? 1 : (axis == 1) ? din[0] : (long long)din[0] * din[1];
    for (int i2 = 0; i2 < dout[2]; ++i2)
        for (int i1 = 0; i1 < dout[1]; ++i1)
            for (int i0 = 0; i0 < dout[0]; ++i0) {
                int c[3] = {i0, i1, i2};
                int m = c[axis];
                c[axis] = 0;
                long long base = ((long long)c[2] * din[1] + c[1]) * din[0] + c[0];
                double v = 0.0;
                if (deriv) {
                    int k = m - 1;
                    if (k >= 0 && k < n1) v = -(2.0 * k + 3.0) * in[base + k * istride];
                } else {
                    if (m < n1) v += in[base + m * istride];
                    if (m - 2 >= 0 && m - 2 < n1) v -= in[base + (m - 2) * istride];
                }
                out[((size_t)i2 * dout[1] + i1) * dout[0] + i0] = v;
            }
    return out;
}

/* BDLT matrix (Sec. 2.2): B[q][m] = L_m(x_q), m = 0..N. */
static double *bdlt_matrix(int Q, const double *x, int N)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)Q * (N + 1));
    for (int q = 0; q < Q; ++q) or_legendre_all(N, x[q], B + (size_t)q * (N + 1));
    return B;
}

/* FDLT matrix (Sec. 2.2): F[m][q] = (2m+1)/2 w_q L_m(x_q), m = 0..N. */
static double *fdlt_matrix(int Q, const double *x, const double *w, int N)
{
    double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1) * Q);
    double *L = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    for (int q = 0; q < Q; ++q) {
        or_legendre_all(N, x[q], L);
        for (int m = 0; m <= N; ++m) F[(size_t)m * Q + q] = 0.5 * (2.0 * m + 1.0) * w[q] * L[m];
    }
    free(L);
    return F;
}

/* Legendre coefficients (steps 1-2) then grid values of one field of u_N.
 * deriv_axis = -1 gives u_N, otherwise the partial derivative along it. */
static double *field_values(int d, int N, int Q, const double *u, const double *Bm, int deriv_axis)
{
    int n1 = N - 1;
    int dims[3] = {n1, d >= 2 ? n1 : 1, d >= 3 ? n1 : 1};
    double *cur = (double *)malloc(sizeof(double) * (size_t)dims[0] * dims[1] * dims[2]);
    memcpy(cur, u, sizeof(double) * (size_t)dims[0] * dims[1] * dims[2]);
    /* step 1: Legendre coefficients along every axis */
    for (int ax = 0; ax < d; ++ax) {
        int nd[3];
        double *nx = phi_to_leg_axis(cur, dims, ax, ax == deriv_axis, N, nd);
        free(cur); cur = nx; memcpy(dims, nd, sizeof dims);
    }
    /* step 2: BDLT along every axis */
    for (int ax = 0; ax < d; ++ax) {
        int nd[3];
        double *nx = apply_axis(cur, dims, ax, Bm, Q, N + 1, nd);
        free(cur); cur = nx; memcpy(dims, nd, sizeof dims);
    }
    return cur;
}

/* Step 3: pointwise product with a coefficient at the grid, then FDLT along
 * every axis, giving Legendre coefficients c[.] with N+1 entries per axis. */
static double *fdlt_of_product(int d, int N, int Q, const double *vals, const double *coef,
                               const double *Fm)
{
    size_t tot = 1;
    for (int ax = 0; ax < d; ++ax) tot *= (size_t)Q;
    double *g = (double *)malloc(sizeof(double) * tot);
    for (size_t i = 0; i < tot; ++i) g[i] = coef[i] * vals[i];
    int dims[3] = {Q, d >= 2 ? Q : 1, d >= 3 ? Q : 1};
    for (int ax = 0; ax < d; ++ax) {
        int nd[3];
        double *nx = apply_axis(g, dims, ax, Fm, N + 1, Q, nd);
        free(g); g = nx; memcpy(dims, nd, sizeof dims);
    }
    return g;
}

/* Fast matvec y = (A+B) u following Sec. 4.3 step by step (1D, 2D and 3D
 * cases), with the paper's step-4 recombination formulas.  Reading: the grid
 * has Q >= N+1 Gauss points (the paper uses Q = N+1); with Q >= N+1 the
 * projections (I g, L_m), m <= N, are Gauss-exact, so this is the Galerkin
 * matrix built by Q-point quadrature.  beta = a (diffusion), alpha = b
 * (reaction), both sampled on the grid, x fastest. */
int or_apply_K_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2,
                   const double *b, const double *u, double *y);
int or_apply_K(int d, int N, int Q, const double *a, const double *b,
               const double *u, double *y)
{
    return or_apply_K_dir(d, N, Q, a, a, a, b, u, y);
}

/* The same product for the diffusion term -sum_j d/dx_j (beta_j d u/dx_j), one
 * coefficient per direction (Sec. 5, Example 4, problems `problem2` and
 * `problem3`): step 3 multiplies the j-th gradient field by beta_j instead of
 * beta.  a0, a1, a2: beta_1..beta_d sampled on the grid (unused ones ignored). */
int or_apply_K_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2,
                   const double *b, const double *u, double *y)
{
    if (d < 1 || d > 3 || N < 3 || Q < N + 1) return OR_ERR_ARG;
    const double *ad[3] = {a0, a1, a2};
    int n1 = N - 1, NL = N + 1;
    double *x = (double *)malloc(sizeof(double) * Q), *w = (double *)malloc(sizeof(double) * Q);
    or_gauss(Q, x, w);
    double *Bm = bdlt_matrix(Q, x, N);
    double *Fm = fdlt_matrix(Q, x, w, N);

    double *bu = NULL, *ca = NULL;
    double *bd[3] = {NULL, NULL, NULL};
    /* B part: alpha_hat = FDLT(I_N(alpha u_N)) */
    double *uv = field_values(d, N, Q, u, Bm, -1);
    ca = fdlt_of_product(d, N, Q, uv, b, Fm);
    free(uv);
    (void)bu;
    /* A part: beta_hat^{x,y,z} = FDLT(I_N(beta d_i u_N)) */
    for (int ax = 0; ax < d; ++ax) {
        double *dv = field_values(d, N, Q, u, Bm, ax);
        bd[ax] = fdlt_of_product(d, N, Q, dv, ad[ax], Fm);
        free(dv);
    }

    /* step 4 */
    if (d == 1) {
        for (int j = 0; j < n1; ++j) {
            double A = -2.0 * bd[0][j + 1];
            double B = 2.0 * ca[j] / (2.0 * j + 1.0) - 2.0 * ca[j + 2] / (2.0 * j + 5.0);
            y[j] = A + B;
        }
    } else if (d == 2) {
#define C2(arr, k, j) (arr)[(size_t)(j) * NL + (k)]
        for (int j = 0; j < n1; ++j)
            for (int k = 0; k < n1; ++k) {
                const double *bx = bd[0], *by = bd[1];
                double A = 4.0 / (2 * j + 5) * C2(bx, k + 1, j + 2) - 4.0 / (2 * j + 1) * C2(bx, k + 1, j)
                         + 4.0 / (2 * k + 5) * C2(by, k + 2, j + 1) - 4.0 / (2 * k + 1) * C2(by, k, j + 1);
                double B = 4.0 * C2(ca, k, j) / ((2.0 * k + 1) * (2.0 * j + 1))
                         - 4.0 * C2(ca, k, j + 2) / ((2.0 * k + 1) * (2.0 * j + 5))
                         - 4.0 * C2(ca, k + 2, j) / ((2.0 * k + 5) * (2.0 * j + 1))
                         + 4.0 * C2(ca, k + 2, j + 2) / ((2.0 * k + 5) * (2.0 * j + 5));
                y[(size_t)j * n1 + k] = A + B;
            }
#undef C2
    } else {
#define C3(arr, k, j, l) (arr)[((size_t)(l) * NL + (j)) * NL + (k)]
        for (int l = 0; l < n1; ++l)
            for (int j = 0; j < n1; ++j)
                for (int k = 0; k < n1; ++k) {
                    const double *bx = bd[0], *by = bd[1], *bz = bd[2];
                    double k1 = 2.0 * k + 1, k5 = 2.0 * k + 5, j1 = 2.0 * j + 1, j5 = 2.0 * j + 5;
                    double l1 = 2.0 * l + 1, l5 = 2.0 * l + 5;
                    double A =
                        -8.0 / (j1 * l1) * C3(bx, k + 1, j, l) + 8.0 / (j5 * l1) * C3(bx, k + 1, j + 2, l)
                        + 8.0 / (j1 * l5) * C3(bx, k + 1, j, l + 2) - 8.0 / (j5 * l5) * C3(bx, k + 1, j + 2, l + 2)
                        - 8.0 / (k1 * l1) * C3(by, k, j + 1, l) + 8.0 / (k5 * l1) * C3(by, k + 2, j + 1, l)
                        + 8.0 / (k1 * l5) * C3(by, k, j + 1, l + 2) - 8.0 / (k5 * l5) * C3(by, k + 2, j + 1, l + 2)
                        - 8.0 / (k1 * j1) * C3(bz, k, j, l + 1) + 8.0 / (k5 * j1) * C3(bz, k + 2, j, l + 1)
                        + 8.0 / (k1 * j5) * C3(bz, k, j + 2, l + 1) - 8.0 / (k5 * j5) * C3(bz, k + 2, j + 2, l + 1);
                    double B =
                        -8.0 * C3(ca, k, j, l + 2) / (k1 * j1 * l5) + 8.0 * C3(ca, k, j, l) / (k1 * j1 * l1)
                        - 8.0 * C3(ca, k, j + 2, l) / (k1 * j5 * l1) + 8.0 * C3(ca, k, j + 2, l + 2) / (k1 * j5 * l5)
                        - 8.0 * C3(ca, k + 2, j, l) / (k5 * j1 * l1) + 8.0 * C3(ca, k + 2, j + 2, l) / (k5 * j5 * l1)
                        + 8.0 * C3(ca, k + 2, j, l + 2) / (k5 * j1 * l5) - 8.0 * C3(ca, k + 2, j + 2, l + 2) / (k5 * j5 * l5);
                    y[((size_t)l * n1 + j) * n1 + k] = A + B;
                }
#undef C3
    }
    for (int ax = 0; ax < d; ++ax) free(bd[ax]);
    free(ca); free(Bm); free(Fm); free(x); free(w);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense quadrature Galerkin matrix (Sec. 3, `algebraicsystem`, with the
 * integrals replaced by Q-point Gauss quadrature): for tiny sizes only.
 * K[r][c] = sum_grid W * (a grad Psi_r . grad Psi_c + b Psi_r Psi_c),
 * Psi_(k,j,l) = phi_k(x) phi_j(y) phi_l(z), phi'_k from the derivative
 * recurrence.  Row/column index r = k + n1 j + n1^2 l. */
int or_dense_K_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2,
                   const double *b, double *K);
int or_dense_K(int d, int N, int Q, const double *a, const double *b, double *K)
{
    return or_dense_K_dir(d, N, Q, a, a, a, b, K);
}

/* The dense matrix of the per-direction diffusion term (Sec. 5, Example 4):
 * K[r][c] = sum_grid W * (sum_j beta_j d_j Psi_r d_j Psi_c + alpha Psi_r Psi_c). */
int or_dense_K_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2,
                   const double *b, double *K)
{
    if (d < 1 || d > 3 || N < 3 || Q < 1) return OR_ERR_ARG;
    const double *ad[3] = {a0, a1, a2};
    int n1 = N - 1;
    double *x = (double *)malloc(sizeof(double) * Q), *w = (double *)malloc(sizeof(double) * Q);
    or_gauss(Q, x, w);
    double *ph = (double *)malloc(sizeof(double) * (size_t)Q * n1);
    double *dph = (double *)malloc(sizeof(double) * (size_t)Q * n1);
    double *L = (double *)malloc(sizeof(double) * (N + 2));
    double *dL = (double *)malloc(sizeof(double) * (N + 2));
    for (int q = 0; q < Q; ++q) {
        or_legendre_all(N + 1, x[q], L);
        or_legendre_deriv_all(N + 1, x[q], dL);
        for (int k = 0; k < n1; ++k) {
            ph[(size_t)q * n1 + k] = L[k] - L[k + 2];
            dph[(size_t)q * n1 + k] = dL[k] - dL[k + 2];
        }
    }
    int nd = 1, nq = 1;
    for (int i = 0; i < d; ++i) { nd *= n1; nq *= Q; }
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < nd; ++r) {
        int ri[3] = {r % n1, (r / n1) % n1, r / (n1 * n1)};
        for (int c = 0; c < nd; ++c) {
            int ci[3] = {c % n1, (c / n1) % n1, c / (n1 * n1)};
            double s = 0.0;
            for (int g = 0; g < nq; ++g) {
                int gi[3] = {g % Q, (g / Q) % Q, g / (Q * Q)};
                double W = 1.0, pr = 1.0, pc = 1.0, grad = 0.0;
                for (int ax = 0; ax < d; ++ax) {
                    W *= w[gi[ax]];
                    pr *= ph[(size_t)gi[ax] * n1 + ri[ax]];
                    pc *= ph[(size_t)gi[ax] * n1 + ci[ax]];
                }
                for (int ax = 0; ax < d; ++ax) {
                    double tr = 1.0, tc = 1.0;
                    for (int bx = 0; bx < d; ++bx) {
                        tr *= (bx == ax) ? dph[(size_t)gi[bx] * n1 + ri[bx]] : ph[(size_t)gi[bx] * n1 + ri[bx]];
                        tc *= (bx == ax) ? dph[(size_t)gi[bx] * n1 + ci[bx]] : ph[(size_t)gi[bx] * n1 + ci[bx]];
                    }
                    grad += ad[ax][g] * tr * tc;
                }
                s += W * (grad + b[g] * pr * pc);
            }
            K[(size_t)r * nd + c] = s;
        }
    }
    free(ph); free(dph); free(L); free(dL); free(x); free(w);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Load vector F_k = (f, Psi_k) by Q-point quadrature of sampled f (Sec. 3:
 * f_k = (f, phi_k), tensor products in 2D/3D), sum over the grid axis by axis. */
int or_load_vector(int d, int N, int Q, const double *f, double *F)
{
    if (d < 1 || d > 3 || N < 3 || Q < 1) return OR_ERR_ARG;
    int n1 = N - 1;
    double *x = (double *)malloc(sizeof(double) * Q), *w = (double *)malloc(sizeof(double) * Q);
    or_gauss(Q, x, w);
    double *P = (double *)malloc(sizeof(double) * (size_t)n1 * Q);
    double *L = (double *)malloc(sizeof(double) * (N + 2));
    for (int q = 0; q < Q; ++q) {
        or_legendre_all(N + 1, x[q], L);
        for (int k = 0; k < n1; ++k) P[(size_t)k * Q + q] = w[q] * (L[k] - L[k + 2]);
    }
    int dims[3] = {Q, d >= 2 ? Q : 1, d >= 3 ? Q : 1};
    size_t tot = (size_t)dims[0] * dims[1] * dims[2];
    double *cur = (double *)malloc(sizeof(double) * tot);
    memcpy(cur, f, sizeof(double) * tot);
    for (int ax = 0; ax < d; ++ax) {
        int nd[3];
        double *nx = apply_axis(cur, dims, ax, P, n1, Q, nd);
        free(cur); cur = nx; memcpy(dims, nd, sizeof dims);
    }
    memcpy(F, cur, sizeof(double) * (size_t)dims[0] * dims[1] * dims[2]);
    free(cur); free(P); free(L); free(x); free(w);
    return OR_OK;
}

/* Load vector from the Legendre coefficients of f (degree <= deg per axis) in
 * closed form by orthogonality (Sec. 2.1): (L_p, L_q) = 2/(2p+1) delta_pq and
 * phi_k = L_k - L_{k+2}, so (f, phi_k) = 2 f_k/(2k+1) - 2 f_{k+2}/(2k+5) per
 * axis.  fc is (deg+1)^d, first index fastest. */
int or_load_vector_legendre(int d, int N, int deg, const double *fc, double *F)
{
    if (d < 1 || d > 3 || N < 3 || deg < 0) return OR_ERR_ARG;
    int n1 = N - 1, D1 = deg + 1;
    int nd = 1;
    for (int i = 0; i < d; ++i) nd *= n1;
    for (int r = 0; r < nd; ++r) {
        int ki[3] = {r % n1, (r / n1) % n1, r / (n1 * n1)};
        double s = 0.0;
        int ncomb = 1 << d;
        for (int m = 0; m < ncomb; ++m) {
            double fac = 1.0;
            int p[3] = {0, 0, 0};
            int ok = 1;
            for (int ax = 0; ax < d; ++ax) {
                int hi = (m >> ax) & 1;
                p[ax] = ki[ax] + 2 * hi;
                if (p[ax] > deg) { ok = 0; break; }
                fac *= (hi ? -1.0 : 1.0) * 2.0 / (2.0 * p[ax] + 1.0);
            }
            if (!ok) continue;
            s += fac * fc[((size_t)p[2] * D1 + p[1]) * D1 + p[0]];
        }
        F[r] = s;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Truncated coefficient series (Sec. 4.1, `Appbeta`, `1DM`-`3DM`; FDLT of
 * Sec. 2.2 applied to the given samples): for every t_i <= T,
 * chat_t = prod_i (2 t_i + 1)/2 * sum_grid W c L_t.  Reading: truncation of
 * the Q-point discrete Legendre series of the samples (tensor degree <= T). */
int or_coef_trunc(int d, int Q, int T, const double *c, double *chat)
{
    if (d < 1 || d > 3 || Q < 1 || T < 0) return OR_ERR_ARG;
    double *x = (double *)malloc(sizeof(double) * Q), *w = (double *)malloc(sizeof(double) * Q);
    or_gauss(Q, x, w);
    double *Lt = (double *)malloc(sizeof(double) * (size_t)Q * (T + 1));
    for (int q = 0; q < Q; ++q) or_legendre_all(T, x[q], Lt + (size_t)q * (T + 1));
    int T1 = T + 1;
    int nt = 1, nq = 1;
    for (int i = 0; i < d; ++i) { nt *= T1; nq *= Q; }
    for (int ti = 0; ti < nt; ++ti) {
        int t[3] = {ti % T1, (ti / T1) % T1, ti / (T1 * T1)};
        double s = 0.0;
        for (int g = 0; g < nq; ++g) {
            int gi[3] = {g % Q, (g / Q) % Q, g / (Q * Q)};
            double v = c[g];
            for (int ax = 0; ax < d; ++ax) v *= w[gi[ax]] * Lt[(size_t)gi[ax] * T1 + t[ax]];
            s += v;
        }
        for (int ax = 0; ax < d; ++ax) s *= (2.0 * t[ax] + 1.0) / 2.0;
        chat[ti] = s;
    }
    free(Lt); free(x); free(w);
    return OR_OK;
}

/* Per-direction truncation (Sec. 4.1 `Appbeta`/`Appalpha` with separate
 * degrees; Sec. 5 Example 4's t_1j): the coefficients of or_coef_trunc with
 * t_i <= deg[i] in direction i, the others zero; chat holds (T+1)^d entries
 * with T >= every deg[i]. */
int or_coef_trunc_dir(int d, int Q, int T, const int *deg, const double *c, double *chat)
{
    int rc = or_coef_trunc(d, Q, T, c, chat);
    if (rc != OR_OK) return rc;
    int T1 = T + 1, nt = 1;
    for (int i = 0; i < d; ++i) {
        if (deg[i] < 0 || deg[i] > T) return OR_ERR_ARG;
        nt *= T1;
    }
    for (int ti = 0; ti < nt; ++ti) {
        int t[3] = {ti % T1, (ti / T1) % T1, ti / (T1 * T1)};
        for (int ax = 0; ax < d; ++ax)
            if (t[ax] > deg[ax]) chat[ti] = 0.0;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 1D band matrices of Sec. 4.2 (Kronecker form of M):
 *   S[t][i][m] = (L_t phi'_i, phi'_m),  Mm[t][i][m] = (L_t phi_i, phi_m),
 * 0 <= i,m <= N-2 (the paper's 0..N-1 is read as 0..N-2), computed for
 * |i-m| <= T+2 (Proposition 4.1 bounds the band) by Gauss quadrature with
 * QM = N + ceil(T/2) + 2 points, exact since the integrands have degree
 * <= 2N+T.  Output dense n1 x n1 per t (zeros outside the band). */
int or_band_matrices(int N, int T, double *S, double *Mm)
{
    if (N < 3 || T < 0) return OR_ERR_ARG;
    int n1 = N - 1, QM = N + (T + 1) / 2 + 2;
    double *x = (double *)malloc(sizeof(double) * QM), *w = (double *)malloc(sizeof(double) * QM);
    or_gauss(QM, x, w);
    int LM = (N + 1 > T) ? N + 1 : T;
    double *L = (double *)malloc(sizeof(double) * (size_t)QM * (LM + 1));
    for (int q = 0; q < QM; ++q) or_legendre_all(LM, x[q], L + (size_t)q * (LM + 1));
#define LV(q, m) L[(size_t)(q) * (LM + 1) + (m)]
    memset(S, 0, sizeof(double) * (size_t)(T + 1) * n1 * n1);
    memset(Mm, 0, sizeof(double) * (size_t)(T + 1) * n1 * n1);
    for (int t = 0; t <= T; ++t)
        for (int i = 0; i < n1; ++i)
            for (int m = 0; m < n1; ++m) {
                if (abs(i - m) > T + 2) continue;
                double ss = 0.0, sm = 0.0;
                for (int q = 0; q < QM; ++q) {
                    double dpi = -(2.0 * i + 3.0) * LV(q, i + 1), dpm = -(2.0 * m + 3.0) * LV(q, m + 1);
                    double pi = LV(q, i) - LV(q, i + 2), pm = LV(q, m) - LV(q, m + 2);
                    ss += w[q] * LV(q, t) * dpi * dpm;
                    sm += w[q] * LV(q, t) * pi * pm;
                }
                S[((size_t)t * n1 + i) * n1 + m] = ss;
                Mm[((size_t)t * n1 + i) * n1 + m] = sm;
            }
#undef LV
    free(L); free(x); free(w);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Structural pattern of M.  Reading of NZ(M) (Sec. 4.2 defines it by
 * nonzero entries): the union of the structural patterns of the Kronecker
 * terms of M (Sec. 4.2, `2DM`, `3DM`), without value-based dropping.  By
 * Proposition 4.1 and orthogonality, (L_t phi'_i, phi'_m) vanishes unless
 * |i-m| <= t with i+m+t even, and (L_t phi_i, phi_m) unless |i-m| <= t+2 with
 * i+m+t even; the union over t <= T gives the 1D offset sets below.  The mass
 * term b_hat enters only when b is not identically zero. */
static int band_s(int o, int T) { return abs(o) <= T; }
static int band_m(int o, int T)
{
    int a = abs(o);
    if (a > T + 2) return 0;
    if (T == 0) return (a % 2) == 0;
    return 1;
}
/* Degrees of the coefficient series: ta[3 j + i] is the degree of beta_j's series
 * in direction i (beta_j multiplies the j-th gradient term), tb[i] that of
 * alpha's.  The isotropic problem with one degree T has every entry T; Sec. 4.1's
 * separate t_1 (beta) and t_2 (alpha) fill ta with t_1 and tb with t_2. */
static void iso_degrees(int T, int *ta, int *tb)
{
    for (int i = 0; i < 9; ++i) ta[i] = T;
    for (int i = 0; i < 3; ++i) tb[i] = T;
}

/* Kronecker term j (stiffness in direction j): S band of degree ta[j][j] in
 * direction j, M bands of degree ta[j][i] in the others; the mass term (when
 * alpha is present): M bands of degree tb[i] in every direction. */
static int in_pattern_dir(int d, const int *o, const int *ta, const int *tb, int has_b)
{
    for (int j = 0; j < d; ++j) {
        int ok = band_s(o[j], ta[3 * j + j]);
        for (int i = 0; i < d && ok; ++i)
            if (i != j) ok = band_m(o[i], ta[3 * j + i]);
        if (ok) return 1;
    }
    if (has_b) {
        int ok = 1;
        for (int i = 0; i < d && ok; ++i) ok = band_m(o[i], tb[i]);
        if (ok) return 1;
    }
    return 0;
}

/* Half-width of the offset box that holds every band of the pattern. */
static int pattern_width(int d, const int *ta, const int *tb)
{
    int w = 0;
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) {
            int h = (i == j) ? ta[3 * j + i] : ta[3 * j + i] + 2;
            if (h > w) w = h;
        }
    for (int i = 0; i < d; ++i)
        if (tb[i] + 2 > w) w = tb[i] + 2;
    return w;
}

/* Number of structural nonzeros of M (rows in natural order). */
long long or_pattern_nnz_dir(int d, int N, const int *ta, const int *tb, int has_b)
{
    int n1 = N - 1, w = pattern_width(d, ta, tb);
    long long nd = 1;
    for (int i = 0; i < d; ++i) nd *= n1;
    long long nnz = 0;
    for (long long r = 0; r < nd; ++r) {
        int ri[3] = {(int)(r % n1), (int)((r / n1) % n1), (int)(r / ((long long)n1 * n1))};
        for (int oz = (d >= 3 ? -w : 0); oz <= (d >= 3 ? w : 0); ++oz)
            for (int oy = (d >= 2 ? -w : 0); oy <= (d >= 2 ? w : 0); ++oy)
                for (int ox = -w; ox <= w; ++ox) {
                    int o[3] = {ox, oy, oz};
                    int ok = 1;
                    for (int ax = 0; ax < d; ++ax) {
                        int c = ri[ax] + o[ax];
                        if (c < 0 || c >= n1) ok = 0;
                    }
                    if (ok && in_pattern_dir(d, o, ta, tb, has_b)) ++nnz;
                }
    }
    return nnz;
}

long long or_pattern_nnz(int d, int N, int T, int has_b)
{
    int ta[9], tb[3];
    iso_degrees(T, ta, tb);
    return or_pattern_nnz_dir(d, N, ta, tb, has_b);
}

/* Preconditioner M (Sec. 4.1 `1DM`/`2DM`/`3DM` with p_t the truncated series,
 * in the Kronecker form of Sec. 4.2) assembled in CSR, columns ascending:
 *   2D: M = sum_{t,k} ahat0_tk M^(k)_y (x) S^(t)_x + ahat1_tk S^(k)_y (x) M^(t)_x
 *           + bhat_tk M^(k)_y (x) M^(t)_x
 *   3D: the three stiffness terms (S in direction j with beta_j's series ahat_j,
 *       M in the others) and the mass term, summed over t,k,l.
 * With one beta (the isotropic problem) ahat0 = ahat1 = ahat2.  Each series is
 * (T+1)^d, x-degree fastest, zero beyond its per-direction degrees (ta, tb as
 * above, every degree <= T).  S, Mm from or_band_matrices(N, T). */
int or_assemble_M_dir(int d, int N, int T, const double *ahat0, const double *ahat1, const double *ahat2,
                      const double *bhat, const int *ta, const int *tb, int has_b,
                      const double *S, const double *Mm,
                      int64_t *rowptr, int32_t *col, double *val)
{
    if (d < 1 || d > 3 || N < 3 || T < 0) return OR_ERR_ARG;
    for (int i = 0; i < 9; ++i)
        if (ta[i] < 0 || ta[i] > T) return OR_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (tb[i] < 0 || tb[i] > T) return OR_ERR_ARG;
    int n1 = N - 1, w = pattern_width(d, ta, tb), T1 = T + 1;
    long long nd = 1;
    for (int i = 0; i < d; ++i) nd *= n1;
    /* row pointers first (pattern only) */
    rowptr[0] = 0;
    for (long long r = 0; r < nd; ++r) {
        int ri[3] = {(int)(r % n1), (int)((r / n1) % n1), (int)(r / ((long long)n1 * n1))};
        long long cnt = 0;
        for (int oz = (d >= 3 ? -w : 0); oz <= (d >= 3 ? w : 0); ++oz)
            for (int oy = (d >= 2 ? -w : 0); oy <= (d >= 2 ? w : 0); ++oy)
                for (int ox = -w; ox <= w; ++ox) {
                    int o[3] = {ox, oy, oz};
                    int ok = 1;
                    for (int ax = 0; ax < d; ++ax) {
                        int c = ri[ax] + o[ax];
                        if (c < 0 || c >= n1) ok = 0;
                    }
                    if (ok && in_pattern_dir(d, o, ta, tb, has_b)) ++cnt;
                }
        rowptr[r + 1] = rowptr[r] + cnt;
    }
#define SB(t, i, m) S[((size_t)(t) * n1 + (i)) * n1 + (m)]
#define MB(t, i, m) Mm[((size_t)(t) * n1 + (i)) * n1 + (m)]
#pragma omp parallel for schedule(dynamic, 64)
    for (long long r = 0; r < nd; ++r) {
        int ri[3] = {(int)(r % n1), (int)((r / n1) % n1), (int)(r / ((long long)n1 * n1))};
        long long pos = rowptr[r];
        for (int oz = (d >= 3 ? -w : 0); oz <= (d >= 3 ? w : 0); ++oz)
            for (int oy = (d >= 2 ? -w : 0); oy <= (d >= 2 ? w : 0); ++oy)
                for (int ox = -w; ox <= w; ++ox) {
                    int o[3] = {ox, oy, oz};
                    int ci[3] = {0, 0, 0};
                    int ok = 1;
                    for (int ax = 0; ax < d; ++ax) {
                        ci[ax] = ri[ax] + o[ax];
                        if (ci[ax] < 0 || ci[ax] >= n1) ok = 0;
                    }
                    if (!ok || !in_pattern_dir(d, o, ta, tb, has_b)) continue;
                    double v = 0.0;
                    if (d == 1) {
                        for (int t = 0; t < T1; ++t) {
                            v += ahat0[t] * SB(t, ri[0], ci[0]);
                            if (has_b) v += bhat[t] * MB(t, ri[0], ci[0]);
                        }
                    } else if (d == 2) {
                        int i = ri[0], m = ci[0], j = ri[1], nn = ci[1];
                        for (int t = 0; t < T1; ++t)
                            for (int k = 0; k < T1; ++k) {
                                size_t tk = (size_t)k * T1 + t;
                                v += ahat0[tk] * MB(k, j, nn) * SB(t, i, m) + ahat1[tk] * SB(k, j, nn) * MB(t, i, m);
                                if (has_b) v += bhat[tk] * MB(k, j, nn) * MB(t, i, m);
                            }
                    } else {
                        int i = ri[0], m = ci[0], j = ri[1], nn = ci[1], k3 = ri[2], l3 = ci[2];
                        for (int t = 0; t < T1; ++t)
                            for (int k = 0; k < T1; ++k)
                                for (int l = 0; l < T1; ++l) {
                                    size_t tkl = ((size_t)l * T1 + k) * T1 + t;
                                    v += ahat0[tkl] * MB(l, k3, l3) * MB(k, j, nn) * SB(t, i, m)
                                       + ahat1[tkl] * MB(l, k3, l3) * SB(k, j, nn) * MB(t, i, m)
                                       + ahat2[tkl] * SB(l, k3, l3) * MB(k, j, nn) * MB(t, i, m);
                                    if (has_b) v += bhat[tkl] * MB(l, k3, l3) * MB(k, j, nn) * MB(t, i, m);
                                }
                    }
                    long long c = ci[0] + (long long)n1 * ci[1] + (long long)n1 * n1 * ci[2];
                    col[pos] = (int32_t)c;
                    val[pos] = v;
                    ++pos;
                }
    }
#undef SB
#undef MB
    return OR_OK;
}

int or_assemble_M(int d, int N, int T, const double *ahat, const double *bhat, int has_b,
                  const double *S, const double *Mm,
                  int64_t *rowptr, int32_t *col, double *val)
{
    int ta[9], tb[3];
    iso_degrees(T, ta, tb);
    return or_assemble_M_dir(d, N, T, ahat, ahat, ahat, bhat, ta, tb, has_b, S, Mm, rowptr, col, val);
}

/* ------------------------------------------------------------------------ */
/* ILU(0), Algorithm 2 (IKJ form, in place over NZ(H)): for each row i, for
 * each k < i in the row (ascending), H(i,k) /= H(k,k), then for each j > k in
 * row i, H(i,j) -= H(i,k) * H(k,j), where H(k,j) is zero when (k,j) is not in
 * NZ.  Reading of "assuming they exist": a pivot U(i,i) <= 1e-14 |M(i,i)|
 * stops with a breakdown status. */
int or_ilu0(long long n, const int64_t *rowptr, const int32_t *col, double *H)
{
    int64_t *diag = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!diag || !pos) { free(diag); free(pos); return OR_ERR_NOMEM; }
    for (long long i = 0; i < n; ++i) {
        diag[i] = -1;
        pos[i] = -1;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] == i) diag[i] = p;
        if (diag[i] < 0) { free(diag); free(pos); return OR_ERR_ARG; }
    }
    int status = OR_OK;
    for (long long i = 0; i < n; ++i) {
        double mii = H[diag[i]];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[col[p]] = p;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1] && col[p] < i; ++p) {
            long long k = col[p];
            H[p] = H[p] / H[diag[k]];
            double hik = H[p];
            for (int64_t q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
                int64_t pj = pos[col[q]];
                if (pj >= 0) H[pj] -= hik * H[q];
            }
        }
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[col[p]] = -1;
        if (!(H[diag[i]] > 1e-14 * fabs(mii))) status = OR_ERR_BREAKDOWN;
    }
    free(diag); free(pos);
    return status;
}

/* Algorithm 3 (forward substitution, unit lower L) followed by Algorithm 4
 * (backward substitution, upper U), the one-step ILU(0) solve of M z = r
 * (Sec. 4.2, steps 2 and 3).  LU holds L (strictly lower) and U in place. */
int or_ilu_solve(long long n, const int64_t *rowptr, const int32_t *col, const double *LU,
                 const double *r, double *z)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    if (!y) return OR_ERR_NOMEM;
    for (long long i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1] && col[p] < i; ++p) s += LU[p] * y[col[p]];
        y[i] = r[i] - s;
    }
    for (long long i = n - 1; i >= 0; --i) {
        double s = y[i], uii = 0.0;
        for (int64_t p = rowptr[i + 1] - 1; p >= rowptr[i] && col[p] >= i; --p) {
            if (col[p] == i) uii = LU[p];
            else s -= LU[p] * z[col[p]];
        }
        z[i] = s / uii;
    }
    free(y);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (PCG).  Readings: x holds the initial guess on entry; the stop
 * test is on the recursive residual sqrt(r^T r) <= eps ||F||_2; "iterations"
 * counts completed loop passes k.  The preconditioner solve is the ILU(0)
 * one-step process; K x is the matrix-free product above.  Also returns the
 * true relative residual ||F - K x|| / ||F||.  p^T w <= 0 stops with
 * OR_ERR_NOT_CONVERGED. */
int or_pcg_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2, const double *b,
               const int64_t *rowptr, const int32_t *col, const double *LU,
               const double *F, double *x, double eps, int kmax,
               int *iters, double *relres_rec, double *relres_true);
int or_pcg(int d, int N, int Q, const double *a, const double *b,
           const int64_t *rowptr, const int32_t *col, const double *LU,
           const double *F, double *x, double eps, int kmax,
           int *iters, double *relres_rec, double *relres_true)
{
    return or_pcg_dir(d, N, Q, a, a, a, b, rowptr, col, LU, F, x, eps, kmax, iters, relres_rec, relres_true);
}

/* Algorithm 1 for the per-direction diffusion term (Sec. 5, Example 4). */
int or_pcg_dir(int d, int N, int Q, const double *a0, const double *a1, const double *a2, const double *b,
               const int64_t *rowptr, const int32_t *col, const double *LU,
               const double *F, double *x, double eps, int kmax,
               int *iters, double *relres_rec, double *relres_true)
{
    int n1 = N - 1;
    long long n = 1;
    for (int i = 0; i < d; ++i) n *= n1;
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *wv = (double *)malloc(sizeof(double) * n);
    if (!r || !z || !p || !wv) return OR_ERR_NOMEM;
    double nF = 0.0;
    for (long long i = 0; i < n; ++i) nF += F[i] * F[i];
    nF = sqrt(nF);
    or_apply_K_dir(d, N, Q, a0, a1, a2, b, x, wv);
    for (long long i = 0; i < n; ++i) r[i] = F[i] - wv[i];
    double rr = 0.0;
    for (long long i = 0; i < n; ++i) rr += r[i] * r[i];
    int k = 0, status = OR_OK;
    double rho = 0.0;
    while (sqrt(rr) > eps * nF && k < kmax) {
        or_ilu_solve(n, rowptr, col, LU, r, z);
        k = k + 1;
        if (k == 1) {
            for (long long i = 0; i < n; ++i) p[i] = z[i];
            rho = 0.0;
            for (long long i = 0; i < n; ++i) rho += r[i] * z[i];
        } else {
            double rho_t = rho;
            rho = 0.0;
            for (long long i = 0; i < n; ++i) rho += r[i] * z[i];
            double beta = rho / rho_t;
            for (long long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        or_apply_K_dir(d, N, Q, a0, a1, a2, b, p, wv);
        double pw = 0.0;
        for (long long i = 0; i < n; ++i) pw += p[i] * wv[i];
        if (!(pw > 0.0)) { status = OR_ERR_NOT_CONVERGED; break; }
        double alpha = rho / pw;
        for (long long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * wv[i]; }
        rr = 0.0;
        for (long long i = 0; i < n; ++i) rr += r[i] * r[i];
    }
    if (status == OR_OK && sqrt(rr) > eps * nF) status = OR_ERR_NOT_CONVERGED;
    *iters = k;
    *relres_rec = (nF > 0) ? sqrt(rr) / nF : sqrt(rr);
    or_apply_K_dir(d, N, Q, a0, a1, a2, b, x, wv);
    double tr = 0.0;
    for (long long i = 0; i < n; ++i) tr += (F[i] - wv[i]) * (F[i] - wv[i]);
    *relres_true = (nF > 0) ? sqrt(tr) / nF : sqrt(tr);
    free(r); free(z); free(p); free(wv);
    return status;
}
