// transform.cu -- the matrix-free product y = K x = (A + B) x of Sec. 4.3 in
// FP64 on the GB300, as sum-factorised contractions with the basis tables.
//
// Sec. 4.3 evaluates K x by (1) Legendre coefficients of u_N and grad u_N,
// (2) transforms to the Gauss grid, (3) pointwise products with a and b and
// transforms back, (4) recombination into the phi basis.  Steps 1+2 and 3+4
// are each one linear map per direction: contraction with the tables
// Phi[q][k] = phi_k(x_q) and D[q][k] = phi'_k(x_q) (forward) and their
// transposes (backward).  With Q-point Gauss quadrature this is exactly the
// quadrature Galerkin matrix; the kernels below apply it direction by
// direction ("contract the fastest axis, write the new axis slowest"), so that
// after d contractions the axes are back in x-fastest order.
//
// Parity folding: nodes are symmetric and phi_k(-x) = (-1)^k phi_k(x),
// phi'_k(-x) = (-1)^(k+1) phi'_k(x), so every contraction splits into an even
// and an odd half of half the length -- half the flops of the plain tables.
#include "lsg_internal.cuh"

namespace lsg {

template <typename T>
struct XfTerm {
    const T *x;
    int tab;  // 0: phi (mirror sign +1), 1: phi' (mirror sign -1)
};
template <typename T>
struct XfOut {
    T *y;
    const T *scale;  // optional pointwise factor at the output (W a or W b)
    int nterm;
    XfTerm<T> t[2];
};
template <typename T>
struct XfJob {
    int nout;
    XfOut<T> o[4];
    long long B;     // batch: product of the untouched axes (output row length)
    int Q, Qh, n1, KP;
    const T *tabE[2], *tabO[2];  // [QhP][KP]
    const int *done;             // optional: skip when *done != 0
};

constexpr int XT = 256;  // threads per transform CTA

// Forward: coefficients (fastest axis, length n1) -> grid values (new slowest
// axis, length Q).  out[q][b] = sum_k T[q][k] x[b][k] for the term's table T.
// Tile: TP half-nodes x TB batch columns; 16x16 threads, each RP x RB outputs
// for the even and the odd half.
// MODE 0: the node-symmetry fold above (outputs at nodes p and Q-1-p).  MODE 1: the
// tables are parity blocks of a matrix that couples only indices of equal parity (the
// eigenvector matrices of the constant-coefficient preconditioner): the even half of the
// input gives output rows 2p, the odd half rows 2p+1 (n1 rows in all).
template <typename T, int TP, int TB, int TK, int MODE = 0>
__global__ void __launch_bounds__(XT) k_xf_fwd(const __grid_constant__ XfJob<T> job)
{
    if (job.done && *job.done) return;
    const XfOut<T> &O = job.o[blockIdx.z];
    constexpr int RP = TP / 16, RB = TB / 16;
    __shared__ T sAe[TK][TP + 1], sAo[TK][TP + 1];
    __shared__ T sXe[TK][TB + 1], sXo[TK][TB + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int p0 = blockIdx.x * TP;
    const long long b0 = (long long)blockIdx.y * TB;
    const XfTerm<T> tm = O.t[0];
    const T *TE = job.tabE[tm.tab], *TO = job.tabO[tm.tab];
    const int n1 = job.n1, KP = job.KP;
    const long long B = job.B;

    T ae[RP][RB], ao[RP][RB];
#pragma unroll
    for (int i = 0; i < RP; ++i)
#pragma unroll
        for (int j = 0; j < RB; ++j) ae[i][j] = ao[i][j] = 0.0;

    const int ne = (n1 + 1) / 2;
    for (int m0 = 0; m0 < ne; m0 += TK) {
        // tables: [p][m] rows padded to QhP, columns to KP (zeros)
        for (int idx = tid; idx < TK * TP; idx += XT) {
            int mm = idx % TK, pp = idx / TK;
            size_t off = (size_t)(p0 + pp) * KP + (m0 + mm);
            sAe[mm][pp] = TE[off];
            sAo[mm][pp] = TO[off];
        }
        // input: x[b][a] with a in [2 m0, 2 m0 + 2 TK), split even/odd
        for (int idx = tid; idx < 2 * TK * TB; idx += XT) {
            int aa = idx % (2 * TK), bb = idx / (2 * TK);
            int a = 2 * m0 + aa;
            long long b = b0 + bb;
            T v = (b < B && a < n1) ? tm.x[b * n1 + a] : T(0);
            if (aa & 1)
                sXo[aa >> 1][bb] = v;
            else
                sXe[aa >> 1][bb] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T re[RP], ro[RP], ce[RB], co[RB];
#pragma unroll
            for (int i = 0; i < RP; ++i) {
                re[i] = sAe[kk][ty + 16 * i];
                ro[i] = sAo[kk][ty + 16 * i];
            }
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                ce[j] = sXe[kk][tx + 16 * j];
                co[j] = sXo[kk][tx + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < RP; ++i)
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    ae[i][j] = fma(re[i], ce[j], ae[i][j]);
                    ao[i][j] = fma(ro[i], co[j], ao[i][j]);
                }
        }
        __syncthreads();
    }
    if (MODE == 1) {
#pragma unroll
        for (int i = 0; i < RP; ++i) {
            const int p = p0 + ty + 16 * i, re = 2 * p, ro = 2 * p + 1;
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                const long long b = b0 + tx + 16 * j;
                if (b >= B) continue;
                if (re < n1) O.y[(size_t)re * B + b] = O.scale ? ae[i][j] * O.scale[(size_t)re * B + b] : ae[i][j];
                if (ro < n1) O.y[(size_t)ro * B + b] = O.scale ? ao[i][j] * O.scale[(size_t)ro * B + b] : ao[i][j];
            }
        }
        return;
    }
    const T sg = tm.tab ? T(-1) : T(1);
    const int Q = job.Q, Qh = job.Qh;
#pragma unroll
    for (int i = 0; i < RP; ++i) {
        int p = p0 + ty + 16 * i;
        if (p >= Qh) continue;
        int q1 = p, q2 = Q - 1 - p;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            long long b = b0 + tx + 16 * j;
            if (b >= B) continue;
            T v1 = ae[i][j] + ao[i][j];
            T v2 = sg * (ae[i][j] - ao[i][j]);
            if (O.scale) {
                v1 *= O.scale[(size_t)q1 * B + b];
                v2 *= O.scale[(size_t)q2 * B + b];
            }
            O.y[(size_t)q1 * B + b] = v1;
            if (q2 != q1) O.y[(size_t)q2 * B + b] = v2;
        }
    }
}

// Backward: grid values (fastest axis, length Q) -> coefficients (new slowest
// axis, length n1).  out[k][b] = sum_terms sum_q T[q][k] x[b][q]; the input is
// folded on load into x[q] + s x[Q-1-q] (even k) and x[q] - s x[Q-1-q] (odd k).
template <typename T, int TM, int TB, int TK>
__global__ void __launch_bounds__(XT) k_xf_bwd(const __grid_constant__ XfJob<T> job)
{
    if (job.done && *job.done) return;
    const XfOut<T> &O = job.o[blockIdx.z];
    constexpr int RM = TM / 16, RB = TB / 16;
    __shared__ T sTe[TK][TM + 1], sTo[TK][TM + 1];
    __shared__ T sP[TK][TB + 1], sM[TK][TB + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * TM;
    const long long b0 = (long long)blockIdx.y * TB;
    const int Q = job.Q, Qh = job.Qh, KP = job.KP;
    const long long B = job.B;

    T ae[RM][RB], ao[RM][RB];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RB; ++j) ae[i][j] = ao[i][j] = 0.0;

    for (int term = 0; term < O.nterm; ++term) {
        const XfTerm<T> tm = O.t[term];
        const T *TE = job.tabE[tm.tab], *TO = job.tabO[tm.tab];
        const T sg = tm.tab ? T(-1) : T(1);
        for (int q0 = 0; q0 < Qh; q0 += TK) {
            for (int idx = tid; idx < TK * TM; idx += XT) {
                int mm = idx % TM, qq = idx / TM;
                size_t off = (size_t)(q0 + qq) * KP + (m0 + mm);
                sTe[qq][mm] = TE[off];
                sTo[qq][mm] = TO[off];
            }
            for (int idx = tid; idx < TK * TB; idx += XT) {
                int qq = idx % TK, bb = idx / TK;
                int q = q0 + qq, q2 = Q - 1 - q;
                long long b = b0 + bb;
                T v1 = 0, v2 = 0;
                if (q < Qh && b < B) {
                    v1 = tm.x[b * Q + q];
                    if (q2 != q) v2 = tm.x[b * Q + q2];
                }
                sP[qq][bb] = v1 + sg * v2;
                sM[qq][bb] = v1 - sg * v2;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < TK; ++kk) {
                T re[RM], ro[RM], cp[RB], cm[RB];
#pragma unroll
                for (int i = 0; i < RM; ++i) {
                    re[i] = sTe[kk][ty + 16 * i];
                    ro[i] = sTo[kk][ty + 16 * i];
                }
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    cp[j] = sP[kk][tx + 16 * j];
                    cm[j] = sM[kk][tx + 16 * j];
                }
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RB; ++j) {
                        ae[i][j] = fma(re[i], cp[j], ae[i][j]);
                        ao[i][j] = fma(ro[i], cm[j], ao[i][j]);
                    }
            }
            __syncthreads();
        }
    }
    const int n1 = job.n1;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        int m = m0 + ty + 16 * i;
        int ke = 2 * m, ko = 2 * m + 1;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            long long b = b0 + tx + 16 * j;
            if (b >= B) continue;
            if (ke < n1) O.y[(size_t)ke * B + b] = ae[i][j];
            if (ko < n1) O.y[(size_t)ko * B + b] = ao[i][j];
        }
    }
}

template <typename T>
static void job_init_t(XfJob<T> &j, const lsg_ctx *c, const T *tab, long long B, const int *done)
{
    const Geom &g = c->g;
    j.nout = 0;
    j.B = B;
    j.Q = g.Q;
    j.Qh = g.Qh;
    j.n1 = g.n1;
    j.KP = g.KP;
    size_t blk = (size_t)g.QhP * g.KP;
    j.tabE[0] = tab;
    j.tabO[0] = tab + blk;
    j.tabE[1] = tab + 2 * blk;
    j.tabO[1] = tab + 3 * blk;
    j.done = done;
}
static void job_init(XfJob<double> &j, const lsg_ctx *c, long long B, const int *done)
{
    job_init_t<double>(j, c, c->tab, B, done);
}
template <typename T>
struct ident {
    using type = T;
};
template <typename T>
static void add_out(XfJob<T> &j, typename ident<T>::type *y, const typename ident<T>::type *scale,
                    const typename ident<T>::type *x0, int t0, const typename ident<T>::type *x1 = nullptr,
                    int t1 = 0)
{
    XfOut<T> &o = j.o[j.nout++];
    o.y = y;
    o.scale = scale;
    o.nterm = x1 ? 2 : 1;
    o.t[0] = XfTerm<T>{x0, t0};
    o.t[1] = XfTerm<T>{x1, t1};
}

// Tile shapes of the contractions: (rows of the output per CTA, batch columns per
// CTA), 16 x 16 threads each computing (rows/16) x (columns/16) outputs of both
// parity halves.  Which one runs for each contraction of K x is chosen per problem
// size by the autotuner (lsg_autotune_transforms) or taken from its committed table;
// variant -1 is the fixed default.
template <typename T, int TA, int TB>
static void fwd_v(const XfJob<T> &j, cudaStream_t s)
{
    dim3 grid((j.Qh + TA - 1) / TA, (unsigned)((j.B + TB - 1) / TB), j.nout);
    k_xf_fwd<T, TA, TB, 16><<<grid, XT, 0, s>>>(j);
}
template <typename T, int TA, int TB>
static void bwd_v(const XfJob<T> &j, cudaStream_t s)
{
    const int ne = (j.n1 + 1) / 2;
    dim3 grid((ne + TA - 1) / TA, (unsigned)((j.B + TB - 1) / TB), j.nout);
    k_xf_bwd<T, TA, TB, 16><<<grid, XT, 0, s>>>(j);
}
template <typename T>
static int launch_fwd(const XfJob<T> &j, cudaStream_t s, int v = -1)
{
    ::lsg::count_launch();
    switch (v) {
    case 0: fwd_v<T, 16, 16>(j, s); break;
    case 1: fwd_v<T, 16, 32>(j, s); break;
    case 2: fwd_v<T, 32, 32>(j, s); break;
    case 4: fwd_v<T, 64, 32>(j, s); break;
    default: fwd_v<T, 32, 64>(j, s); break;  // variant 3, the default
    }
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}
template <typename T>
static int launch_bwd(const XfJob<T> &j, cudaStream_t s, int v = -1)
{
    if (v < 0) v = j.B >= 2048 ? 3 : 2;  // the default
    ::lsg::count_launch();
    switch (v) {
    case 0: bwd_v<T, 16, 16>(j, s); break;
    case 1: bwd_v<T, 16, 32>(j, s); break;
    case 2: bwd_v<T, 32, 32>(j, s); break;
    case 4: bwd_v<T, 64, 32>(j, s); break;
    default: bwd_v<T, 32, 64>(j, s); break;
    }
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

size_t workspace_elems(const Geom &g)
{
    size_t Q = g.Q, n1 = g.n1;
    if (g.d == 1) return 4 * Q + 2 * n1;
    if (g.d == 2) return 2 * Q * n1 + 3 * Q * Q;
    return 2 * Q * n1 * n1 + 3 * Q * Q * n1 + 4 * Q * Q * Q;
}

// y = K x (Sec. 4.3), every stage on the device.  `done` (optional) makes every
// kernel a no-op once a device-side PCG has converged.
template <typename T>
static int apply_K_t(lsg_ctx *c, const T *x, T *y, const int *done, T *ws, const T *const *Wd, const T *Wb,
                     cudaStream_t s)
{
    const Geom &g = c->g;
    const long long Q = g.Q, n1 = g.n1;
    XfJob<T> j;
    const signed char *vf = c->xf_fwd, *vb = c->xf_bwd;  // tile variant of each contraction
    if (g.d == 1) {
        T *H = ws, *Gx = ws + Q;
        job_init(j, c, 1, done);
        add_out(j, H, Wb, x, 0);
        add_out(j, Gx, Wd[0], x, 1);
        LSG_TRY(launch_fwd(j, s, vf[0]));
        job_init(j, c, 1, done);
        add_out(j, y, nullptr, H, 0, Gx, 1);
        return launch_bwd(j, s, vb[0]);
    }
    if (g.d == 2) {
        T *AP = ws, *AD = ws + Q * n1;           // [Q][n1]
        T *H = ws + 2 * Q * n1, *Gy = H + Q * Q, *Gx = Gy + Q * Q;  // [Q][Q]
        T *P1 = AP, *P2 = AD;                    // [n1][Q] (reuse)
        job_init(j, c, n1, done);                     // contract x: U[j][k]
        add_out(j, AP, nullptr, x, 0);
        add_out(j, AD, nullptr, x, 1);
        LSG_TRY(launch_fwd(j, s, vf[0]));
        job_init(j, c, Q, done);                      // contract y: A[q][j]
        add_out(j, H, Wb, AP, 0);
        add_out(j, Gy, Wd[1], AP, 1);
        add_out(j, Gx, Wd[0], AD, 0);
        LSG_TRY(launch_fwd(j, s, vf[1]));
        job_init(j, c, Q, done);                      // contract x-nodes: [r][q]
        add_out(j, P1, nullptr, H, 0, Gx, 1);
        add_out(j, P2, nullptr, Gy, 0);
        LSG_TRY(launch_bwd(j, s, vb[0]));
        job_init(j, c, n1, done);                     // contract y-nodes: [m][r]
        add_out(j, y, nullptr, P1, 0, P2, 1);
        return launch_bwd(j, s, vb[1]);
    }
    // d == 3
    T *A0 = ws, *A1 = ws + Q * n1 * n1;                       // [Q][n1][n1]
    T *B0 = ws + 2 * Q * n1 * n1, *B1 = B0 + Q * Q * n1, *B2 = B1 + Q * Q * n1;  // [Q][Q][n1]
    T *F0 = B2 + Q * Q * n1, *F1 = F0 + Q * Q * Q, *F2 = F1 + Q * Q * Q, *F3 = F2 + Q * Q * Q;
    T *H = F0, *Gz = F1, *Gy = F2, *Gx = F3;
    job_init(j, c, n1 * n1, done);                 // x: U[l][j][k] -> [q][l][j]
    add_out(j, A0, nullptr, x, 0);
    add_out(j, A1, nullptr, x, 1);
    LSG_TRY(launch_fwd(j, s, vf[0]));
    job_init(j, c, Q * n1, done);                  // y: [q][l][j] -> [r][q][l]
    add_out(j, B0, nullptr, A0, 0);                // phi_x phi_y
    add_out(j, B1, nullptr, A0, 1);                // phi_x phi'_y
    add_out(j, B2, nullptr, A1, 0);                // phi'_x phi_y
    LSG_TRY(launch_fwd(j, s, vf[1]));
    job_init(j, c, Q * Q, done);                   // z: [r][q][l] -> [s][r][q]
    add_out(j, H, Wb, B0, 0);
    add_out(j, Gz, Wd[2], B0, 1);
    add_out(j, Gy, Wd[1], B1, 0);
    add_out(j, Gx, Wd[0], B2, 0);
    LSG_TRY(launch_fwd(j, s, vf[2]));
    T *Pa = B0, *Pb = B1, *Pc = B2;           // [n1][Q][Q] = [m][s][r]
    job_init(j, c, Q * Q, done);
    add_out(j, Pa, nullptr, H, 0, Gx, 1);
    add_out(j, Pb, nullptr, Gy, 0);
    add_out(j, Pc, nullptr, Gz, 0);
    LSG_TRY(launch_bwd(j, s, vb[0]));
    T *Ra = A0, *Rc = A1;                     // [n1][n1][Q] = [n'][m][s]
    job_init(j, c, n1 * Q, done);
    add_out(j, Ra, nullptr, Pa, 0, Pb, 1);
    add_out(j, Rc, nullptr, Pc, 0);
    LSG_TRY(launch_bwd(j, s, vb[1]));
    job_init(j, c, n1 * n1, done);                 // [l'][n'][m]
    add_out(j, y, nullptr, Ra, 0, Rc, 1);
    return launch_bwd(j, s, vb[2]);
}

int apply_K(lsg_ctx *c, const double *x, double *y, const int *done, cudaStream_t s)
{
    const double *Wd[3] = {c->Wa, c->Way, c->Waz};  // W a_j of the j-th gradient term
    return apply_K_t<double>(c, x, y, done, c->ws, Wd, c->Wb, s);
}


__global__ void k_mul(long long n, const double *a, const double *b, double *out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * b[i];
}

// F = sum_grid W f Psi_k: the backward contractions with the phi tables only.
int load_vector(lsg_ctx *c, const double *f, double *F, cudaStream_t s)
{
    const Geom &g = c->g;
    const long long Q = g.Q, n1 = g.n1;
    double *ws = c->ws;
    double *G = ws + workspace_elems(g) - g.nq;  // W f at the end of the workspace
    ::lsg::count_launch();
    k_mul<<<(unsigned)((g.nq + 255) / 256), 256, 0, s>>>(g.nq, c->Wg, f, G);
    LSG_CK(cudaGetLastError());
    XfJob<double> j;
    if (g.d == 1) {
        job_init(j, c, 1, nullptr);
        add_out(j, F, nullptr, G, 0);
        return launch_bwd(j, s);
    }
    if (g.d == 2) {
        double *P = ws;
        job_init(j, c, Q, nullptr);
        add_out(j, P, nullptr, G, 0);
        LSG_TRY(launch_bwd(j, s));
        job_init(j, c, n1, nullptr);
        add_out(j, F, nullptr, P, 0);
        return launch_bwd(j, s);
    }
    double *P = ws, *R = ws + n1 * Q * Q;
    job_init(j, c, Q * Q, nullptr);
    add_out(j, P, nullptr, G, 0);
    LSG_TRY(launch_bwd(j, s));
    job_init(j, c, n1 * Q, nullptr);
    add_out(j, R, nullptr, P, 0);
    LSG_TRY(launch_bwd(j, s));
    job_init(j, c, n1 * n1, nullptr);
    add_out(j, F, nullptr, R, 0);
    return launch_bwd(j, s);
}

// u_N at the grid: the forward contractions with the phi tables only.
int eval_grid(lsg_ctx *c, const double *u, double *vals, cudaStream_t s)
{
    const Geom &g = c->g;
    const long long Q = g.Q, n1 = g.n1;
    double *ws = c->ws;
    XfJob<double> j;
    if (g.d == 1) {
        job_init(j, c, 1, nullptr);
        add_out(j, vals, nullptr, u, 0);
        return launch_fwd(j, s);
    }
    if (g.d == 2) {
        job_init(j, c, n1, nullptr);
        add_out(j, ws, nullptr, u, 0);
        LSG_TRY(launch_fwd(j, s));
        job_init(j, c, Q, nullptr);
        add_out(j, vals, nullptr, ws, 0);
        return launch_fwd(j, s);
    }
    double *A = ws, *Bv = ws + Q * n1 * n1;
    job_init(j, c, n1 * n1, nullptr);
    add_out(j, A, nullptr, u, 0);
    LSG_TRY(launch_fwd(j, s));
    job_init(j, c, Q * n1, nullptr);
    add_out(j, Bv, nullptr, A, 0);
    LSG_TRY(launch_fwd(j, s));
    job_init(j, c, Q * Q, nullptr);
    add_out(j, vals, nullptr, Bv, 0);
    return launch_fwd(j, s);
}

}  // namespace lsg

// ---------------------------------------------------------------------------
// The constant-coefficient preconditioner of PCG-I (Sec. 5): M_0, the operator with
// every coefficient replaced by the constant term of its Legendre series, solved
// directly by fast diagonalisation.  With E the generalised eigenvectors of the 1D
// mass and stiffness matrices (E^T S E = I, E^T M E = Lambda), E (x) E (x) E turns
// M_0 into a diagonal D, so z = (E (x) ..)(D^{-1} o ((E^T (x) ..) r)): d contractions
// with E^T (the last one scaled by 1/D), then d with E.  E couples only indices of
// equal parity, so each contraction is the parity-split MODE 1 of k_xf_fwd.
namespace lsg {

int apply_const_precond(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s)
{
    const Geom &g = c->g;
    const long long n1 = g.n1;
    const size_t blk = (size_t)g.KP * g.KP;
    const double *Et = c->ctab, *E = c->ctab + 2 * blk;  // [even, odd] halves of E^T, then of E
    double *buf[2] = {c->ws, c->ws + g.n};
    const double *in = r;
    int cur = 0;
    for (int pass = 0; pass < 2 * g.d; ++pass) {
        const bool fwd = pass < g.d;
        const bool last = pass == 2 * g.d - 1;
        XfJob<double> j;
        j.nout = 0;
        j.B = g.n / n1;
        j.Q = g.Q;
        j.Qh = (int)((n1 + 1) / 2);
        j.n1 = (int)n1;
        j.KP = g.KP;
        j.tabE[0] = fwd ? Et : E;
        j.tabO[0] = (fwd ? Et : E) + blk;
        j.tabE[1] = j.tabE[0];
        j.tabO[1] = j.tabO[0];
        j.done = done;
        double *out = last ? z : buf[cur];
        add_out(j, out, pass == g.d - 1 ? c->cdinv : nullptr, in, 0);
        dim3 grid((unsigned)((j.Qh + 15) / 16), (unsigned)((j.B + 31) / 32), 1);
        ::lsg::count_launch();
        k_xf_fwd<double, 16, 32, 16, 1><<<grid, XT, 0, s>>>(j);
        LSG_CK(cudaGetLastError());
        in = out;
        cur ^= 1;
    }
    return LSG_OK;
}

}  // namespace lsg

// ---------------------------------------------------------------------------
// Autotuner of the contraction tiles.  K x is d forward and d backward
// contractions whose shapes (output rows x batch columns) depend on N and Q; for
// each one in turn it times K x with every tile variant (the other contractions
// at their current choice), keeps the fastest, and repeats the sweep once.  The
// results for the sizes the workloads use are committed in xf_tiles_gb300.inc
// (written by paper_2004_13961_gb300/autotune.py on a GB300) and applied at
// setup; other sizes keep the default unless the context asks to be tuned.
#include <map>
#include <mutex>
#include <tuple>

namespace lsg {

namespace {
struct TileRow {
    int d, N, Q;
    signed char f[3], b[3];
};
const TileRow kTileTable[] = {
#include "xf_tiles_gb300.inc"
    {0, 0, 0, {-1, -1, -1}, {-1, -1, -1}}};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TileRow> g_tuned;  // sizes tuned in this process
}  // namespace

bool tile_table_lookup(lsg_ctx *c)
{
    const Geom &g = c->g;
    auto apply = [&](const TileRow &r) {
        for (int i = 0; i < 3; ++i) c->xf_fwd[i] = r.f[i], c->xf_bwd[i] = r.b[i];
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(std::make_tuple(g.d, g.N, g.Q));
        if (it != g_tuned.end()) {
            apply(it->second);
            return true;
        }
    }
    for (const TileRow &r : kTileTable)
        if (r.d == g.d && r.N == g.N && r.Q == g.Q) {
            apply(r);
            return true;
        }
    return false;
}

int autotune_transforms(lsg_ctx *c, int reps, cudaStream_t s)
{
    const Geom &g = c->g;
    if (reps < 1) reps = 5;
    double *x = c->xs, *y = c->ys;
    LSG_CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)g.n, s));
    cudaEvent_t e0, e1;
    LSG_CK(cudaEventCreate(&e0));
    LSG_CK(cudaEventCreate(&e1));
    auto time_kx = [&](float *ms) -> int {
        LSG_TRY(apply_K(c, x, y, nullptr, s));  // warm-up
        LSG_CK(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) LSG_TRY(apply_K(c, x, y, nullptr, s));
        LSG_CK(cudaEventRecord(e1, s));
        LSG_CK(cudaEventSynchronize(e1));
        LSG_CK(cudaEventElapsedTime(ms, e0, e1));
        return LSG_OK;
    };
    int st = LSG_OK;
    for (int pass = 0; pass < 2 && st == LSG_OK; ++pass)
        for (int k = 0; k < 2 * g.d && st == LSG_OK; ++k) {
            signed char *slot = k < g.d ? &c->xf_fwd[k] : &c->xf_bwd[k - g.d];
            signed char best = *slot;
            float tbest = 0.f;
            st = time_kx(&tbest);
            for (int v = 0; v < 5 && st == LSG_OK; ++v) {
                *slot = (signed char)v;
                float t = 0.f;
                st = time_kx(&t);
                if (st == LSG_OK && t < tbest) tbest = t, best = (signed char)v;
            }
            *slot = best;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LSG_OK) return st;
    TileRow r{g.d, g.N, g.Q, {c->xf_fwd[0], c->xf_fwd[1], c->xf_fwd[2]}, {c->xf_bwd[0], c->xf_bwd[1], c->xf_bwd[2]}};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(g.d, g.N, g.Q)] = r;
    return LSG_OK;
}

}  // namespace lsg
