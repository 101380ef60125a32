// tables.cu -- setup tables on the device: the Legendre-Gauss rule (Sec. 2.2),
// the parity-folded basis tables used by the transforms (Sec. 4.3), the
// weighted coefficient samples, the truncated coefficient series a_hat, b_hat
// (Sec. 4.1) and the 1D band matrices S^(t), M^(t) of the Kronecker form of M
// (Sec. 4.2).
#include <math.h>

#include <algorithm>

#include "lsg_internal.cuh"

namespace lsg {

Geom make_geom(int d, int N, int T, int Q)
{
    int ta[3][3], tb[3];
    for (int j = 0; j < 3; ++j) {
        tb[j] = T;
        for (int i = 0; i < 3; ++i) ta[j][i] = T;
    }
    return make_geom_dir(d, N, ta, tb, Q);
}

// Degrees per coefficient and direction (Sec. 4.1's t_1 for a and t_2 for b; Sec. 5
// Example 4's t_1j for a_j): T is the largest degree (the size of the series and
// band tables), w the half-width of the offset box that holds every band of the
// pattern: a stiffness band reaches its degree, a mass band its degree + 2.
Geom make_geom_dir(int d, int N, const int ta[3][3], const int tb[3], int Q)
{
    Geom g{};
    g.d = d;
    g.N = N;
    g.n1 = N - 1;
    g.Q = Q;
    g.Qh = (Q + 1) / 2;
    g.T = 0;
    g.w = 0;
    for (int j = 0; j < 3; ++j) {
        g.tb[j] = j < d ? tb[j] : 0;
        for (int i = 0; i < 3; ++i) g.ta[j][i] = (i < d && j < d) ? ta[j][i] : 0;
    }
    for (int i = 0; i < d; ++i) {
        g.T = std::max(g.T, g.tb[i]);
        g.w = std::max(g.w, g.tb[i] + 2);
        for (int j = 0; j < d; ++j) {
            g.T = std::max(g.T, g.ta[j][i]);
            g.w = std::max(g.w, i == j ? g.ta[j][i] : g.ta[j][i] + 2);
        }
    }
    g.W1 = 2 * g.w + 1;
    g.S = 1;
    for (int i = 0; i < d; ++i) g.S *= g.W1;
    g.Sc = (g.S - 1) / 2;
    g.SL = (g.Sc + 7) / 8 * 8;        // 32-byte aligned rows in FP32, 64 in FP64
    g.SU = (g.Sc + 2 + 7) / 8 * 8;    // diagonal, Sc upper slots, and a pad slot holding 1 / U_ii
    g.ne = (g.n1 + 1) / 2;
    g.no = g.n1 / 2;
    g.KP = (g.ne + 63) / 64 * 64;
    g.QhP = (g.Qh + 63) / 64 * 64;
    g.n = 1;
    g.nq = 1;
    for (int i = 0; i < d; ++i) {
        g.n *= g.n1;
        g.nq *= Q;
    }
    g.nlines = g.n / g.n1;
    long long lv = 0, p = 1;
    for (int a = 0; a < d; ++a) {
        lv += p;
        p *= (g.w + 1);
    }
    g.levels = (int)((g.n1 - 1) * lv + 1);
    g.has_b = 1;
    return g;
}

// ---------------------------------------------------------------------------
// Legendre-Gauss rule: Newton on L_Q evaluated by the three-term recurrence
// (Sec. 2.1), one thread per node pair (x, -x).  Weight 2/((1-x^2) L'_Q(x)^2)
// with (1-x^2) L'_Q = Q (L_{Q-1} - x L_Q), i.e. w = 2 (1-x)(1+x) / (Q (L_{Q-1} - x L_Q))^2;
// keeping the x L_Q term matters near the ends, where L_Q(x) at the rounded root
// is not negligible against L_{Q-1}(x).
__device__ static void leg_top2(int Q, double x, double &LQ, double &LQm1)
{
    double p0 = 1.0, p1 = x;
    if (Q == 0) {
        LQ = 1.0;
        LQm1 = 0.0;
        return;
    }
    for (int k = 1; k < Q; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - (double)k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    LQ = p1;
    LQm1 = p0;
}

__global__ void k_gauss(int Q, double *x, double *w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int Qh = (Q + 1) / 2;
    if (i >= Qh) return;
    double xi = -cos(M_PI * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
    double LQ, LQm1;
    bool mid = (Q & 1) && (i == Qh - 1);
    if (mid) {
        xi = 0.0;
    } else {
        for (int it = 0; it < 100; ++it) {
            leg_top2(Q, xi, LQ, LQm1);
            double dL = Q * (xi * LQ - LQm1) / (xi * xi - 1.0);
            double dx = LQ / dL;
            xi -= dx;
            if (fabs(dx) < 1e-16) {
                leg_top2(Q, xi, LQ, LQm1);
                dL = Q * (xi * LQ - LQm1) / (xi * xi - 1.0);
                xi -= LQ / dL;
                break;
            }
        }
    }
    leg_top2(Q, xi, LQ, LQm1);
    double den = Q * (LQm1 - xi * LQ);
    double wi = 2.0 * (1.0 - xi) * (1.0 + xi) / (den * den);
    x[i] = xi;
    x[Q - 1 - i] = -xi;
    w[i] = wi;
    w[Q - 1 - i] = wi;
}

// Folded basis tables.  For node q < Qh (x_q <= 0) and pair index m:
//   phiE[q][m] = phi_{2m}(x_q),   phiO[q][m] = phi_{2m+1}(x_q),
//   dE[q][m]   = phi'_{2m}(x_q),  dO[q][m]   = phi'_{2m+1}(x_q),
// with phi_k = L_k - L_{k+2} and phi'_k = -(2k+3) L_{k+1} (Sec. 3 and the
// derivative recurrence of Sec. 2.1).  Padding rows/columns are zero.
__global__ void k_tables(int Q, int n1, int QhP, int KP, const double *x, double *tab)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= QhP) return;
    int Qh = (Q + 1) / 2;
    size_t blk = (size_t)QhP * KP;
    double *pE = tab, *pO = tab + blk, *dE = tab + 2 * blk, *dO = tab + 3 * blk;
    size_t row = (size_t)q * KP;
    if (q >= Qh) {
        for (int m = 0; m < KP; ++m) {
            pE[row + m] = pO[row + m] = dE[row + m] = dO[row + m] = 0.0;
        }
        return;
    }
    double xq = x[q];
    // running window L_{k}, L_{k+1}, L_{k+2}
    double L0 = 1.0, L1 = xq;
    // L at degree k (a), k+1 (b), k+2 (c)
    double a = L0, b = L1;
    double c = (Q > 0) ? (3.0 * xq * L1 - 1.0 * L0) / 2.0 : 0.0;
    for (int k = 0; k < 2 * KP; ++k) {
        double phi = 0.0, dphi = 0.0;
        if (k < n1) {
            phi = a - c;
            dphi = -(2.0 * k + 3.0) * b;
        }
        int m = k >> 1;
        if (k & 1) {
            pO[row + m] = phi;
            dO[row + m] = dphi;
        } else {
            pE[row + m] = phi;
            dE[row + m] = dphi;
        }
        // advance: degree k+3 from k+2 (c) and k+1 (b)
        double nk = k + 2.0;
        double dnext = ((2.0 * nk + 1.0) * xq * c - nk * b) / (nk + 1.0);
        a = b;
        b = c;
        c = dnext;
    }
}

// Wa = W a, Wb = W b, Wg = W with W the tensor product of Gauss weights.
__global__ void k_weighted(int d, int Q, long long nq, const double *w, const double *a,
                           const double *b, double *Wa, double *Wb, double *Wg, int *err)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= nq) return;
    long long rem = g;
    double W = 1.0;
    for (int ax = 0; ax < d; ++ax) {
        W *= w[rem % Q];
        rem /= Q;
    }
    double av = a[g], bv = b[g];
    if (!isfinite(av) || !isfinite(bv)) set_err(err, DERR_NONFINITE);
    Wa[g] = W * av;
    Wb[g] = W * bv;
    Wg[g] = W;
}

// Wd = W c for a further diffusion coefficient (one per direction).
__global__ void k_weighted_dir(int d, int Q, long long nq, const double *w, const double *c, double *Wd, int *err)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= nq) return;
    long long rem = g;
    double W = 1.0;
    for (int ax = 0; ax < d; ++ax) {
        W *= w[rem % Q];
        rem /= Q;
    }
    const double v = c[g];
    if (!isfinite(v)) set_err(err, DERR_NONFINITE);
    Wd[g] = W * v;
}

__global__ void k_to_float(long long n, const double *a, float *b)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g < n) b[g] = (float)a[g];
}

__global__ void k_any_nonzero(long long n, const double *v, int *flag)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g < n && v[g] != 0.0) atomicOr(flag, 1);
}

// Lw[t][q] = w_q L_t(x_q), t <= T.
__global__ void k_lw(int Q, int T, const double *x, const double *w, double *Lw)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    double xq = x[q], p0 = 1.0, p1 = xq;
    for (int t = 0; t <= T; ++t) {
        double v = (t == 0) ? p0 : p1;
        Lw[(size_t)t * Q + q] = w[q] * v;
        if (t >= 1) {
            double p2 = ((2.0 * t + 1.0) * xq * p1 - (double)t * p0) / (t + 1.0);
            p0 = p1;
            p1 = p2;
        }
    }
}

// out[t][r] = sum_q Lw[t][q] in[r][q]: contract the fastest axis, new axis slowest.
__global__ void k_contract_lw(long long R, int Q, int T1, const double *in, const double *Lw,
                              double *out)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= R * T1) return;
    long long r = idx % R;
    int t = (int)(idx / R);
    const double *row = in + r * Q;
    const double *lt = Lw + (size_t)t * Q;
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += lt[q] * row[q];
    out[(size_t)t * R + r] = s;
}

// The (2t+1)/2 factors of the discrete Legendre transform; terms of degree above
// the series' degree in some direction are dropped (the truncation, per direction).
__global__ void k_scale_series(int d, int T1, int deg0, int deg1, int deg2, double *chat)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int tot = 1;
    for (int i = 0; i < d; ++i) tot *= T1;
    if (idx >= tot) return;
    const int deg[3] = {deg0, deg1, deg2};
    int rem = idx;
    double f = 1.0;
    for (int ax = 0; ax < d; ++ax) {
        int t = rem % T1;
        rem /= T1;
        f *= (2.0 * t + 1.0) * 0.5;
        if (t > deg[ax]) f = 0.0;
    }
    chat[idx] *= f;
}

// LQ[q][m] = L_m(xq[q]), m <= mmax.
__global__ void k_leg_table(int QM, int mmax, const double *x, double *LQ)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= QM) return;
    double xq = x[q], p0 = 1.0, p1 = xq;
    double *row = LQ + (size_t)q * (mmax + 1);
    row[0] = 1.0;
    if (mmax >= 1) row[1] = xq;
    for (int m = 1; m < mmax; ++m) {
        double p2 = ((2.0 * m + 1.0) * xq * p1 - (double)m * p0) / (m + 1.0);
        row[m + 1] = p2;
        p0 = p1;
        p1 = p2;
    }
}

// Band matrices by QM-point Gauss quadrature (exact: integrand degree <= 2N+T):
//   S[t][i][o] = (L_t phi'_i, phi'_{i+o}), M[t][i][o] = (L_t phi_i, phi_{i+o}),
// o = -w..w stored at o+w.  Entries that Proposition 4.1's parity and width
// rules make zero (S: |o| > t or o+t odd; M: |o| > t+2 or o+t odd) are exact 0.
__global__ void k_band(int n1, int T, int w, int QM, int mmax, const double *xw, const double *LQ,
                       double *S, double *M)
{
    int W1 = 2 * w + 1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)(T + 1) * n1 * W1;
    if (idx >= tot) return;
    int oi = (int)(idx % W1);
    int i = (int)((idx / W1) % n1);
    int t = (int)(idx / ((long long)W1 * n1));
    int o = oi - w;
    int m = i + o;
    double sv = 0.0, mv = 0.0;
    bool inr = (m >= 0 && m < n1);
    bool par = ((o + t) & 1) == 0;
    bool sOn = inr && par && abs(o) <= t;
    bool mOn = inr && par && abs(o) <= t + 2;
    if (sOn || mOn) {
        double ci = -(2.0 * i + 3.0), cm = -(2.0 * m + 3.0);
        for (int q = 0; q < QM; ++q) {
            const double *L = LQ + (size_t)q * (mmax + 1);
            double wl = xw[q] * L[t];
            if (sOn) sv += wl * (ci * L[i + 1]) * (cm * L[m + 1]);
            if (mOn) mv += wl * (L[i] - L[i + 2]) * (L[m] - L[m + 2]);
        }
    }
    S[idx] = sv;
    M[idx] = mv;
}

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int gauss_rule(int Q, double *x, double *w, cudaStream_t s)
{
    ::lsg::count_launch();
    k_gauss<<<blocks_for((Q + 1) / 2, 128), 128, 0, s>>>(Q, x, w);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaStreamSynchronize(s));
    return LSG_OK;
}

// Build every table a context needs before the preconditioner: Gauss rule,
// folded basis tables, weighted samples, a_hat, b_hat and the band matrices.
int build_tables(lsg_ctx *c, const double *const *a_dir, const double *b_dev, cudaStream_t s)
{
    const double *a_dev = a_dir[0];
    const Geom &g = c->g;
    ::lsg::count_launch();
    k_gauss<<<blocks_for(g.Qh, 128), 128, 0, s>>>(g.Q, c->gx, c->gw);
    LSG_CK(cudaGetLastError());
    ::lsg::count_launch();
    k_tables<<<blocks_for(g.QhP, 64), 64, 0, s>>>(g.Q, g.n1, g.QhP, g.KP, c->gx, c->tab);
    LSG_CK(cudaGetLastError());
    ::lsg::count_launch();
    k_weighted<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.d, g.Q, g.nq, c->gw, a_dev, b_dev, c->Wa, c->Wb,
                                                      c->Wg, c->err);
    LSG_CK(cudaGetLastError());

    // one diffusion coefficient per direction: the others' weighted samples
    if (c->own_ay) {
        ::lsg::count_launch();
        k_weighted_dir<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.d, g.Q, g.nq, c->gw, a_dir[1], c->Way, c->err);
    }
    if (c->own_az) {
        ::lsg::count_launch();
        k_weighted_dir<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.d, g.Q, g.nq, c->gw, a_dir[2], c->Waz, c->err);
    }
    LSG_CK(cudaGetLastError());
    if (c->Wa32) {
        ::lsg::count_launch();
        k_to_float<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.nq, c->Wa, c->Wa32);
        ::lsg::count_launch();
        k_to_float<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.nq, c->Wb, c->Wb32);
        if (c->own_ay) {
            ::lsg::count_launch();
            k_to_float<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.nq, c->Way, c->Wa32y);
        }
        if (c->own_az) {
            ::lsg::count_launch();
            k_to_float<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.nq, c->Waz, c->Wa32z);
        }
        LSG_CK(cudaGetLastError());
    }
    // has_b: any nonzero b sample
    int *flag = nullptr;
    LSG_CK(cudaMallocAsync((void **)&flag, sizeof(int), s));
    LSG_CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    ::lsg::count_launch();
    k_any_nonzero<<<blocks_for(g.nq, 256), 256, 0, s>>>(g.nq, b_dev, flag);
    int hb = 0;
    LSG_CK(cudaMemcpyAsync(&hb, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSG_CK(cudaFreeAsync(flag, s));

    // truncated series: contract each axis with w_q L_t(x_q), then (2t+1)/2 factors
    int T1 = g.T + 1;
    double *Lw = nullptr, *t0 = nullptr, *t1 = nullptr;
    size_t big = (size_t)T1 * (size_t)std::max<long long>(g.nq / g.Q, 1);
    LSG_CK(cudaMallocAsync((void **)&Lw, sizeof(double) * T1 * g.Q, s));
    LSG_CK(cudaMallocAsync((void **)&t0, sizeof(double) * big, s));
    LSG_CK(cudaMallocAsync((void **)&t1, sizeof(double) * big, s));
    ::lsg::count_launch();
    k_lw<<<blocks_for(g.Q, 128), 128, 0, s>>>(g.Q, g.T, c->gx, c->gw, Lw);
    // series of b, a_x, and (when they are separate) a_y, a_z, each with its degrees
    for (int which = 0; which < 4; ++which) {
        const double *src = which == 0 ? b_dev : a_dir[which - 1];
        double *dst = which == 0 ? c->bhat : which == 1 ? c->ahat : which == 2 ? c->ahaty : c->ahatz;
        const int *deg = which == 0 ? g.tb : g.ta[which - 1];
        if (which >= 1 && which - 1 >= g.d) break;
        if (which == 2 && dst == c->ahat) continue;  // the same series as a_x
        if (which == 3 && (dst == c->ahat || dst == c->ahaty)) continue;
        long long R = g.nq / g.Q;  // rows of the current [R][Q] view
        const double *in = src;
        double *bufs[2] = {t0, t1};
        int cur = 0;
        for (int ax = 0; ax < g.d; ++ax) {
            double *out = (ax == g.d - 1) ? dst : bufs[cur];
            ::lsg::count_launch();
            k_contract_lw<<<blocks_for(R * T1, 128), 128, 0, s>>>(R, g.Q, T1, in, Lw, out);
            LSG_CK(cudaGetLastError());
            in = out;
            cur ^= 1;
            // next view: [T1 * R / Q][Q]
            R = (long long)T1 * R / g.Q;
        }
        ::lsg::count_launch();
        k_scale_series<<<blocks_for(g.d == 1 ? T1 : g.d == 2 ? T1 * T1 : T1 * T1 * T1, 128), 128, 0, s>>>(
            g.d, T1, deg[0], deg[1], deg[2], dst);
        LSG_CK(cudaGetLastError());
    }
    LSG_CK(cudaFreeAsync(Lw, s));
    LSG_CK(cudaFreeAsync(t0, s));
    LSG_CK(cudaFreeAsync(t1, s));

    // band matrices with their own QM-point rule
    int QM = g.N + (g.T + 1) / 2 + 2;
    int mmax = std::max(g.N + 1, g.T);
    double *xm = nullptr, *wm = nullptr, *LQ = nullptr;
    LSG_CK(cudaMallocAsync((void **)&xm, sizeof(double) * QM, s));
    LSG_CK(cudaMallocAsync((void **)&wm, sizeof(double) * QM, s));
    LSG_CK(cudaMallocAsync((void **)&LQ, sizeof(double) * (size_t)QM * (mmax + 1), s));
    ::lsg::count_launch();
    k_gauss<<<blocks_for((QM + 1) / 2, 128), 128, 0, s>>>(QM, xm, wm);
    ::lsg::count_launch();
    k_leg_table<<<blocks_for(QM, 64), 64, 0, s>>>(QM, mmax, xm, LQ);
    long long nb = (long long)T1 * g.n1 * g.W1;
    ::lsg::count_launch();
    k_band<<<blocks_for(nb, 128), 128, 0, s>>>(g.n1, g.T, g.w, QM, mmax, wm, LQ, c->bandS, c->bandM);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaFreeAsync(xm, s));
    LSG_CK(cudaFreeAsync(wm, s));
    LSG_CK(cudaFreeAsync(LQ, s));
    LSG_CK(cudaStreamSynchronize(s));
    c->g.has_b = hb;
    return LSG_OK;
}

}  // namespace lsg
