// constprec.cu -- setup of the constant-coefficient preconditioner of PCG-I, the
// paper's comparison method (Sec. 5: "PCG with a constant-coefficient
// preconditioner", the rows t_1 = 0, t_2 = 0 of Tables 5.7-5.11, whose systems are
// solved by direct methods in each iteration).
//
// M_0 is the preconditioner M of Sec. 4.1 with every truncation degree 0: each
// diffusion coefficient a_j and the reaction coefficient b replaced by the constant
// term of its Legendre series, abar_j = ahat_j[0], bbar = bhat[0].  In Kronecker
// form (Sec. 4.2) with the 1D stiffness S = S^(0) = diag(4k+6) and mass M = M^(0):
//   M_0 = sum_j abar_j (M (x) .. S in direction j .. (x) M) + bbar (M (x) .. (x) M).
// The generalised eigenproblem M e = lambda S e is solved on the device: S is
// diagonal, so A = S^{-1/2} M S^{-1/2} is symmetric, and M^(0) couples only indices of
// equal parity, so A splits into two symmetric tridiagonal matrices (even and odd
// indices).  One thread per eigenpair: the eigenvalue by bisection on the Sturm
// count, the eigenvector by inverse iteration with a partially pivoted tridiagonal
// elimination.  E = S^{-1/2} Y then gives E^T S E = I, E^T M E = Lambda, and
//   (E (x) E (x) E)^T M_0 (E (x) E (x) E) = D,
//   D[l][j][i] = abar_x lam_j lam_l + abar_y lam_i lam_l + abar_z lam_i lam_j + bbar lam_i lam_j lam_l
// (2D: abar_x lam_j + abar_y lam_i + bbar lam_i lam_j; 1D: abar + bbar lam_i).  The
// apply (transform.cu, apply_const_precond) is then 2d dense contractions and a
// pointwise division.
#include <math.h>

#include <algorithm>

#include "lsg_internal.cuh"

namespace lsg {

// Sturm count of the symmetric tridiagonal (a, e^2): eigenvalues below x.
__device__ int sturm_below(int m, const double *a, const double *e2, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (int k = 0; k < m; ++k) {
        q = a[k] - x - (k > 0 ? e2[k - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Parity block p of A: a[k] = M[i][i] / S_i, e[k] = M[i][i+2] / sqrt(S_i S_{i+2}),
// i = 2k + p.  Band arrays: bandM[t=0][i][o + w], o = -w..w.
__global__ void k_const_blocks(int n1, int w, int W1, const double *bandM, double *a, double *e, double *e2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1) return;
    const int p = i & 1, k = i >> 1, half = (n1 + 1) / 2;
    const double Si = 4.0 * i + 6.0;
    a[p * half + k] = bandM[(size_t)i * W1 + w] / Si;
    if (i + 2 < n1) {
        const double Sj = 4.0 * (i + 2) + 6.0;
        const double v = bandM[(size_t)i * W1 + w + 2] / sqrt(Si * Sj);
        e[p * half + k] = v;
        e2[p * half + k] = v * v;
    } else {
        e[p * half + k] = 0.0;
        e2[p * half + k] = 0.0;
    }
}

// One thread per eigenpair (parity p, index k in ascending order of the block's
// eigenvalues).  Writes lam[2k+p] and the eigenvector's tables: the parity blocks of
// E^T (rows: eigen index, columns: basis index) and of E (the transposes), each
// KP x KP with zero padding, E = S^{-1/2} Y.  scratch: 5 ceil(n1/2) doubles per thread.
__global__ void k_const_eig(int n1, int KP, const double *a, const double *e, const double *e2, double *lam,
                            double *tab, double *scratch, int *err)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = (n1 + 1) / 2;
    if (t >= n1) return;
    const int p = t & 1, k = t >> 1;
    const int m = p == 0 ? half : n1 / 2;
    if (k >= m) return;
    const double *A = a + p * half, *Ee = e + p * half, *E2 = e2 + p * half;
    // Gershgorin interval
    double lo = 1e300, hi = -1e300;
    for (int r = 0; r < m; ++r) {
        const double rad = (r > 0 ? fabs(Ee[r - 1]) : 0.0) + (r + 1 < m ? fabs(Ee[r]) : 0.0);
        lo = fmin(lo, A[r] - rad);
        hi = fmax(hi, A[r] + rad);
    }
    // bisection for the k-th smallest eigenvalue
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(m, A, E2, mid) > k) hi = mid;
        else lo = mid;
    }
    const double lamk = 0.5 * (lo + hi);
    lam[2 * k + p] = lamk;
    // inverse iteration: (A - lam) y = v, partial pivoting on the tridiagonal
    // per-thread scratch at a fixed stride (the two parity blocks differ in size when n1 is odd)
    double *dl = scratch + (size_t)t * 5 * half, *dd = dl + m, *du = dd + m, *du2 = du + m, *y = du2 + m;
    const double shift = lamk + 1e-15 * fmax(fabs(lamk), 1e-300);
    for (int r = 0; r < m; ++r) y[r] = 1.0 + 0.01 * (double)((r * 7 + k * 3) % 11);
    for (int iter = 0; iter < 3; ++iter) {
        for (int r = 0; r < m; ++r) {
            dd[r] = A[r] - shift;
            du[r] = r + 1 < m ? Ee[r] : 0.0;
            dl[r] = r + 1 < m ? Ee[r] : 0.0;  // sub-diagonal entry (r+1, r)
            du2[r] = 0.0;
        }
        // elimination: rows r and r+1, pivot on the larger of dd[r] and dl[r]
        for (int r = 0; r + 1 < m; ++r) {
            if (fabs(dd[r]) >= fabs(dl[r])) {
                const double f = dl[r] / (dd[r] != 0.0 ? dd[r] : 1e-300);
                dd[r + 1] -= f * du[r];
                y[r + 1] -= f * y[r];
                dl[r] = 0.0;
            } else {
                // swap rows r and r+1
                const double f = dd[r] / dl[r];
                const double d1 = dl[r], u1 = dd[r + 1], u2 = r + 2 < m ? du[r + 1] : 0.0;
                const double yr = y[r];
                dd[r] = d1;
                const double old_du = du[r];
                du[r] = u1;
                du2[r] = u2;
                dd[r + 1] = old_du - f * u1;
                if (r + 2 < m) du[r + 1] = -f * u2;
                y[r] = y[r + 1];
                y[r + 1] = yr - f * y[r];
                dl[r] = 0.0;
            }
        }
        // back substitution
        for (int r = m - 1; r >= 0; --r) {
            double v = y[r];
            if (r + 1 < m) v -= du[r] * y[r + 1];
            if (r + 2 < m) v -= du2[r] * y[r + 2];
            const double piv = dd[r] != 0.0 ? dd[r] : 1e-300;
            y[r] = v / piv;
        }
        double nrm = 0.0;
        for (int r = 0; r < m; ++r) nrm += y[r] * y[r];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            set_err(err, DERR_NONFINITE);
            return;
        }
        for (int r = 0; r < m; ++r) y[r] /= nrm;
    }
    // a consistent sign: the first entry of largest magnitude positive
    int rmax = 0;
    for (int r = 1; r < m; ++r)
        if (fabs(y[r]) > fabs(y[rmax])) rmax = r;
    const double sg = y[rmax] < 0.0 ? -1.0 : 1.0;
    const size_t blk = (size_t)KP * KP;
    double *Et = tab + (size_t)p * blk, *Ev = tab + 2 * blk + (size_t)p * blk;
    for (int r = 0; r < m; ++r) {
        const int i = 2 * r + p;
        const double v = sg * y[r] / sqrt(4.0 * i + 6.0);
        Et[(size_t)k * KP + r] = v;  // E^T: row = eigen index, column = basis index
        Ev[(size_t)r * KP + k] = v;  // E
    }
}

// 1 / D at every index (i fastest), from the eigenvalues and the constant terms.
__global__ void k_const_dinv(int d, int n1, long long n, const double *lam, const double *ahx, const double *ahy,
                             const double *ahz, const double *bhat, int has_b, double *dinv, int *err)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int i = (int)(r % n1), j = d >= 2 ? (int)((r / n1) % n1) : 0, l = d == 3 ? (int)(r / ((long long)n1 * n1)) : 0;
    const double li = lam[i], lj = d >= 2 ? lam[j] : 1.0, ll = d == 3 ? lam[l] : 1.0;
    const double ax = ahx[0], ay = ahy[0], az = ahz[0], bb = has_b ? bhat[0] : 0.0;
    double D;
    if (d == 1) D = ax + bb * li;
    else if (d == 2) D = ax * lj + ay * li + bb * li * lj;
    else D = ax * lj * ll + ay * li * ll + az * li * lj + bb * li * lj * ll;
    if (!(D > 0.0)) set_err(err, DERR_BREAKDOWN);
    dinv[r] = 1.0 / D;
}

int build_const_preconditioner(lsg_ctx *c, cudaStream_t s)
{
    const Geom &g = c->g;
    const int n1 = g.n1, half = (n1 + 1) / 2;
    double *a = nullptr, *e = nullptr, *e2 = nullptr, *scr = nullptr;
    LSG_CK(cudaMallocAsync((void **)&a, sizeof(double) * 2 * half, s));
    LSG_CK(cudaMallocAsync((void **)&e, sizeof(double) * 2 * half, s));
    LSG_CK(cudaMallocAsync((void **)&e2, sizeof(double) * 2 * half, s));
    LSG_CK(cudaMallocAsync((void **)&scr, sizeof(double) * (size_t)n1 * 5 * half, s));
    LSG_CK(cudaMemsetAsync(c->ctab, 0, sizeof(double) * 4 * (size_t)g.KP * g.KP, s));
    ::lsg::count_launch();
    k_const_blocks<<<(n1 + 127) / 128, 128, 0, s>>>(n1, g.w, g.W1, c->bandM, a, e, e2);
    ::lsg::count_launch();
    k_const_eig<<<(n1 + 63) / 64, 64, 0, s>>>(n1, g.KP, a, e, e2, c->clam, c->ctab, scr, c->err);
    ::lsg::count_launch();
    k_const_dinv<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g.d, n1, g.n, c->clam, c->ahat, c->ahaty, c->ahatz,
                                                               c->bhat, g.has_b, c->cdinv, c->err);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaFreeAsync(a, s));
    LSG_CK(cudaFreeAsync(e, s));
    LSG_CK(cudaFreeAsync(e2, s));
    LSG_CK(cudaFreeAsync(scr, s));
    return LSG_OK;
}

}  // namespace lsg
