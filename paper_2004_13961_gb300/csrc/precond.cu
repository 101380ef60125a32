// precond.cu -- the preconditioner M of Sec. 4.1/4.2 on the device: assembly of
// M from the truncated series and band matrices (Kronecker form), its ILU(0)
// factorisation in natural order (Algorithm 2) and the forward / backward
// substitutions (Algorithms 3 and 4).
//
// Storage: M and its factors live in a stencil layout.  Row r = (i, j, k)
// (i fastest) has S = (2w+1)^d slots, one per offset (dx, dy, dz) in the box
// |d*| <= w = T+2, ordered lexicographically with dx fastest, so slot order is
// column order.  Slots s < Sc (strictly lower) are stored in Lv[r][s], slots
// s >= Sc (diagonal, then strictly upper) in Uv[r][s - Sc]; rows are padded to
// SL / SU entries.  Slots outside the grid or outside the structural pattern
// hold 0 and are never updated.
#include <math.h>

#include <algorithm>

#include "lsg_internal.cuh"
#include "stencil.cuh"

namespace lsg {

// ---------------------------------------------------------------------------
// M assembly.  With band matrices S^(t)[i][o], M^(t)[i][o] (o = column - row),
// `2DM` in Kronecker form (Sec. 4.2) gives for row (i,j), offset (ox,oy):
//   M = sum_k [ M^(k)[j][oy] X1[k][i][ox] + S^(k)[j][oy] X2[k][i][ox] ],
//   X1[k][i][ox] = sum_t (a_tk S^(t)[i][ox] + b_tk M^(t)[i][ox]),
//   X2[k][i][ox] = sum_t a_tk M^(t)[i][ox]          (t: x degree, k: y degree)
// and `3DM` similarly with a second contraction over the z degree.
__global__ void k_precontract(int d, int T, int n1, int W1, const double *ahat, const double *bhat,
                              int has_b, const double *bS, const double *bM, double *X1, double *X2)
{
    // X[K][i][o] with K = (k) in 2D or (k,l) in 3D, (T+1)^(d-1) values of K
    int T1 = T + 1;
    long long nK = (d == 3) ? (long long)T1 * T1 : T1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long tot = nK * n1 * W1;
    if (idx >= tot) return;
    int o = (int)(idx % W1);
    int i = (int)((idx / W1) % n1);
    long long K = idx / ((long long)W1 * n1);
    double x1 = 0.0, x2 = 0.0;
    for (int t = 0; t < T1; ++t) {
        double at = ahat[K * T1 + t], bt = bhat[K * T1 + t];
        double s = bS[((size_t)t * n1 + i) * W1 + o], m = bM[((size_t)t * n1 + i) * W1 + o];
        x1 += at * s + (has_b ? bt * m : 0.0);
        x2 += at * m;
    }
    X1[idx] = x1;
    X2[idx] = x2;
}

template <typename V>
__global__ void k_assemble(StencilGeo G, const double *ahat, const double *bhat, const double *bS,
                           const double *bM, const double *X1, const double *X2, V *Lv, V *Uv,
                           double *Mkeep)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= G.n * G.S) return;
    int s = (int)(idx % G.S);
    long long r = idx / G.S;
    int i = (int)(r % G.n1);
    int j = (G.d >= 2) ? (int)((r / G.n1) % G.n1) : 0;
    int k = (G.d == 3) ? (int)(r / ((long long)G.n1 * G.n1)) : 0;
    int dx, dy, dz;
    slot_offsets(G, s, dx, dy, dz);
    int ci = i + dx, cj = j + dy, ck = k + dz;
    double v = 0.0;
    bool ingrid = ci >= 0 && ci < G.n1 && cj >= 0 && cj < G.n1 && ck >= 0 && ck < G.n1;
    if (ingrid && structural(G, dx, dy, dz)) {
        int T1 = G.T + 1, W1 = G.W1, n1 = G.n1, w = G.w;
        if (G.d == 1) {
            for (int t = 0; t < T1; ++t) {
                size_t bi = ((size_t)t * n1 + i) * W1 + dx + w;
                v += ahat[t] * bS[bi] + (G.has_b ? bhat[t] * bM[bi] : 0.0);
            }
        } else if (G.d == 2) {
            for (int kk = 0; kk < T1; ++kk) {
                size_t by = ((size_t)kk * n1 + j) * W1 + dy + w;
                size_t bx = ((size_t)kk * n1 + i) * W1 + dx + w;
                v += bM[by] * X1[bx] + bS[by] * X2[bx];
            }
        } else {
            for (int l = 0; l < T1; ++l) {
                size_t bz = ((size_t)l * n1 + k) * W1 + dz + w;
                double mz = bM[bz], sz = bS[bz];
                for (int kk = 0; kk < T1; ++kk) {
                    size_t by = ((size_t)kk * n1 + j) * W1 + dy + w;
                    size_t bx = (((size_t)l * T1 + kk) * n1 + i) * W1 + dx + w;
                    double my = bM[by], sy = bS[by];
                    v += my * mz * X1[bx] + (sy * mz + my * sz) * X2[bx];
                }
            }
        }
    }
    if (s < G.Sc)
        Lv[r * G.SL + s] = (V)v;
    else
        Uv[r * G.SU + (s - G.Sc)] = (V)v;
    if (Mkeep) Mkeep[idx] = v;
}

// ---------------------------------------------------------------------------
// Wavefront levels of the natural ordering: row (i,j,k) depends on its lower
// neighbours, the latest of which are (i-1,j,k) and (i+w, j-1, k) (and
// (i+w, j+w, k-1) in 3D), so level = i + (w+1) j + (w+1)^2 k.
__global__ void k_level_count(StencilGeo G, int *count)
{
    long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= G.n) return;
    long long i = r % G.n1, j = (r / G.n1) % G.n1, k = r / ((long long)G.n1 * G.n1);
    if (G.d < 2) j = 0;
    if (G.d < 3) k = 0;
    long long lv = i + (G.w + 1) * j + (long long)(G.w + 1) * (G.w + 1) * k;
    atomicAdd(&count[lv], 1);
}
__global__ void k_level_scan(int levels, int *count)  // exclusive scan in place, one block
{
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < levels; base += blockDim.x) {
        int idx = base + threadIdx.x;
        int v = idx < levels ? count[idx] : 0;
        // block inclusive scan (Hillis-Steele in shared memory)
        __shared__ int buf[1024];
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (idx < levels) count[idx] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
}
__global__ void k_level_scatter(StencilGeo G, int *cursor, int *order)
{
    long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= G.n) return;
    long long i = r % G.n1, j = (r / G.n1) % G.n1, k = r / ((long long)G.n1 * G.n1);
    if (G.d < 2) j = 0;
    if (G.d < 3) k = 0;
    long long lv = i + (G.w + 1) * j + (long long)(G.w + 1) * (G.w + 1) * k;
    int pos = atomicAdd(&cursor[lv], 1);
    order[pos] = (int)r;
}

// ILU(0), Algorithm 2 in IKJ form on the stencil: for each lower slot k of row
// r in ascending column order, H(r,k) /= U(k,k), then H(r,j) -= H(r,k) U(k,j)
// for every upper slot j of row k whose column is in row r's pattern.  One warp
// per row; rows are claimed in wavefront order, so every row a warp waits for
// was claimed earlier by a running warp.  A row waits for a dependency line
// only when its first entry from that line is due (the wait is on the last
// row it needs from the line, which implies the earlier ones).
template <typename V>
__global__ void __launch_bounds__(256) k_ilu0(StencilGeo G, V *Lv, V *Uv, const int *order,
                                              unsigned *rowflag, unsigned *counter, int *err)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        long long idx = 0;
        if (lane == 0) idx = atomicAdd(counter, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= G.n) return;
        const long long r = order[idx];
        const int i = (int)(r % G.n1);
        const int j = (G.d >= 2) ? (int)((r / G.n1) % G.n1) : 0;
        const int k = (G.d == 3) ? (int)(r / ((long long)G.n1 * G.n1)) : 0;
        V *Lr = Lv + r * G.SL;
        V *Ur = Uv + r * G.SU;
        const double mii = (double)Ur[0];
        int seg_dy = 1 << 20, seg_dz = 1 << 20;
        bool ok = true;
        for (int s = 0; s < G.Sc && ok; ++s) {
            int dx, dy, dz;
            slot_offsets(G, s, dx, dy, dz);
            int ci = i + dx, cj = j + dy, ck = k + dz;
            if (ci < 0 || ci >= G.n1 || cj < 0 || cj >= G.n1 || ck < 0 || ck >= G.n1) continue;
            if (!structural(G, dx, dy, dz)) continue;
            if (dy != seg_dy || dz != seg_dz) {
                seg_dy = dy;
                seg_dz = dz;
                long long last;
                if (dy == 0 && dz == 0)
                    last = r - 1;
                else
                    last = (long long)min(i + G.w, G.n1 - 1) + G.n1 * ((long long)cj + (long long)G.n1 * ck);
                ok = wait_flag(rowflag + last, 1u, err);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
            }
            const long long kc = r + dx + (long long)G.n1 * (dy + (long long)G.n1 * dz);
            const V *Uk = Uv + kc * G.SU;
            __syncwarp();
            V hrk = Lr[s] / __ldcg(Uk);
            __syncwarp();
            if (lane == 0) Lr[s] = hrk;
            for (int u = 1 + lane; u <= G.Sc; u += 32) {
                int ex, ey, ez;
                slot_offsets(G, G.Sc + u, ex, ey, ez);
                int tx = dx + ex, ty = dy + ey, tz = dz + ez;
                if (tx < -G.w || tx > G.w || ty < -G.w || ty > G.w || tz < -G.w || tz > G.w) continue;
                int ti = i + tx, tj = j + ty, tk = k + tz;
                if (ti < 0 || ti >= G.n1 || tj < 0 || tj >= G.n1 || tk < 0 || tk >= G.n1) continue;
                if (!structural(G, tx, ty, tz)) continue;
                V ukj = __ldcg(Uk + u);
                int ts = slot_index(G, tx, ty, tz);
                if (ts < G.Sc)
                    Lr[ts] -= hrk * ukj;
                else
                    Ur[ts - G.Sc] -= hrk * ukj;
            }
            __syncwarp();
        }
        __syncwarp();
        if (lane == 0 && ok) {
            double uii = (double)Ur[0];
            if (!(uii > 1e-14 * fabs(mii))) set_err(err, DERR_BREAKDOWN);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(rowflag + r, 1u);
    }
}

// ---------------------------------------------------------------------------
template <typename V>
static int assemble_and_factor(lsg_ctx *c, cudaStream_t s)
{
    const Geom &g = c->g;
    StencilGeo G = sgeo(g);
    int T1 = g.T + 1;
    long long nK = (g.d == 3) ? (long long)T1 * T1 : T1;
    double *X1 = nullptr, *X2 = nullptr;
    cudaEvent_t e0, e1, e2;
    LSG_CK(cudaEventCreate(&e0));
    LSG_CK(cudaEventCreate(&e1));
    LSG_CK(cudaEventCreate(&e2));
    LSG_CK(cudaEventRecord(e0, s));
    if (g.d >= 2) {
        size_t nx = (size_t)nK * g.n1 * g.W1;
        LSG_CK(cudaMallocAsync((void **)&X1, sizeof(double) * nx, s));
        LSG_CK(cudaMallocAsync((void **)&X2, sizeof(double) * nx, s));
        ::lsg::count_launch();
        k_precontract<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(g.d, g.T, g.n1, g.W1, c->ahat, c->bhat,
                                                                   g.has_b, c->bandS, c->bandM, X1, X2);
        LSG_CK(cudaGetLastError());
    }
    LSG_CK(cudaMemsetAsync(c->Lv, 0, sizeof(V) * (size_t)g.n * g.SL, s));
    LSG_CK(cudaMemsetAsync(c->Uv, 0, sizeof(V) * (size_t)g.n * g.SU, s));
    long long tot = g.n * g.S;
    ::lsg::count_launch();
    k_assemble<V><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, c->ahat, c->bhat, c->bandS, c->bandM, X1, X2,
                                                               (V *)c->Lv, (V *)c->Uv, c->Mkeep);
    LSG_CK(cudaGetLastError());
    if (X1) LSG_CK(cudaFreeAsync(X1, s));
    if (X2) LSG_CK(cudaFreeAsync(X2, s));

    // wavefront order
    int *cnt = nullptr;
    LSG_CK(cudaMallocAsync((void **)&cnt, sizeof(int) * (size_t)g.levels, s));
    LSG_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)g.levels, s));
    unsigned nbk = (unsigned)((g.n + 255) / 256);
    ::lsg::count_launch();
    k_level_count<<<nbk, 256, 0, s>>>(G, cnt);
    ::lsg::count_launch();
    k_level_scan<<<1, 1024, 0, s>>>(g.levels, cnt);
    ::lsg::count_launch();
    k_level_scatter<<<nbk, 256, 0, s>>>(G, cnt, c->order);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaFreeAsync(cnt, s));

    // ILU(0)
    LSG_CK(cudaEventRecord(e1, s));
    LSG_CK(cudaMemsetAsync(c->rowflag, 0, sizeof(unsigned) * (size_t)g.n, s));
    LSG_CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned) * 8, s));
    int dev = 0, nsm = 0;
    LSG_CK(cudaGetDevice(&dev));
    LSG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    long long warps = std::min<long long>(g.n, (long long)nsm * 32);
    unsigned blocks = (unsigned)((warps + 7) / 8);
    ::lsg::count_launch();
    k_ilu0<V><<<blocks, 256, 0, s>>>(G, (V *)c->Lv, (V *)c->Uv, c->order, c->rowflag, c->counters, c->err);
    LSG_CK(cudaGetLastError());
    LSG_CK(cudaEventRecord(e2, s));
    LSG_CK(cudaEventSynchronize(e2));
    LSG_CK(cudaEventElapsedTime(&c->t_assemble_ms, e0, e1));
    LSG_CK(cudaEventElapsedTime(&c->t_ilu_ms, e1, e2));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return LSG_OK;
}

int build_preconditioner(lsg_ctx *c, cudaStream_t s)
{
    if (c->precision == LSG_FP64) return assemble_and_factor<double>(c, s);
    return assemble_and_factor<float>(c, s);
}

}  // namespace lsg
