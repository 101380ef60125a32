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

#include <mutex>

#include "lsg_internal.cuh"
#include "stencil.cuh"

namespace lsg {

// ---------------------------------------------------------------------------
// M assembly.  With band matrices S^(t)[i][o], M^(t)[i][o] (o = column - row),
// `2DM` in Kronecker form (Sec. 4.2), with the series a_x, a_y of the two gradient
// terms (the same one for a scalar coefficient) and b, gives for row (i,j),
// offset (ox,oy):
//   M = sum_k [ M^(k)[j][oy] X1[k][i][ox] + S^(k)[j][oy] X2[k][i][ox] ],
//   X1[k][i][ox] = sum_t (ax_tk S^(t)[i][ox] + b_tk M^(t)[i][ox]),
//   X2[k][i][ox] = sum_t ay_tk M^(t)[i][ox]          (t: x degree, k: y degree)
// and `3DM` similarly with a second contraction over the z degree and a third
// array X3 (the series of a_z).  Series are zero beyond their degrees.
__global__ void k_precontract(int d, int T, int n1, int W1, const double *ahx, const double *ahy,
                              const double *ahz, const double *bhat, int has_b, const double *bS,
                              const double *bM, double *X1, double *X2, double *X3)
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
    double x1 = 0.0, x2 = 0.0, x3 = 0.0;
    for (int t = 0; t < T1; ++t) {
        double bt = bhat[K * T1 + t];
        double s = bS[((size_t)t * n1 + i) * W1 + o], m = bM[((size_t)t * n1 + i) * W1 + o];
        x1 += ahx[K * T1 + t] * s + (has_b ? bt * m : 0.0);
        x2 += ahy[K * T1 + t] * m;
        if (X3) x3 += ahz[K * T1 + t] * m;
    }
    X1[idx] = x1;
    X2[idx] = x2;
    if (X3) X3[idx] = x3;
}

template <typename V>
__global__ void k_assemble(StencilGeo G, const double *ahat, const double *bhat, const double *bS,
                           const double *bM, const double *X1, const double *X2, const double *X3, V *Lv,
                           V *Uv, double *Mkeep)
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
                    v += my * mz * X1[bx] + sy * mz * X2[bx] + my * sz * X3[bx];
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
// for every upper slot j of row k whose column is in row r's pattern.
//
// One warp per row, rows claimed in wavefront order (a warp only waits for
// rows claimed earlier by running warps).  The row lives in shared memory for
// the whole elimination.  In stencil slot numbering the target of U(k, Sc+u)
// is slot s+u of row r (s: the step's lower slot), valid when the target
// offset stays in the box and in the pattern; columns outside the grid hold
// exact zeros in both rows, so they need no test.
//
// Each step waits only for its own row k (not for the whole line k belongs
// to), so a row follows the rows it depends on closely: once the newest of
// them finishes, only the last step or two remain.  The U rows of the next
// D-1 steps are prefetched into a ring of shared-memory buffers with 16-byte
// cp.async copies when their rows are already finished (checked without
// blocking); a step whose row was not ready at prefetch time waits for it and
// copies it then.  A finished row stores 1 / U(r,r) in the pad slot SU-1.
constexpr int ILU_MAX_WARPS = 8;
#ifndef ILU_LEVELS
// Rows in flight of a 2D factorisation set up beside other work (LSG_SETUP_SHARED_GPU), in
// wavefront levels' worth of rows: measured on a GB300, 8 and 16 levels slowed the N=512
// factorisation 5x and 2.6x (a row's elimination overlaps far more levels than its last steps
// suggest), 48 cost 3 % there (a lone N=256 factorisation 54 %: 13.6 -> 20.9 ms) and made the
// 256 set-ups of the batched form (N = 32..256 on 8 streams) 27 % faster.
#define ILU_LEVELS 48
#endif

struct IluSmem {
    size_t off, smask, ord, warps, per_warp, total;
};
__host__ __device__ inline size_t al16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ inline IluSmem ilu_layout(int S, int SU, int D, int vsize, int nw)
{
    IluSmem L;
    L.off = 0;
    L.smask = al16((size_t)S * 4);
    L.ord = L.smask + al16((size_t)S);
    L.warps = L.ord + al16((size_t)(S - 1) / 2 * 2);  // Sc step-order entries
    // the row, the U-row ring, and one bit per step: its row had finished when this row started
    L.per_warp = al16((size_t)S * vsize) + (size_t)D * SU * vsize + al16(((size_t)(S - 1) / 2 + 31) / 32 * 4);
    L.total = L.warps + (size_t)nw * L.per_warp;
    return L;
}

__device__ __forceinline__ void ilu_cp16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void ilu_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
template <int N>
__device__ __forceinline__ void ilu_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// unpack a slot offset stored as three biased bytes
__device__ __forceinline__ void ilu_off(int m, int &dx, int &dy, int &dz)
{
    dx = (m & 255) - 128;
    dy = ((m >> 8) & 255) - 128;
    dz = ((m >> 16) & 255) - 128;
}

// first position >= p of the step order whose slot's column is in the grid of row (i,j,k)
__device__ __forceinline__ int ilu_next(const StencilGeo &G, const int *off, const short *ord, int nord, int p, int i,
                                        int j, int k)
{
    for (; p < nord; ++p) {
        int dx, dy, dz;
        ilu_off(off[ord[p]], dx, dy, dz);
        const int ci = i + dx, cj = j + dy, ck = k + dz;
        if (ci >= 0 && ci < G.n1 && cj >= 0 && cj < G.n1 && ck >= 0 && ck < G.n1) return p;
    }
    return nord;
}

__device__ __forceinline__ long long ilu_row_of(const StencilGeo &G, long long r, int m)
{
    int dx, dy, dz;
    ilu_off(m, dx, dy, dz);
    return r + dx + (long long)G.n1 * (dy + (long long)G.n1 * dz);
}

// All lanes copy U row kr into ring buffer dst (16-byte chunks).
template <typename V>
__device__ __forceinline__ void ilu_copy_row(const StencilGeo &G, const V *Uv, long long kr, V *dst)
{
    constexpr int CE = 16 / (int)sizeof(V);
    const V *src = Uv + kr * G.SU;
    for (int c = (threadIdx.x & 31); c < G.SU / CE; c += 32) ilu_cp16(dst + c * CE, src + c * CE);
}

template <typename V, int D>
__global__ void __launch_bounds__(32 * ILU_MAX_WARPS, 2) k_ilu0(StencilGeo G, V *Lv, V *Uv, const int *order,
                                                            unsigned *rowflag, unsigned *counter, int *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int S = G.S, Sc = G.Sc, nU = S - Sc, SU = G.SU;
    const IluSmem Lo = ilu_layout(S, SU, D, (int)sizeof(V), nw);
    int *off = (int *)(smem + Lo.off);           // offset (dx,dy,dz) of every slot, biased bytes
    unsigned char *smask = smem + Lo.smask;      // structural flag per slot
    short *ord = (short *)(smem + Lo.ord);       // the step order: structural lower slots
    V *a = (V *)(smem + Lo.warps + (size_t)wid * Lo.per_warp);
    V *ring = (V *)((unsigned char *)a + al16((size_t)S * sizeof(V)));
    for (int t = threadIdx.x; t < S; t += blockDim.x) {
        int dx, dy, dz;
        slot_offsets(G, t, dx, dy, dz);
        off[t] = (dx + 128) | ((dy + 128) << 8) | ((dz + 128) << 16);
        smask[t] = structural(G, dx, dy, dz) ? 1 : 0;
    }
    __syncthreads();
    // Step order.  Step k can change H(r,k') only if k' - k is an upper offset in the
    // box, and such an offset raises the wavefront level i + (w+1) j + (w+1)^2 k by at
    // least one; so taking the lower slots by increasing level (then column) is a
    // valid elimination order, and it leaves the steps on the rows of the previous
    // level (the last to finish) for the end: two of them in 2D, three in 3D, where
    // column order would leave w+1.  The result is the same; only the order in which
    // the updates of each entry are added differs.
    auto lev = [&](int t) {
        int dx, dy, dz;
        ilu_off(off[t], dx, dy, dz);
        return dx + (G.w + 1) * (dy + (G.w + 1) * dz);
    };
    for (int t = threadIdx.x; t < Sc; t += blockDim.x) {
        if (!smask[t]) continue;
        const int lt = lev(t);
        int rank = 0;
        for (int u = 0; u < Sc; ++u) {
            if (!smask[u]) continue;
            const int lu = lev(u);
            rank += (lu < lt || (lu == lt && u < t)) ? 1 : 0;
        }
        ord[rank] = (short)t;
    }
    __shared__ int s_nord;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int t = 0; t < Sc; ++t) c += smask[t];
        s_nord = c;
    }
    __syncthreads();
    const int nord = s_nord;

    for (;;) {
        long long idx = 0;
        if (lane == 0) idx = atomicAdd(counter, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= G.n) return;
        if (*(volatile int *)err != 0) return;
        const long long r = order[idx];
        const int i = (int)(r % G.n1);
        const int j = (G.d >= 2) ? (int)((r / G.n1) % G.n1) : 0;
        const int k = (G.d == 3) ? (int)(r / ((long long)G.n1 * G.n1)) : 0;
        for (int t = lane; t < Sc; t += 32) a[t] = Lv[r * G.SL + t];
        for (int u = lane; u < nU; u += 32) a[Sc + u] = Uv[r * SU + u];
        // which of the rows this row uses had finished already (most of them: rows are
        // claimed well ahead of the wavefront): their flags, read by all lanes at once
        // (relaxed reads, then one fence), spare the per-step check below
        unsigned *done = (unsigned *)((unsigned char *)ring + (size_t)D * SU * sizeof(V));
        for (int p0 = 0; p0 < nord; p0 += 4 * 32) {
            unsigned fl[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int p = p0 + 32 * g + lane;
                fl[g] = 0;
                if (p < nord) {
                    int dx, dy, dz;
                    ilu_off(off[ord[p]], dx, dy, dz);
                    const int ci = i + dx, cj = j + dy, ck = k + dz;
                    if (ci >= 0 && ci < G.n1 && cj >= 0 && cj < G.n1 && ck >= 0 && ck < G.n1)
                        fl[g] = ld_relaxed_u32(rowflag + r + dx + (long long)G.n1 * (dy + (long long)G.n1 * dz));
                }
            }
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const unsigned m = __ballot_sync(0xffffffffu, fl[g] != 0);
                if (lane == 0 && p0 + 32 * g < nord) done[(p0 >> 5) + g] = m;
            }
        }
        __threadfence();
        __syncwarp();
        const V mii = a[Sc];

        // producer cursor ps: the next step whose U row goes to ring slot pq; bit q of
        // `ready` says whether slot q holds its step's row (prefetched) or must be
        // fetched when consumed (its row was not finished at prefetch time)
        int ps = ilu_next(G, off, ord, nord, 0, i, j, k), pq = 0;
        unsigned ready = 0;
        auto prefetch = [&]() {
            if (ps < nord) {
                const long long kr = ilu_row_of(G, r, off[ord[ps]]);
                unsigned f = (done[ps >> 5] >> (ps & 31)) & 1u;
                if (!f) {
                    if (lane == 0) f = ld_acquire(rowflag + kr);
                    f = __shfl_sync(0xffffffffu, f, 0);
                }
                __syncwarp();
                if (f) {
                    ilu_copy_row<V>(G, Uv, kr, ring + (size_t)pq * SU);
                    ready |= 1u << pq;
                } else {
                    ready &= ~(1u << pq);
                }
                ps = ilu_next(G, off, ord, nord, ps + 1, i, j, k);
                pq = (pq + 1 == D) ? 0 : pq + 1;
            }
            ilu_commit();
        };
#pragma unroll 1
        for (int q = 0; q < D - 1; ++q) prefetch();
        int cp = ilu_next(G, off, ord, nord, 0, i, j, k), q = 0;
        bool ok = true;
        while (cp < nord) {
            const int cs = ord[cp];
            prefetch();  // step cs + D - 1 into the slot freed by the previous step
            ilu_wait<D - 1>();
            V *Uk = ring + (size_t)q * SU;
            if (!(ready >> q & 1u)) {
                // the row was not finished when prefetched: wait for it, then copy
                const long long kr = ilu_row_of(G, r, off[cs]);
                ok = __all_sync(0xffffffffu, wait_flag(rowflag + kr, 1u, err));
                if (!ok) break;
                ilu_copy_row<V>(G, Uv, kr, Uk);
                ilu_commit();
                ilu_wait<0>();
            }
            __syncwarp();
            const V l = a[cs] * Uk[SU - 1];  // H(r,k) / U(k,k) by the stored reciprocal pivot
            int dx, dy, dz;
            ilu_off(off[cs], dx, dy, dz);
            // Only the upper offsets e of row k whose target d+e stays in the box are
            // enumerated, packed over the lanes: per axis the valid e form a range, so the
            // targets are the runs (ez, ey, ex in [exlo, exhi]), with the half-plane ez = 0
            // restricted to ey > 0, or ey = 0 and ex > 0 (e above the diagonal).
            const int wy = G.d >= 2 ? G.w : 0, wz = G.d == 3 ? G.w : 0;
            const int exlo = max(-G.w, -G.w - dx), exhi = min(G.w, G.w - dx);
            const int eylo = max(-wy, -wy - dy), eyhi = min(wy, wy - dy);
            const int Lx = exhi - exlo + 1, Ly = eyhi - eylo + 1, Lz = min(wz, wz - dz) + 1;
            const int ex0 = max(1, exlo);
            const int len0 = max(0, exhi - ex0 + 1);     // ez = 0, ey = 0
            const int n0 = len0 + max(0, eyhi) * Lx;      // ez = 0, ey in [1, eyhi]
            const int cnt = n0 + (Lz - 1) * Ly * Lx;      // ez in [1, Lz)
            const float ilx = 1.0f / (float)Lx, ilyx = 1.0f / (float)(Ly * Lx);
            const int sbase = G.w + G.W1 * (wy + G.W1 * wz) - Sc;  // slot(e) - Sc = ex + W1 ey + W1^2 ez + sbase
            for (int f = lane; f < cnt; f += 32) {
                int ex, ey, ez;
                if (f < len0) {
                    ez = 0;
                    ey = 0;
                    ex = ex0 + f;
                } else if (f < n0) {
                    const int g = f - len0, qy = (int)(((float)g + 0.5f) * ilx);
                    ez = 0;
                    ey = 1 + qy;
                    ex = exlo + (g - qy * Lx);
                } else {
                    const int h = f - n0, qz = (int)(((float)h + 0.5f) * ilyx);
                    const int rem = h - qz * Ly * Lx, qy = (int)(((float)rem + 0.5f) * ilx);
                    ez = 1 + qz;
                    ey = eylo + qy;
                    ex = exlo + (rem - qy * Lx);
                }
                const int u = ex + G.W1 * (ey + G.W1 * ez) + sbase;
                if (!smask[cs + u]) continue;
                a[cs + u] -= l * Uk[u];
            }
            __syncwarp();
            if (lane == 0) a[cs] = l;
            q = (q + 1 == D) ? 0 : q + 1;
            cp = ilu_next(G, off, ord, nord, cp + 1, i, j, k);
        }
        ilu_wait<0>();
        __syncwarp();
        if (!ok) return;  // a wait gave up: the error word is set, other warps stop too
        const V uii = a[Sc];
        if (lane == 0 && !((double)uii > 1e-14 * fabs((double)mii))) set_err(err, DERR_BREAKDOWN);
        // the U row (all that later rows read) is published first; the L row only
        // matters to the sweeps, after this kernel
        for (int u = lane; u < nU; u += 32) Uv[r * SU + u] = a[Sc + u];
        if (lane == 0) Uv[r * SU + SU - 1] = V(1) / uii;
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(rowflag + r, 1u);
        for (int t = lane; t < Sc; t += 32) Lv[r * G.SL + t] = a[t];
    }
}

template <typename V, int D>
static int launch_ilu0_d(lsg_ctx *c, const StencilGeo &G, int nsm, cudaStream_t s)
{
    const size_t budget = 224 * 1024;  // of the 227 KB a CTA may opt in to
    const IluSmem one = ilu_layout(G.S, G.SU, D, (int)sizeof(V), 1);
    if (one.total > budget) return LSG_ERR_ARG;  // stencil too wide for a shared-memory row
    int nw = (int)std::min<size_t>(ILU_MAX_WARPS, 1 + (budget - one.total) / one.per_warp);
    long long ctas = 0;
    if (G.d == 2 && (c->flags & LSG_SETUP_SHARED_GPU)) {
        // rows in flight: about n1/(w+1) rows per wavefront level times ILU_LEVELS; more
        // warps only spin on rows far ahead, and a grid that fills the GPU keeps the
        // factorisations of other problems (batched and served solves on other streams)
        // from running beside it.  Spread over the SMs: the fewest warps per CTA that
        // reach every SM.
        const long long warps = ((long long)(G.n1 + G.w) / (G.w + 1) + 2) * ILU_LEVELS;
        if (warps < (long long)nsm * 2 * nw) {
            nw = (int)std::max<long long>(1, std::min<long long>(nw, (warps + nsm - 1) / nsm));
            ctas = (warps + nw - 1) / nw;
        }
    }
    const size_t smem = ilu_layout(G.S, G.SU, D, (int)sizeof(V), nw).total;
    {
        // the attribute only grows: set-ups on other host threads may be launching with more
        static std::mutex mu;
        static size_t attr = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (smem > attr) {
            LSG_CK(cudaFuncSetAttribute(k_ilu0<V, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = smem;
        }
    }
    if (ctas == 0) {
        int per_sm = 0;
        LSG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ilu0<V, D>, 32 * nw, smem));
        if (per_sm < 1) return LSG_ERR_ARG;
        ctas = std::min<long long>((long long)nsm * per_sm, (G.n + nw - 1) / nw);
    }
    ctas = std::min<long long>(ctas, (G.n + nw - 1) / nw);
    ::lsg::count_launch();
    k_ilu0<V, D><<<(unsigned)ctas, 32 * nw, smem, s>>>(G, (V *)c->Lv, (V *)c->Uv, c->order, c->rowflag,
                                                        c->counters, c->err);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

template <typename V>
static int launch_ilu0(lsg_ctx *c, const StencilGeo &G, int nsm, cudaStream_t s)
{
    // ring depth: four U rows in flight for lines (1D/2D), two for the wide 3D rows
    if (G.d <= 2) return launch_ilu0_d<V, 4>(c, G, nsm, s);
    return launch_ilu0_d<V, 2>(c, G, nsm, s);
}

// ---------------------------------------------------------------------------
template <typename V>
static int assemble_and_factor(lsg_ctx *c, cudaStream_t s)
{
    const Geom &g = c->g;
    StencilGeo G = sgeo(g);
    int T1 = g.T + 1;
    long long nK = (g.d == 3) ? (long long)T1 * T1 : T1;
    double *X1 = nullptr, *X2 = nullptr, *X3 = nullptr;
    cudaEvent_t e0, e1, e2;
    LSG_CK(cudaEventCreate(&e0));
    LSG_CK(cudaEventCreate(&e1));
    LSG_CK(cudaEventCreate(&e2));
    LSG_CK(cudaEventRecord(e0, s));
    if (g.d >= 2) {
        size_t nx = (size_t)nK * g.n1 * g.W1;
        LSG_CK(cudaMallocAsync((void **)&X1, sizeof(double) * nx, s));
        LSG_CK(cudaMallocAsync((void **)&X2, sizeof(double) * nx, s));
        if (g.d == 3) LSG_CK(cudaMallocAsync((void **)&X3, sizeof(double) * nx, s));
        ::lsg::count_launch();
        k_precontract<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(g.d, g.T, g.n1, g.W1, c->ahat, c->ahaty,
                                                                   c->ahatz, c->bhat, g.has_b, c->bandS,
                                                                   c->bandM, X1, X2, X3);
        LSG_CK(cudaGetLastError());
    }
    LSG_CK(cudaMemsetAsync(c->Lv, 0, sizeof(V) * (size_t)g.n * g.SL, s));
    LSG_CK(cudaMemsetAsync(c->Uv, 0, sizeof(V) * (size_t)g.n * g.SU, s));
    long long tot = g.n * g.S;
    ::lsg::count_launch();
    k_assemble<V><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, c->ahat, c->bhat, c->bandS, c->bandM, X1, X2,
                                                               X3, (V *)c->Lv, (V *)c->Uv, c->Mkeep);
    LSG_CK(cudaGetLastError());
    if (X1) LSG_CK(cudaFreeAsync(X1, s));
    if (X2) LSG_CK(cudaFreeAsync(X2, s));
    if (X3) LSG_CK(cudaFreeAsync(X3, s));

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
    LSG_TRY(launch_ilu0<V>(c, G, nsm, s));
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
