// sweep.cu -- the one-step ILU(0) solve M z ~= r (Sec. 4.2): forward
// substitution with the unit lower factor (Algorithm 3) and backward
// substitution with the upper factor (Algorithm 4), on the stencil storage.
//
// Dependency structure (natural order, stencil half-width w): row (i,j,k)
// needs every lower neighbour; the newest ones are (i-1,j,k) and (i+w,j-1,k)
// (and (i+w,j+w,k-1) in 3D), one wavefront level earlier.  A line (fixed j,k)
// is therefore a chain whose position i may only be finished after the
// previous line (j-1,k) has finished position i+w.
//
// Kernel design (GB300): a CTA owns a band of B consecutive lines and runs two
// warps per line.
//   * The bulk warp streams the line's factor rows through a cp.async ring in
//     shared memory and, for each row, sums every entry except the K newest
//     ones of its own line and of the previous line (the "late" entries); it
//     hands the row over through a small record ring (bulk sum, right-hand
//     side, the late factor values, the inverse pivot).
//   * The finaliser warp applies only the <= 2K late entries, reading the
//     solution values of its own and the previous line from shared memory,
//     so the chain from one wavefront level to the next is a few shared-memory
//     operations instead of a full dot product and reduction.
// Lines of the band exchange values and progress through shared memory; bands
// exchange them through global memory (values) and release/acquire progress
// words, published by the bulk warps.  Bands are claimed in sweep order, so a
// CTA only ever waits for lines claimed earlier by a running CTA.  Every wait
// is bounded and reports LSG_ERR_TIMEOUT through the device error word.
#include "stencil.cuh"

namespace lsg {

constexpr int SW_MAXB = 8;          // lines per CTA (two warps each)
constexpr int SW_K = 4;             // late depth (clamped to w)
constexpr int SW_R = 16;            // record ring depth (rows a bulk warp may run ahead)
constexpr int SW_LATE = 2 * SW_K;   // late entries per row
constexpr int SW_PUB = 8;           // rows between global progress publications

struct SweepArgs {
    StencilGeo G;
    const void *F;       // factor rows: Lv (forward) or Uv (backward)
    int RL;              // row length of F (elements)
    const double *rhs;
    double *out;
    unsigned *gprog;     // per line progress in sweep order (virtual positions finished)
    unsigned *counter;   // band claim counter
    const int *done;
    int *err;
    int B;               // lines per CTA
    int K;               // late depth
};

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bounded spin on a shared-memory progress word.  Only SM-local state is read
// while spinning (a producer in this CTA that gives up releases its dependants
// itself), so a satisfied wait costs no off-SM round trip.
__device__ __forceinline__ bool spin_smem(volatile unsigned *p, unsigned need, int *err)
{
    if (*p >= need) return true;
    const long long t0 = clock64();
    for (;;) {
        if (*p >= need) return true;
        if (clock64() - t0 > kSpinBudgetCycles) {
            set_err(err, DERR_TIMEOUT);
            return false;
        }
    }
}

struct SweepSmem {
    size_t sy, rbulk, rrhs, rdiag, rlate, rhsring, ring, meta, total;
};

__host__ __device__ inline SweepSmem sweep_layout(int n1, int B, int D, int RL, int vsize, int nslot)
{
    SweepSmem L;
    size_t o = 0;
    L.sy = o;      o += (size_t)B * n1 * 8;
    L.rbulk = o;   o += (size_t)B * SW_R * 8;
    L.rrhs = o;    o += (size_t)B * SW_R * 8;
    L.rdiag = o;   o += (size_t)B * SW_R * 8;
    L.rlate = o;   o += (size_t)B * SW_R * SW_LATE * 8;
    L.rhsring = o; o += (size_t)B * D * 8;
    o = (o + 127) / 128 * 128;
    L.ring = o;    o += (size_t)B * D * RL * vsize;
    L.meta = o;    o += (size_t)nslot * 4;
    L.total = o;
    return L;
}

template <typename V, int DIR, int D>
__global__ void __launch_bounds__(64 * SW_MAXB) k_sweep(const __grid_constant__ SweepArgs A)
{
    if (A.done && *A.done) return;
    const StencilGeo G = A.G;
    const int n1 = G.n1, w = G.w, B = A.B, K = A.K, RL = A.RL;
    const int nslot = G.Sc;
    extern __shared__ __align__(128) unsigned char smem[];
    const SweepSmem Lo = sweep_layout(n1, B, D, RL, (int)sizeof(V), nslot);
    volatile double *sy = (volatile double *)(smem + Lo.sy);
    volatile double *rbulk = (volatile double *)(smem + Lo.rbulk);
    volatile double *rrhs = (volatile double *)(smem + Lo.rrhs);
    volatile double *rdiag = (volatile double *)(smem + Lo.rdiag);
    volatile double *rlate = (volatile double *)(smem + Lo.rlate);
    double *rhsring = (double *)(smem + Lo.rhsring);
    V *ring = (V *)(smem + Lo.ring);
    unsigned *meta = (unsigned *)(smem + Lo.meta);
    __shared__ volatile unsigned fin_prog[SW_MAXB], bulk_prog[SW_MAXB];
    __shared__ long long sband;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool is_bulk = wid < B;
    const int b = is_bulk ? wid : wid - B;
    const V *F = (const V *)A.F;

    // slot table: offsets and late class, in virtual (sweep-direction) terms
    for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
        int s = DIR > 0 ? t : G.Sc + 1 + t;
        int dx, dy, dz;
        slot_offsets(G, s, dx, dy, dz);
        int vx = DIR * dx, vy = DIR * dy, vz = DIR * dz;
        unsigned cls = 0;
        if (vy == 0 && vz == 0 && vx >= -K) cls = 1;                 // own line, newest K
        else if (vz == 0 && vy == -1 && vx >= w + 1 - K) cls = 2;    // previous line, newest K
        meta[t] = (unsigned)(dx + 128) | ((unsigned)(dy + 128) << 8) | ((unsigned)(dz + 128) << 16) | (cls << 24);
    }
    const long long nb = (G.nlines + B - 1) / B;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sband = atomicAdd(A.counter, 1u);
        if (threadIdx.x < SW_MAXB) {
            fin_prog[threadIdx.x] = 0;
            bulk_prog[threadIdx.x] = 0;
        }
        __syncthreads();
        const long long band = sband;
        if (band >= nb) return;
        const long long v = band * B + b;  // virtual line index (sweep order)
        if (v >= G.nlines) continue;
        const long long line = DIR > 0 ? v : G.nlines - 1 - v;
        const int j = (G.d >= 2) ? (int)(line % n1) : 0;
        const int k = (G.d == 3) ? (int)(line / n1) : 0;
        const int jv = DIR > 0 ? j : n1 - 1 - j;
        const int kv = DIR > 0 ? k : n1 - 1 - k;
        const bool has_prev = (G.d >= 2) && jv >= 1;        // previous line of the same plane
        const bool prev_in_band = has_prev && b >= 1;
        const long long prev_real = DIR > 0 ? line - 1 : line + 1;
        long long vplane = -1;                              // 3D: line (j+w, k-1) in sweep terms
        if (G.d == 3 && kv >= 1) vplane = (long long)min(jv + w, n1 - 1) + (long long)n1 * (kv - 1);
        const bool plane_in_band = vplane >= band * B;
        const long long plane_real = vplane < 0 ? -1 : (DIR > 0 ? vplane : G.nlines - 1 - vplane);

        if (is_bulk) {
            // ------------------------------------------------------------ bulk warp
            V *myring = ring + (size_t)b * D * RL;
            double *myrhs = rhsring + b * D;
            const int nch = RL * (int)sizeof(V) / 16;
            auto issue = [&](int p) {
                if (p < n1) {
                    int ii = DIR > 0 ? p : n1 - 1 - p;
                    long long r = ii + (long long)n1 * line;
                    const char *src = (const char *)(F + r * RL);
                    char *dst = (char *)(myring + (size_t)(p % D) * RL);
                    for (int c = lane; c < nch; c += 32) cp_async16(dst + 16 * c, src + 16 * c);
                    if (lane == 0) cp_async8(&myrhs[p % D], &A.rhs[r]);
                }
                cp_async_commit();
            };
            for (int p = 0; p < D - 1; ++p) issue(p);
            unsigned pub = 0, seen_prev = 0, seen_plane = 0;
            bool ok = true;
            for (int p = 0; p < n1; ++p) {
                issue(p + D - 1);
                cp_async_wait<D - 1>();
                __syncwarp();
                const int i = DIR > 0 ? p : n1 - 1 - p;
                if (lane == 0) {
                    if (p - SW_R + 1 > 0) ok = ok && spin_smem(&fin_prog[b], (unsigned)(p - SW_R + 1), A.err);
                    if (p - K > 0) ok = ok && spin_smem(&fin_prog[b], (unsigned)(p - K), A.err);
                    if (prev_in_band)
                        ok = ok && spin_smem(&fin_prog[b - 1], (unsigned)min(p + w + 1 - K, n1), A.err);
                    if (vplane >= 0 && plane_in_band)
                        ok = ok && spin_smem(&fin_prog[vplane - band * B], (unsigned)min(p + w + 1, n1), A.err);
                }
                if (has_prev && !prev_in_band)
                    ok = ok && wait_flag_cached(A.gprog + prev_real, (unsigned)min(p + w + 1, n1), A.err, &seen_prev);
                if (vplane >= 0 && !plane_in_band)
                    ok = ok && wait_flag_cached(A.gprog + plane_real, (unsigned)min(p + w + 1, n1), A.err, &seen_plane);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                __threadfence_block();
                const V *row = myring + (size_t)(p % D) * RL;
                double acc = 0.0;
#pragma unroll 4
                for (int t = lane; t < nslot; t += 32) {
                    unsigned m = meta[t];
                    unsigned cls = m >> 24;
                    if (cls == 1 || (cls == 2 && prev_in_band)) continue;
                    int dx = (int)(m & 255u) - 128, dy = (int)((m >> 8) & 255u) - 128, dz = (int)((m >> 16) & 255u) - 128;
                    int ci = i + dx, cj = j + dy, ck = k + dz;
                    if (ci < 0 || ci >= n1 || cj < 0 || cj >= n1 || ck < 0 || ck >= n1) continue;
                    long long cl = line + dy + (long long)n1 * dz;
                    long long vc = DIR > 0 ? cl : G.nlines - 1 - cl;
                    double yv = (vc >= band * B) ? sy[(vc - band * B) * n1 + ci] : __ldcg(A.out + ci + (long long)n1 * cl);
                    acc += (double)row[DIR > 0 ? t : 1 + t] * yv;
                }
                acc = warp_sum(acc);
                const int q = p % SW_R;
                if (lane < 2 * K) {
                    const int t = lane;
                    int vx, vy;
                    if (t < K) {
                        vx = -(t + 1);
                        vy = 0;
                    } else {
                        vx = w - (t - K);
                        vy = -1;
                    }
                    int pos = p + vx;
                    double fv = 0.0;
                    if (pos >= 0 && pos < n1 && (t < K || prev_in_band)) {
                        int s = slot_index(G, DIR * vx, DIR * vy, 0);
                        fv = (double)row[DIR > 0 ? s : s - G.Sc];
                    }
                    rlate[((size_t)b * SW_R + q) * SW_LATE + t] = fv;
                }
                if (lane == 0) {
                    rbulk[b * SW_R + q] = acc;
                    rrhs[b * SW_R + q] = myrhs[p % D];
                    rdiag[b * SW_R + q] = DIR > 0 ? 1.0 : 1.0 / (double)row[0];
                }
                __threadfence_block();
                __syncwarp();
                if (lane == 0) bulk_prog[b] = (unsigned)(p + 1);
                // publish finished values of this line to global memory (lane 0
                // reads the racy progress word once so the branch is warp-uniform)
                unsigned fin = 0;
                if (lane == 0) fin = fin_prog[b];
                fin = __shfl_sync(0xffffffffu, fin, 0);
                if (fin >= pub + SW_PUB) {
                    __threadfence_block();
                    for (unsigned pp = pub + lane; pp < fin; pp += 32) {
                        int ii = DIR > 0 ? (int)pp : n1 - 1 - (int)pp;
                        A.out[ii + (long long)n1 * line] = sy[(long long)b * n1 + ii];
                    }
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) st_release(A.gprog + line, fin);
                    pub = fin;
                }
            }
            cp_async_wait<0>();
            __syncwarp();
            if (ok) {
                if (lane == 0) ok = spin_smem(&fin_prog[b], (unsigned)n1, A.err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __threadfence_block();
                for (unsigned pp = pub + lane; pp < (unsigned)n1; pp += 32) {
                    int ii = DIR > 0 ? (int)pp : n1 - 1 - (int)pp;
                    A.out[ii + (long long)n1 * line] = sy[(long long)b * n1 + ii];
                }
            }
            __threadfence();
            __syncwarp();
            // on failure the error word is set; publishing completion lets dependants finish quickly
            if (lane == 0) st_release(A.gprog + line, (unsigned)n1);
            if (!ok && lane == 0) bulk_prog[b] = (unsigned)n1;
        } else {
            // ------------------------------------------------------------ finaliser warp
            bool ok = true;
            double yprev = 0.0;
            const long long rowb = (long long)b * n1, rowp = (long long)(b - 1) * n1;
            for (int p = 0; p < n1; ++p) {
                if (lane == 0) {
                    const int i = DIR > 0 ? p : n1 - 1 - p;
                    ok = ok && spin_smem(&bulk_prog[b], (unsigned)(p + 1), A.err);
                    __threadfence_block();
                    const int q = p % SW_R;
                    const volatile double *lf = rlate + ((size_t)b * SW_R + q) * SW_LATE;
                    double acc = rrhs[b * SW_R + q] - rbulk[b * SW_R + q];
                    for (int t = 1; t < K; ++t) {
                        int pos = p - 1 - t;
                        if (pos >= 0) acc -= lf[t] * sy[rowb + (DIR > 0 ? pos : n1 - 1 - pos)];
                    }
                    if (prev_in_band) {
                        ok = ok && spin_smem(&fin_prog[b - 1], (unsigned)min(p + w, n1), A.err);
                        __threadfence_block();
                        for (int t = K + 1; t < 2 * K; ++t) {
                            int pos = p + w - (t - K);
                            if (pos >= 0 && pos < n1) acc -= lf[t] * sy[rowp + (DIR > 0 ? pos : n1 - 1 - pos)];
                        }
                        ok = ok && spin_smem(&fin_prog[b - 1], (unsigned)min(p + w + 1, n1), A.err);
                        __threadfence_block();
                        int pos = p + w;
                        if (pos < n1) acc -= lf[K] * sy[rowp + (DIR > 0 ? pos : n1 - 1 - pos)];
                    }
                    if (p >= 1) acc -= lf[0] * yprev;
                    double val = acc * rdiag[b * SW_R + q];
                    sy[rowb + i] = val;
                    yprev = val;
                    __threadfence_block();
                    fin_prog[b] = ok ? (unsigned)(p + 1) : (unsigned)n1;
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
            }
        }
    }
}

template <typename V, int DIR, int D>
static int launch_sweep(const SweepArgs &A, size_t smem, unsigned grid, cudaStream_t s)
{
    static size_t attr = 0;  // benign race: setting the attribute twice is harmless
    if (smem > attr) {
        LSG_CK(cudaFuncSetAttribute(k_sweep<V, DIR, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    ::lsg::count_launch();
    k_sweep<V, DIR, D><<<grid, 64 * A.B, smem, s>>>(A);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

template <typename V>
static int sweeps(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s)
{
    const Geom &g = c->g;
    SweepArgs A;
    A.G = sgeo(g);
    A.done = done;
    A.err = c->err;
    A.K = std::min(SW_K, g.w);
    // lines per CTA and ring depth: the largest that fit in shared memory
    const size_t budget = 200 * 1024;
    int B = SW_MAXB, D = 4;
    auto fits = [&](int b, int d, int RL) {
        return sweep_layout(g.n1, b, d, RL, (int)sizeof(V), g.Sc).total <= budget;
    };
    const int RLmax = std::max(g.SL, g.SU);
    while (B > 1 && !fits(B, D, RLmax)) {
        if (D == 4)
            D = 2;
        else {
            B /= 2;
            D = 4;
        }
    }
    if (!fits(B, D, RLmax)) D = 2;
    if (!fits(B, D, RLmax)) return LSG_ERR_ARG;  // stencil too large for one row in shared memory
    if (B > g.nlines) B = (int)std::max<long long>(1, g.nlines);
    A.B = B;
    int dev = 0, nsm = 0;
    LSG_CK(cudaGetDevice(&dev));
    LSG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    long long nbands = (g.nlines + B - 1) / B;
    unsigned grid = (unsigned)std::min<long long>(nbands, nsm);
    LSG_CK(cudaMemsetAsync(c->prog, 0, sizeof(unsigned) * 2 * (size_t)g.nlines, s));
    LSG_CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(unsigned) * 2, s));
    // forward: L y = r
    A.F = c->Lv;
    A.RL = g.SL;
    A.rhs = r;
    A.out = c->ys;
    A.gprog = c->prog;
    A.counter = c->counters + 1;
    size_t smf = sweep_layout(g.n1, B, D, g.SL, (int)sizeof(V), g.Sc).total;
    if (D == 4)
        LSG_TRY((launch_sweep<V, 1, 4>(A, smf, grid, s)));
    else
        LSG_TRY((launch_sweep<V, 1, 2>(A, smf, grid, s)));
    // backward: U z = y
    A.F = c->Uv;
    A.RL = g.SU;
    A.rhs = c->ys;
    A.out = z;
    A.gprog = c->prog + g.nlines;
    A.counter = c->counters + 2;
    size_t smb = sweep_layout(g.n1, B, D, g.SU, (int)sizeof(V), g.Sc).total;
    if (D == 4)
        LSG_TRY((launch_sweep<V, -1, 4>(A, smb, grid, s)));
    else
        LSG_TRY((launch_sweep<V, -1, 2>(A, smb, grid, s)));
    return LSG_OK;
}

int apply_Minv(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s)
{
    if (c->precision == LSG_FP64) return sweeps<double>(c, r, z, done, s);
    return sweeps<float>(c, r, z, done, s);
}

}  // namespace lsg
