// sweep.cu -- the one-step ILU(0) solve M z ~= r (Sec. 4.2): forward
// substitution with the unit lower factor (Algorithm 3) and backward
// substitution with the upper factor (Algorithm 4), on the stencil storage.
//
// Dependency structure (natural order, stencil half-width w): row (i,j,k)
// needs its lower neighbours; the newest are (i-1,j,k) and (i+w,j-1,k) (and
// (i+w,j+w,k-1) in 3D).  A line (fixed j,k) is a chain whose position i may
// be finished once the previous line has finished position i+w.
//
// Two kernels.  k_sweep_line (further below) runs one line per CTA with the
// line's work split over warps; it is used whenever its shared-memory layout
// fits (1D, 2D with up to 512 lower slots per row, 3D with a ring of at least
// 8 rows).  k_sweep, the band kernel described next, covers the rest (wider 2D
// stencils, 3D rows too long for that ring).
//
// Band kernel design (GB300).  A CTA owns a band of B consecutive lines, one
// compute warp per line.  A line warp advances as soon as its inputs exist:
// it waits only for its predecessor's progress counter in shared memory (the
// halo loader publishes separate counts for the line before the band and the
// older halo lines).  Each row's dot product is split: the stale part -- every
// term but the two newest dependencies (the previous position of the line and
// position +w of the previous line) -- is computed one position ahead, off the
// critical path; finishing a row is then two multiply-adds and, backward, a
// multiply by the reciprocal pivot the factorisation stored.  All data
// movement is done by three helper warps:
//   * a TMA producer streams factor rows into a per-line ring in shared memory
//     with bulk copies (cp.async.bulk) that complete on mbarriers, D rows ahead
//     of the row that reads them;
//   * a halo loader stages the w lines before the band (finished by the
//     previous band) into shared memory with 16-byte cp.async copies as soon
//     as their progress words allow, and publishes how far they are staged;
//   * a publisher copies finished values to global memory and releases
//     per-line progress words.
// The 1D/2D line warps keep their stencil offsets in registers and read padded,
// zero-initialised row buffers, so the dot product has no branches: a slot
// outside the grid carries an exact-zero factor.  In 3D, neighbours in other
// planes are read from global memory (in groups of slots per lane) after the
// plane's progress word is acquired, and a plane's first line does not wait
// for the line before it in sweep order (the last line of the previous plane,
// no neighbour).  Bands are claimed in sweep order, so a CTA only waits for
// lines claimed earlier by a running CTA; every wait is bounded and reports
// LSG_ERR_TIMEOUT through the device error word.
#include "stencil.cuh"

namespace lsg {

constexpr int SW_MAXB = 8;   // compute warps (lines) per CTA
constexpr int SW_HELP = 3;   // helper warps: TMA producer, halo loader, publisher
constexpr int SW_KS = 16;    // register-resident slots per lane (1D/2D path)

struct SweepArgs {
    StencilGeo G;
    const void *F;       // factor rows: Lv (forward) or Uv (backward)
    int RL;              // row length of F (elements); RL * sizeof(V) is a multiple of 16
    const void *rhs;     // AT[n]
    void *out;           // AT[n]
    unsigned *gprog;     // per line progress in sweep order (positions finished)
    unsigned *counter;   // band claim counter
    const int *done;
    int *err;
    int B;               // lines per CTA (k_sweep)
    int K;               // fresh window (k_sweep_line)
    long long budget;    // SM clock cycles a dependency wait may take before it reports a timeout
};

// ---- asynchronous copy and mbarrier primitives (inline PTX, sm_90+) --------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// TMA bulk copy global -> shared, completion counted on an mbarrier.
__device__ __forceinline__ void tma_load(void *sdst, const void *gsrc, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk prefetch of global memory into L2 (no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void *gsrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

// Bounded wait for an mbarrier phase (every lane polls, so each gets acquire order).
// Waits for copies this CTA issued itself (before it exits) keep the default budget.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int *err,
                                          long long budget = kSpinBudgetCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > budget) {
            set_err(err, DERR_TIMEOUT);
            return false;
        }
    }
}

struct SweepSmem {
    size_t rowoff, sy, srhs, ring, mbar, meta, total;
    int RS;    // row stride (elements) of the value buffers
    int PADL;  // left padding (elements) before position 0
};

__host__ __device__ inline SweepSmem sweep_layout(int n1, int w, int B, int D, int RL, int vsize, int nslot, int asize)
{
    SweepSmem L;
    const int ce = 16 / asize;                          // elements per 16-byte chunk
    L.PADL = ((w + ce - 1) / ce + 1) * ce;              // room for i+dx >= -w and chunk alignment
    L.RS = ((L.PADL + n1 + w + 2 * ce + ce - 1) / ce) * ce;
    size_t o = 0;
    L.rowoff = o;  o += (size_t)(w + SW_MAXB) * 4;
    o = (o + 127) / 128 * 128;
    L.sy = o;      o += (size_t)(w + B) * L.RS * asize;
    o = (o + 15) / 16 * 16;
    L.srhs = o;    o += (size_t)B * n1 * asize;
    o = (o + 127) / 128 * 128;
    L.ring = o;    o += (size_t)B * D * RL * vsize;
    o = (o + 7) / 8 * 8;
    L.mbar = o;    o += (size_t)B * D * 8;
    L.meta = o;    o += (size_t)nslot * 4;
    L.total = o;
    return L;
}

__device__ __forceinline__ int ld_acquire_cta(const volatile int *p)
{
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32((const void *)p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(volatile int *p, int v)
{
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)p)), "r"(v) : "memory");
}

// Thread-block clusters: the 2D line sweep hands each finished value to the CTA of
// the next line through distributed shared memory.
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size()
{
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}
// every thread of every CTA of the cluster arrives; memory before it is visible after it
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// the shared::cluster address of this CTA's shared address `a` in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_map(unsigned a, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(unsigned a, double v)
{
    asm volatile("st.relaxed.cluster.shared::cluster.b64 [%0], %1;" ::"r"(a), "l"(__double_as_longlong(v)) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned a, float v)
{
    asm volatile("st.relaxed.cluster.shared::cluster.b32 [%0], %1;" ::"r"(a), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ void st_cluster_u64(unsigned a, unsigned long long v)
{
    asm volatile("st.relaxed.cluster.shared::cluster.b64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

// Bounded spin until a shared counter reaches `need`: tight polls first (the
// producer is a warp of this CTA a few hundred cycles away), then sleeps.
__device__ __forceinline__ bool wait_count(const volatile int *c, int need, const volatile int *abort_flag, int *err,
                                           long long budget)
{
    if (*c >= need) return true;
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (*c >= need) return true;
        if (it >= 64) __nanosleep(32);
        if ((it & 15) == 15) {
            if (*abort_flag) return false;
            if (clock64() - t0 > budget) {
                set_err(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

// SW_D: factor ring depth (rows in flight per line), a compile-time constant so
// that slot indices are cheap; 6, or 4 where the rows are too long for 6
template <typename V, typename AT, int DIR, int SW_D>
__global__ void __launch_bounds__(32 * (SW_MAXB + SW_HELP), 1) k_sweep(const __grid_constant__ SweepArgs A)
{
    if (A.done && *A.done) return;
    const StencilGeo G = A.G;
    const int n1 = G.n1, w = G.w, B = A.B, RL = A.RL;
    const int nslot = G.Sc;
    extern __shared__ __align__(128) unsigned char smem[];
    const SweepSmem Lo = sweep_layout(n1, w, B, SW_D, RL, (int)sizeof(V), nslot, (int)sizeof(AT));
    const int RS = Lo.RS, PADL = Lo.PADL;
    int *rowoff = (int *)(smem + Lo.rowoff);
    AT *sy = (AT *)(smem + Lo.sy);
    AT *srhs = (AT *)(smem + Lo.srhs);
    V *ring = (V *)(smem + Lo.ring);
    uint64_t *mbar = (uint64_t *)(smem + Lo.mbar);
    unsigned *meta = (unsigned *)(smem + Lo.meta);
    __shared__ volatile int s_abort;
    __shared__ volatile int s_prog[SW_MAXB];  // positions finished by each line of the band
    __shared__ volatile int s_near;           // positions of the line before the band staged in shared memory
    __shared__ volatile int s_far;            // ... of every older halo line (minimum)
    __shared__ int s_fresh[2];                // slots of the two newest dependencies (own line, previous line)
    __shared__ long long sband;
    __shared__ int s_issued[SW_MAXB];         // factor rows the producer issued per line (this band)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int role = wid - B;  // < 0: compute warp; 0: TMA producer; 1: halo loader; 2: publisher
    const AT *rhs = (const AT *)A.rhs;
    AT *out = (AT *)A.out;
    const V *F = (const V *)A.F;
    constexpr int CE = 16 / (int)sizeof(AT);
    const bool regpath = G.d < 3 && nslot <= 32 * SW_KS;

    for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
        int s = DIR > 0 ? t : G.Sc + 1 + t;
        int dx, dy, dz;
        slot_offsets(G, s, dx, dy, dz);
        meta[t] = (unsigned)(dx + 128) | ((unsigned)(dy + 128) << 8) | ((unsigned)(dz + 128) << 16);
        // in sweep order the newest dependencies of a row are the previous position of
        // its own line and position +w of the previous line
        if (dx == -DIR && dy == 0 && dz == 0) s_fresh[0] = t;
        if (G.d >= 2 && dx == DIR * w && dy == -DIR && dz == 0) s_fresh[1] = t;
    }
    if (threadIdx.x == 0) {
        if (G.d < 2) s_fresh[1] = -1;
        for (int i = 0; i < B * SW_D; ++i) mbar_init(&mbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    unsigned phase = 0;  // compute warps: expected parity of each ring slot (bit s)
    int consumed_rows = 0;
    bool last_ok = true;
    const long long nb = (G.nlines + B - 1) / B;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            sband = atomicAdd(A.counter, 1u);
            for (int b = 0; b < SW_MAXB; ++b) s_prog[b] = 0, s_issued[b] = 0;
            s_near = 0;
            s_far = 0;
            s_abort = (*(volatile int *)A.err != 0) ? 1 : 0;
        }
        __syncthreads();
        const long long band = sband;
        if (band >= nb) return;
        const long long v0 = band * B;
        const int nbl = (int)min((long long)B, G.nlines - v0);
        // row buffers: rows 0..w-1 hold the halo (virtual lines v0-w..v0-1), rows
        // w..w+B-1 the band; position q of a row sits at rowoff[row] + q, aligned
        // like the line in global memory so 16-byte copies land on 16-byte boundaries
        if (threadIdx.x < w + B) {
            long long vl = v0 - w + threadIdx.x;
            int shift = 0;
            if (vl >= 0 && vl < G.nlines) {
                long long gl = DIR > 0 ? vl : G.nlines - 1 - vl;
                shift = (int)((gl * (long long)n1) % CE);
            }
            rowoff[threadIdx.x] = threadIdx.x * RS + PADL + shift;
        }
        for (int e = threadIdx.x; e < (w + B) * RS; e += blockDim.x) sy[e] = AT(0);
        const bool aborted = s_abort != 0;
        if (role < 0 && wid < nbl && !aborted) {
            const long long line = DIR > 0 ? v0 + wid : G.nlines - 1 - (v0 + wid);
            for (int q = lane; q < n1; q += 32) srhs[wid * n1 + q] = rhs[q + (long long)n1 * line];
        }
        if (threadIdx.x == 0 && v0 == 0) s_near = n1, s_far = n1;  // the first band has no halo
        __syncthreads();

        if (role == 0) {
            // -------------------------------------------------------------- TMA producer
            // row q of line b goes to ring slot q % D once row q - D (same slot) is no
            // longer read, i.e. once the line has finished position q - D
            if (lane == 0 && !aborted) {
                const unsigned rowbytes = (unsigned)(RL * sizeof(V));
                int q[SW_MAXB];
                for (int b = 0; b < SW_MAXB; ++b) q[b] = (b < nbl) ? 0 : n1;
                const long long t0 = clock64();
                for (int it = 0;; ++it) {
                    if (s_abort) break;
                    bool all = true, any = false;
                    for (int b = 0; b < nbl; ++b) {
                        const int fin = s_prog[b];
                        __threadfence_block();
                        const long long line = DIR > 0 ? v0 + b : G.nlines - 1 - (v0 + b);
                        while (q[b] < n1 && q[b] - SW_D + 1 <= fin) {
                            if (!any) fence_proxy_async();
                            any = true;
                            const int p = q[b];
                            const int ii = DIR > 0 ? p : n1 - 1 - p;
                            uint64_t *bar = &mbar[b * SW_D + p % SW_D];
                            mbar_expect_tx(bar, rowbytes);
                            tma_load(ring + ((size_t)b * SW_D + p % SW_D) * RL, F + (ii + (long long)n1 * line) * RL,
                                     rowbytes, bar);
                            ++q[b];
                        }
                        all = all && q[b] >= n1;
                    }
                    if (all) break;
                    if (!any) {
                        if (it > 64) __nanosleep(32);
                        if (clock64() - t0 > 4 * A.budget) {
                            set_err(A.err, DERR_TIMEOUT);
                            break;
                        }
                    }
                }
                for (int b = 0; b < nbl; ++b) s_issued[b] = q[b];
            }
        } else if (role == 1) {
            // -------------------------------------------------------------- halo loader
            // lane h-1 stages virtual line v0-h: copies every 16-byte chunk whose
            // positions of that line are finished (progress acquired from global
            // memory), waits for the copies, then publishes how far the nearest line
            // and the older ones are staged
            // a line of another plane (3D) is no neighbour of the band's first line: it is
            // neither staged nor waited for (its slots carry zero factors)
            const bool hl = lane < w && (v0 - 1 - lane) >= 0 && (v0 - 1 - lane) / n1 == v0 / n1 && !aborted;
            const long long hv = v0 - 1 - lane;
            const long long hline = hl ? (DIR > 0 ? hv : G.nlines - 1 - hv) : 0;
            long long hchunk = 0;
            int hvis = hl ? 0 : n1;
            if (hl) hchunk = (DIR > 0 ? hline * n1 : hline * n1 + n1 - 1) / CE;
            AT *hrow = sy + (hl ? rowoff[w - 1 - lane] : 0);
            const long long lo = hline * n1, hi = lo + n1 - 1;
            const long long t0 = clock64();
            bool live = v0 > 0 && !aborted;
            for (int it = 0; live; ++it) {
                if (hvis < n1) {
                    const unsigned P = ld_acquire(A.gprog + hline);
                    for (;;) {
                        long long e0 = hchunk * CE, e1 = e0 + CE - 1;
                        int q_first = (int)(max(e0, lo) - lo), q_last = (int)(min(e1, hi) - lo);
                        int vend = DIR > 0 ? q_last + 1 : n1 - q_first;
                        if (vend > (int)P || hvis >= n1) break;
                        AT *dst = hrow + (int)(e0 - lo);
                        if (e0 >= lo && e1 <= hi) {
                            cp_async16(dst, out + e0);
                        } else {
                            // a chunk that straddles the line's ends: copy only this line's
                            // elements, so the padding stays zero (a neighbour's stale value
                            // could be NaN, and 0 * NaN would poison a dot product)
                            for (long long e = max(e0, lo); e <= min(e1, hi); ++e) dst[e - e0] = __ldcg(out + e);
                        }
                        hvis = vend;
                        hchunk += DIR;
                    }
                }
                cp_async_commit();
                cp_async_wait<0>();
                const int near = __shfl_sync(0xffffffffu, hvis, 0);
                const int far = (int)__reduce_min_sync(0xffffffffu, (unsigned)(lane == 0 ? n1 : hvis));
                if (lane == 0) {
                    __threadfence_block();
                    s_far = far;
                    s_near = near;
                }
                if (near >= n1 && far >= n1) break;
                if (it > 32) __nanosleep(32);
                // warp-uniform exits (the loop uses full-warp collectives)
                if (__any_sync(0xffffffffu, s_abort != 0)) break;
                if (__any_sync(0xffffffffu, clock64() - t0 > 4 * A.budget)) {
                    if (lane == 0) set_err(A.err, DERR_TIMEOUT);
                    break;
                }
            }
        } else if (role == 2) {
            // -------------------------------------------------------------- publisher
            // copies each line's finished positions to global memory and releases its
            // progress word; every pass publishes whatever the lines finished meanwhile
            const bool mine = lane < nbl;
            const long long line = DIR > 0 ? v0 + lane : G.nlines - 1 - (v0 + lane);
            int pub = 0;
            bool finished = !mine;
            const long long t0 = clock64();
            for (int it = 0; !__all_sync(0xffffffffu, finished); ++it) {
                const bool ab = s_abort != 0;
                const int fin = (mine && !finished) ? (ab ? n1 : s_prog[lane]) : 0;
                __threadfence_block();
                bool moved = false;
                if (mine && !finished && fin > pub) {
                    if (!ab) {
                        const int row = rowoff[w + lane];
                        for (; pub < fin; ++pub) {
                            const int i = DIR > 0 ? pub : n1 - 1 - pub;
                            out[i + (long long)n1 * line] = sy[row + i];
                        }
                    }
                    pub = fin;
                    moved = true;
                }
                if (__any_sync(0xffffffffu, moved)) {
                    __threadfence();
                    if (moved) st_release(A.gprog + line, (unsigned)pub);
                    if (moved && pub == n1) finished = true;
                } else {
                    if (it > 64) __nanosleep(32);
                    if (clock64() - t0 > 4 * A.budget) {  // the compute warps' waits are bounded
                        set_err(A.err, DERR_TIMEOUT);
                        finished = true;
                    }
                }
            }
        } else {
            // -------------------------------------------------------------- compute warp
            // Position q of the line: y_q = (r_q - S_q - l_own y_{q-1} - l_prev y'_{q+w}) [/ U_qq],
            // where S_q (every other term of the row) is computed one position ahead,
            // while the line waits for y_{q-1} and the previous line's y'_{q+w}.
            const int b = wid;
            const bool live = b < nbl;
            const long long v = v0 + b;
            const long long line = DIR > 0 ? v : G.nlines - 1 - v;
            const int j = (G.d >= 2 && live) ? (int)(line % n1) : 0;
            const int k = (G.d == 3 && live) ? (int)(line / n1) : 0;
            const int kv = DIR > 0 ? k : n1 - 1 - k;
            const int jv = DIR > 0 ? j : n1 - 1 - j;
            long long vplane = -1;
            if (live && G.d == 3 && kv >= 1) vplane = (long long)min(jv + w, n1 - 1) + (long long)n1 * (kv - 1);
            const long long plane_real = vplane < 0 ? -1 : (DIR > 0 ? vplane : G.nlines - 1 - vplane);
            unsigned seen_plane = 0;
            const int f_own = s_fresh[0], f_prev = s_fresh[1];
            const int nk = (nslot + 31) / 32;  // slots per lane
            // register-resident stencil: offset of each of this lane's slots in the row buffers
            int off[SW_KS];
            unsigned freshmask = 0;
#pragma unroll
            for (int kk = 0; kk < SW_KS; ++kk) {
                const int t = lane + 32 * kk;
                off[kk] = 0;
                if (regpath && t < nslot) {
                    const unsigned m = meta[t];
                    const int dx = (int)(m & 255u) - 128, dy = (int)((m >> 8) & 255u) - 128;
                    off[kk] = rowoff[b + w + DIR * dy] + dx;
                }
                if (t == f_own || t == f_prev) freshmask |= 1u << kk;
            }
            const V *myring = ring + (size_t)b * SW_D * RL;
            uint64_t *mybar = mbar + b * SW_D;
            const int myrow = rowoff[b + w];
            // the previous line's buffer row and the stencil offset of its newest dependency
            const int prevoff = rowoff[b + w - 1] + DIR * w;
            const volatile int *prevc = (b == 0) ? &s_near : &s_prog[b - 1];
            bool ok = live && !aborted;
            int waited = 0;  // factor rows whose ring slot this warp has waited for

            // wait until position q (sweep order) may be finished and S_{q+1} computed:
            // previous line up to q+w, older lines up to q+w+1, other planes likewise
            // the first line of a plane (3D) has no previous line in its plane: the line
            // before it in sweep order is the last of the previous plane, no neighbour
            const bool needprev = !(G.d == 3 && jv == 0);
            auto wait_deps = [&](int q) -> bool {
                const int need = needprev ? min(q + w + 1, n1) : 0, needfar = min(q + w + 2, n1);
                // fast path: every lane observes the counters with acquire loads
                bool fast = ld_acquire_cta(prevc) >= need && (b != 0 || ld_acquire_cta(&s_far) >= needfar);
                if (vplane >= 0) fast = fast && seen_plane >= (unsigned)needfar;
                if (__all_sync(0xffffffffu, fast)) return true;
                bool good = wait_count(prevc, need, &s_abort, A.err, A.budget);
                if (good && b == 0) good = wait_count(&s_far, needfar, &s_abort, A.err, A.budget);
                if (good && vplane >= 0)
                    good = wait_flag_cached(A.gprog + plane_real, (unsigned)needfar, A.err, &seen_plane, A.budget);
                good = __all_sync(0xffffffffu, good);
                __threadfence_block();
                return good;
            };
            // T_q = r_q - S_q, S_q the row's dot product without its two newest terms
            // (all lanes get it); lane 0 starts its partial sum at -r_q
            auto stale = [&](int q) -> AT {
                const int i = DIR > 0 ? q : n1 - 1 - q;
                const V *row = myring + (size_t)(q % SW_D) * RL + (DIR > 0 ? 0 : 1);
                AT acc0 = lane == 0 ? -srhs[b * n1 + i] : AT(0);
                if (regpath && nk <= 8) {
                    // up to 8 slots per lane (T <= 9 in 2D): every load is issued (predicated)
                    // before the first multiply-add; the multiply-adds stop at a warp-uniform
                    // trip count, since an FP64 instruction costs its full issue time even when
                    // every lane is predicated off
                    V fv[8];
                    AT yv[8];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int t0 = lane + 32 * kk;
                        const bool use = kk < nk && t0 < nslot && !(freshmask >> kk & 1u);
                        fv[kk] = use ? row[t0] : V(0);
                        yv[kk] = use ? sy[off[kk] + i] : AT(0);
                    }
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        if (kk >= nk) break;
                        acc0 += (AT)fv[kk] * yv[kk];
                    }
                } else if (regpath) {
#pragma unroll
                    for (int kk = 0; kk < SW_KS; ++kk) {
                        if (kk >= nk) break;
                        const int t0 = lane + 32 * kk;
                        if (t0 < nslot && !(freshmask >> kk & 1u)) acc0 += (AT)row[t0] * sy[off[kk] + i];
                    }
                } else {
                    // 8 (FP64) or 12 slots per lane at a time: all their loads are issued before the
                    // first multiply-add, so the L2 latency of the other planes' values is
                    // paid once per group rather than once per slot
                    constexpr int G8 = sizeof(AT) == 8 ? 8 : 12;
                    for (int t0 = lane; t0 < nslot; t0 += 32 * G8) {
                        AT yv[G8];
                        V fv[G8];
#pragma unroll
                        for (int u = 0; u < G8; ++u) {
                            if ((t0 - lane) + 32 * u >= nslot) break;  // warp-uniform
                            const int t = t0 + 32 * u;
                            yv[u] = AT(0);
                            fv[u] = V(0);
                            if (t >= nslot || t == f_own || t == f_prev) continue;
                            const unsigned m = meta[t];
                            const int dx = (int)(m & 255u) - 128, dy = (int)((m >> 8) & 255u) - 128,
                                      dz = (int)((m >> 16) & 255u) - 128;
                            const int ci = i + dx, cj = j + dy, ck = k + dz;
                            if (ci < 0 || ci >= n1 || cj < 0 || cj >= n1 || ck < 0 || ck >= n1) continue;
                            fv[u] = row[t];
                            yv[u] = dz == 0 ? sy[rowoff[b + w + DIR * dy] + ci]
                                            : __ldcg(out + ci + (long long)n1 * (cj + (long long)n1 * ck));
                        }
#pragma unroll
                        for (int u = 0; u < G8; ++u) {
                            if ((t0 - lane) + 32 * u >= nslot) break;  // warp-uniform: no idle FP64 issue
                            acc0 += (AT)fv[u] * yv[u];
                        }
                    }
                }
                return -warp_sum(acc0);
            };
            auto wait_row = [&](int q) -> bool {
                const int slot = q % SW_D;
                bool good = mbar_wait(&mybar[slot], (phase >> slot) & 1u, A.err, A.budget);
                phase ^= 1u << slot;
                ++waited;
                return __all_sync(0xffffffffu, good);
            };

            // T = r_q - S_q of the next position; yprev = y_{q-1}; lo, lp, ri: the factors of
            // the two newest terms and 1 / U(i,i) of the next position (read ahead by lane 0)
            AT T = 0, yprev = 0, lo = 0, lp = 0, ri = 1;
            auto fresh_factors = [&](int q) {
                if (lane == 0) {
                    const V *row = myring + (size_t)(q % SW_D) * RL + (DIR > 0 ? 0 : 1);
                    lo = (AT)row[f_own];
                    lp = f_prev >= 0 ? (AT)row[f_prev] : AT(0);
                    if (DIR < 0) ri = (AT)row[RL - 2];  // 1 / U(i,i), stored by the factorisation
                }
            };
            if (ok) ok = wait_deps(-1) && wait_row(0);
            if (ok) {
                T = stale(0);
                fresh_factors(0);
            }
            int q = 0;
            for (; q < n1 && ok; ++q) {
                const int i = DIR > 0 ? q : n1 - 1 - q;
                // the own-line term is known before the previous line's value arrives
                const AT t = T - lo * yprev;
                ok = wait_deps(q);
                if (!ok) break;
                if (lane == 0) {
                    AT val = t - lp * sy[prevoff + i];
                    if (DIR < 0) val = val * ri;
                    sy[myrow + i] = val;
                    yprev = val;
                    st_release_cta(&s_prog[b], q + 1);
                }
                __syncwarp();
                if (q + 1 < n1) {
                    if (!wait_row(q + 1)) {
                        ok = false;
                        break;
                    }
                    T = stale(q + 1);
                    fresh_factors(q + 1);
                }
            }
            if (live && !ok && lane == 0) s_abort = 1;
            consumed_rows = waited;
            last_ok = ok || !live;
        }
        // after an abort, wait (bounded) for factor rows the producer issued but this
        // warp did not consume, so no bulk copy lands in shared memory after the band
        __syncthreads();
        if (role < 0 && !last_ok && wid < nbl) {
            for (int pp = consumed_rows; pp < s_issued[wid]; ++pp) {
                const int slot = pp % SW_D;
                mbar_wait(&mbar[wid * SW_D + slot], (phase >> slot) & 1u, A.err);
                phase ^= 1u << slot;
            }
        }
    }
}

// ============================================================================
// Line-parallel sweep (1D, 2D and 3D): one line per CTA, a position's work
// split over warps.
//
// In k_sweep the warp of a line computes each row's whole dot product between
// two of its positions, so a position costs a full FP64 reduction (~1 us) and a
// 2D sweep, a chain of about n1 (w+1) + n1 positions, keeps only ~n1/(w+1) lines
// busy at a time.  Here a CTA owns one line:
//   * L1_NS stale warps (L1_NS3 in 3D) compute T_q = r_q - (every term of row q
//     except the K newest values of the own line and the K newest of the previous
//     line), position q by the warp of index q modulo their count, K positions
//     ahead of the finisher;
//   * the finisher holds the window of the next K positions in its lanes
//     (lane j: position s+j) and applies each new value -- y_{s-1} of the own
//     line, y'_{s+w} of the previous one -- to the whole window with one
//     multiply-add, so finishing a position is one addition (T_s), two
//     multiply-adds and, backward, the multiply by the stored 1 / U(i,i);
//   * a TMA producer streams the line's factor rows into a ring of D rows;
//   * two loader warps stage the w lines before this one (of its own plane, in
//     3D) into shared memory straight from the output vector, where the
//     finisher stores each value.  The output is filled with a signalling NaN
//     before the sweep and every value is stored once, so a word that differs
//     from the fill is final: no progress words, no fences.  (Arithmetic never
//     produces a signalling NaN.)  In 3D the stale warps read the other planes'
//     values from the output the same way, through L1.
// Lines are claimed in sweep order, so a CTA only waits for lines claimed
// earlier by running CTAs; every wait is bounded and reports LSG_ERR_TIMEOUT.
constexpr int L1_NS = 6;                 // stale warps in 1D/2D
constexpr int L1_NS3 = 9;                // ... in 3D, where their sums (other planes' values read through L1) bound the step
constexpr int L1_DT = 32;                // ring of stale results (positions)
// warps per CTA (a template parameter): 12 in 1D/2D (finisher, six stale warps, TMA producer, two
// loaders, two idle), 16 in 3D (three more stale warps: at 512 threads the register cap of 128
// per thread slowed the 2D finisher's step by 16 %, while 3D gains 16 %)
constexpr int L1_WARPS2 = 12, L1_WARPS3 = 16;
constexpr int L1_CLUSTER = 8;            // 2D: lines per cluster group (one per CTA)
constexpr int L1_D = 32;                 // factor ring depth (rows); rows D further ahead are prefetched to L2
constexpr int L1_CH = 4;                 // rows per ring barrier (the finisher checks one per L1_CH positions)
constexpr int L1_DM = 16;                // ring depth where 32 rows do not fit (3D FP64 rows of T <= 4)
constexpr int L1_DS = 8;                 // ... where 16 do not fit either
constexpr int L1_FB = 16;                // finisher steps per block (ring waits at block starts)

template <typename AT>
struct Fill;
template <>
struct Fill<double> {
    using bits = unsigned long long;
    static constexpr bits v = 0x7FF4A5A5A5A5A5A5ull;
    __device__ static double val(bits b) { return __longlong_as_double((long long)b); }
};
template <>
struct Fill<float> {
    using bits = unsigned;
    static constexpr bits v = 0x7FA5A5A5u;
    __device__ static float val(bits b) { return __uint_as_float(b); }
};
__device__ __forceinline__ unsigned long long ld_poll(const double *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_poll(const float *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// L1-cached read of a value that is written once: a copy that differs from the
// fill pattern is the final value.
__device__ __forceinline__ unsigned long long ld_cached(const double *p)
{
    return __ldca(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ unsigned ld_cached(const float *p) { return __ldca(reinterpret_cast<const unsigned *>(p)); }
__device__ __forceinline__ void st_final(double *p, double v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(v)) : "memory");
}
__device__ __forceinline__ void st_final(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(v)) : "memory");
}

// Shared-memory accesses by 32-bit shared address (the finisher's hot loop).
__device__ __forceinline__ unsigned long long lds_vol(unsigned a, unsigned long long)
{
    unsigned long long v;
    asm volatile("ld.volatile.shared.b64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned lds_vol(unsigned a, unsigned)
{
    unsigned v;
    asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_vol(unsigned a, unsigned long long v)
{
    asm volatile("st.volatile.shared.b64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void sts_vol(unsigned a, unsigned v)
{
    asm volatile("st.volatile.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ double lds_val(unsigned a, double)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_val(unsigned a, float)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_val(unsigned a, double v) { asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory"); }
__device__ __forceinline__ void sts_val(unsigned a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory"); }

// Fills the output of one sweep with the signalling NaN and resets its line counter.
template <typename AT>
__global__ void k_line_fill(AT *out, long long n, unsigned *counter, const int *done)
{
    if (done && *done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0u;
    typename Fill<AT>::bits *o = reinterpret_cast<typename Fill<AT>::bits *>(out);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        o[e] = Fill<AT>::v;
}

struct LineSmem {
    size_t sy, srhs, sT, ring, mbar, meta, tab, total;
    int RS, PADL, rows;  // row stride, left padding (elements), value rows (halo + own line)
};

__host__ __device__ inline LineSmem line_layout(int d, int n1, int w, int D, int RL, int vsize, int nslot, int asize)
{
    LineSmem L;
    L.PADL = (w + 1) / 2 * 2;                 // positions -w .. -1 (even: 16-byte row starts)
    L.RS = (L.PADL + n1 + w + 1) / 2 * 2;     // ... n1 .. n1+w-1 on the right
    L.rows = d >= 2 ? w + 1 : 1;
    size_t o = 0;
    L.sy = o;   o += (size_t)L.rows * L.RS * asize;
    L.srhs = o; o += (size_t)n1 * asize;
    o = (o + 15) / 16 * 16;
    L.sT = o;   o += (size_t)L1_DT * asize;
    o = (o + 127) / 128 * 128;
    L.ring = o; o += (size_t)D * RL * vsize;
    o = (o + 7) / 8 * 8;
    L.mbar = o; o += (size_t)D * 8;
    L.meta = o; o += (size_t)nslot * 4;
    o = (o + 7) / 8 * 8;
    L.tab = o;  o += d == 3 ? (size_t)nslot * 8 : 0;  // 3D: per-line slot table
    L.total = o;
    return L;
}

// Bounded spin until a shared counter reaches `need`; every lane polls with
// acquire loads and the result is warp-uniform.
__device__ __forceinline__ bool wait_ge(const volatile int *c, int need, const volatile int *abort_flag, int *err,
                                        long long budget)
{
    bool good = true;
    if (ld_acquire_cta(c) < need) {
        const long long t0 = clock64();
        for (int it = 0;; ++it) {
            if (ld_acquire_cta(c) >= need) break;
            if (it >= 256) __nanosleep(16);
            if ((it & 15) == 15) {
                if (*abort_flag) {
                    good = false;
                    break;
                }
                if (clock64() - t0 > budget) {
                    set_err(err, DERR_TIMEOUT);
                    good = false;
                    break;
                }
            }
        }
    }
    return __all_sync(0xffffffffu, good);
}

// Bounded poll of a shared word that one writer stores once over the fill
// pattern: the value itself is the flag (all lanes read the same address; the
// result is warp-uniform).
template <typename AT>
__device__ __forceinline__ bool poll_value(const AT *p, AT &val, const volatile int *abort_flag, int *err,
                                           long long budget)
{
    using bits_t = typename Fill<AT>::bits;
    const volatile bits_t *vp = reinterpret_cast<const volatile bits_t *>(p);
    bits_t b = *vp;
    bool good = true;
    if (b == Fill<AT>::v) {
        const long long t0 = clock64();
        for (int it = 0;; ++it) {
            b = *vp;
            if (b != Fill<AT>::v) break;
            if (it >= 256) __nanosleep(16);
            if ((it & 15) == 15) {
                if (*abort_flag) {
                    good = false;
                    break;
                }
                if (clock64() - t0 > budget) {
                    set_err(err, DERR_TIMEOUT);
                    good = false;
                    break;
                }
            }
        }
    }
    val = Fill<AT>::val(b);
    return __all_sync(0xffffffffu, good);
}

// Bounded poll of a value of another CTA's line in global memory (final once it
// differs from the fill pattern); per lane, no warp collectives.
template <typename AT>
__device__ __forceinline__ bool poll_global(const AT *p, AT &val, const volatile int *abort_flag, int *err,
                                            long long budget)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        const typename Fill<AT>::bits b = ld_poll(p);
        if (b != Fill<AT>::v) {
            val = Fill<AT>::val(b);
            return true;
        }
        __nanosleep(32);
        if ((it & 15) == 15) {
            if (*abort_flag || *(volatile int *)err != 0) return false;
            if (clock64() - t0 > budget) {
                set_err(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

// The finisher's rare slow path: poll the stale part and (2D/3D) the previous
// line's value until both are final.  Kept out of line so that the step loop
// holds no loop of its own; the operands travel by value (an address taken would
// keep them in local memory on every step: measured 8 % of the sweep).
template <typename AT>
struct FinOps {
    typename Fill<AT>::bits t, p;
    int good;
};
template <typename AT>
__device__ __noinline__ FinOps<AT> poll_operands(const AT *pT, const AT *pP, FinOps<AT> o, const volatile int *abort_flag,
                                                 int *err, long long budget)
{
    using bits_t = typename Fill<AT>::bits;
    bool good = true;
    const long long t0 = clock64();
    for (int it = 0; good; ++it) {
        const bool needT = o.t == Fill<AT>::v, needP = pP != nullptr && o.p == Fill<AT>::v;
        if (!needT && !needP) break;
        if (needT) o.t = *reinterpret_cast<const volatile bits_t *>(pT);
        if (needP) o.p = *reinterpret_cast<const volatile bits_t *>(pP);
        if (it >= 256) __nanosleep(16);
        if ((it & 15) == 15) {
            if (*abort_flag) {
                good = false;
            } else if (clock64() - t0 > budget) {
                set_err(err, DERR_TIMEOUT);
                good = false;
            }
        }
    }
    o.good = __all_sync(0xffffffffu, good) ? 1 : 0;
    return o;
}

// Bounded wait for an mbarrier phase that also gives up when the CTA aborts.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, unsigned parity, const volatile int *abort_flag, int *err,
                                             long long budget)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 15) {
            if (*abort_flag) return false;
            if (clock64() - t0 > budget) {
                set_err(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

template <typename V, typename AT, int DIR, int D, int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_sweep_line(const __grid_constant__ SweepArgs A)
{
    if (A.done && *A.done) return;
    using FB = Fill<AT>;
    using bits_t = typename FB::bits;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NB = D / L1_CH;  // ring barriers, one per chunk of L1_CH rows
    static_assert(D % L1_CH == 0, "ring depth must be a multiple of the chunk");
    static_assert(L1_NS == 6 && L1_NS3 == 9 && (NW == L1_WARPS2 || NW == L1_WARPS3),
                  "stale warps sit on sub-partitions 1-3, two or three each");
    const StencilGeo G = A.G;
    const int n1 = G.n1, w = G.w, RL = A.RL, nslot = G.Sc, K = A.K;
    extern __shared__ __align__(128) unsigned char smem[];
    const LineSmem Lo = line_layout(G.d, n1, w, D, RL, (int)sizeof(V), nslot, (int)sizeof(AT));
    const int RS = Lo.RS, PADL = Lo.PADL, own = Lo.rows - 1;  // value row of the own line; row own-h: line v-h
    AT *sy = (AT *)(smem + Lo.sy);
    AT *srhs = (AT *)(smem + Lo.srhs);
    AT *sT = (AT *)(smem + Lo.sT);
    V *ring = (V *)(smem + Lo.ring);
    uint64_t *mbar = (uint64_t *)(smem + Lo.mbar);
    unsigned *meta = (unsigned *)(smem + Lo.meta);
    __shared__ volatile int s_abort;
    __shared__ volatile int s_prog;            // positions the finisher completed
    __shared__ volatile int s_near, s_near2;   // positions of lines v-1 and v-2 staged in shared memory
    __shared__ volatile int s_far;             // ... of lines v-3 .. v-w (minimum)
    __shared__ int s_fown[32], s_fprev[32];    // slots of the window's fresh terms (lane j)
    __shared__ long long s_line;
    __shared__ int s_issued;                   // chunks the producer issued (this line)
    __shared__ unsigned long long s_group;     // cluster mode: the group rank 0 claimed (all ones: stop)
    __shared__ unsigned long long s_zero8;     // zero word for the finisher's factor-less lanes
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // warp roles (warp w runs on SM sub-partition w % 4): the finisher alone on
    // sub-partition 0 (with two idle warps); the stale warps two per sub-partition 1-3,
    // with the producer, the near loader and the far loader one each (the far loader
    // polls up to eight lines without pause: beside the finisher it slowed the
    // backward sweep's step by 12 %)
    enum { R_FIN, R_STALE, R_PROD, R_NEAR, R_FAR, R_IDLE };
    // stale warps: 1, 2, 3, 5, 6, 7 (index 0-5) and, with 16 warps (3D), 13, 14, 15 (index 6-8)
    const int ns = NW == L1_WARPS3 ? L1_NS3 : L1_NS;
    const int sw = wid < 4 ? wid - 1 : wid < 8 ? wid - 2 : wid - 7;  // stale warp index (R_STALE)
    const int role = wid == 0 ? R_FIN : (wid == 4 || wid == 8 || wid == 12) ? R_IDLE : wid == 9 ? R_PROD
                   : wid == 10 ? R_NEAR : wid == 11 ? R_FAR : sw < ns ? R_STALE : R_IDLE;
    // cluster mode (2D, launched in clusters): CTA `crank` of a cluster takes line
    // csz g + crank of the group g that rank 0 claims, and stores each value it finishes
    // into the previous-line row of CTA crank + 1 as well
    const unsigned csz = cluster_size(), crank = cluster_rank();
    const bool clu = csz > 1;
    const AT *rhs = (const AT *)A.rhs;
    AT *out = (AT *)A.out;
    const V *F = (const V *)A.F;

    if (threadIdx.x < 32) s_fown[threadIdx.x] = -1, s_fprev[threadIdx.x] = -1;
    if (threadIdx.x == 0) s_zero8 = 0ull;
    __syncthreads();
    for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
        const int s = DIR > 0 ? t : G.Sc + 1 + t;
        int dx, dy, dz;
        slot_offsets(G, s, dx, dy, dz);
        meta[t] = (unsigned)(dx + 128) | ((unsigned)(dy + 128) << 8) | ((unsigned)(dz + 128) << 16);
        // in sweep order: own-line position q-m is offset dx = -DIR m; previous-line
        // position q+w-j is offset (DIR (w-j), -DIR)
        const int m = -DIR * dx, jj = w - DIR * dx;
        if (dy == 0 && dz == 0 && m >= 1 && m <= K) s_fown[m - 1] = t;
        if (G.d >= 2 && dz == 0 && dy == -DIR && jj >= 0 && jj < K) s_fprev[jj] = t;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NB; ++i) mbar_init(&mbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // chunk c (rows L1_CH c ..) lands in ring rows (L1_CH c) % D .. and completes
    // barrier c % NB; per line that barrier takes ceil((nch - b) / NB) chunks, so
    // the phase parity of row q in this CTA's line `it` is:
    const int nch = (n1 + L1_CH - 1) / L1_CH;
    auto parity = [&](int it, int q) -> unsigned {
        const int c = q / L1_CH, cnt = (nch - c % NB + NB - 1) / NB;
        return (unsigned)(((it & cnt) ^ (c / NB)) & 1);
    };
    auto wait_chunk = [&](int it, int q) -> bool {
        return __all_sync(FULL, mbar_wait_ab(&mbar[(q / L1_CH) % NB], parity(it, q), &s_abort, A.err, A.budget));
    };

    // stale warps: register-resident stencil offsets (row buffers of this CTA) and
    // the window's slots among this lane's (bit kk: slot lane + 32 kk)
    const int nk = (nslot + 31) / 32;
    int off[SW_KS];
    unsigned freshmask = 0;
    if (role == R_STALE) {
#pragma unroll
        for (int kk = 0; kk < SW_KS; ++kk) {
            const int t = lane + 32 * kk;
            off[kk] = 0;
            if (t < nslot) {
                const unsigned m = meta[t];
                const int dx = (int)(m & 255u) - 128, dy = (int)((m >> 8) & 255u) - 128;
                off[kk] = (own + DIR * dy) * RS + PADL + dx;
            }
        }
        for (int kk = 0; kk < SW_KS && kk < nk; ++kk) {
            const int t = lane + 32 * kk;
            for (int f = 0; f < K; ++f)
                if (t == s_fown[f] || t == s_fprev[f]) freshmask |= 1u << kk;
        }
    }

    for (int it = 0;;) {
        __syncthreads();
        if (clu) {
            // every CTA of the cluster is done with the previous group, so none stores into
            // another's rows any more; rank 0 claims the next group for all (stop: past the
            // last line, or an error anywhere)
            cluster_sync_all();
            if (crank == 0 && threadIdx.x == 0) {
                const unsigned long long g = atomicAdd(A.counter, 1u);
                const bool stop = (long long)g * csz >= G.nlines || *(volatile int *)A.err != 0;
                for (unsigned r = 0; r < csz; ++r) st_cluster_u64(cluster_map(smem_u32(&s_group), r), stop ? ~0ull : g);
            }
            cluster_sync_all();
            if (s_group == ~0ull) return;  // all CTAs of the cluster alike; nothing in flight
        }
        if (threadIdx.x == 0) {
            s_line = clu ? (long long)s_group * csz + crank : (long long)atomicAdd(A.counter, 1u);
            s_prog = 0;
            s_near = 0;
            s_near2 = 0;
            s_far = 0;
            s_issued = 0;
            s_abort = (*(volatile int *)A.err != 0) ? 1 : 0;
        }
        __syncthreads();
        const long long v = s_line;
        if (!clu && (v >= G.nlines || s_abort)) return;  // no copy is in flight between lines
        // cluster mode: a CTA past the last line sits the group out (the next claim stops)
        const bool live = v < G.nlines && !s_abort;
        const long long line = DIR > 0 ? v : G.nlines - 1 - v;
        // the finisher polls the values of line v-1 and the stale results for the
        // fill pattern; everything else starts at zero (padding, absent lines)
        // index of the line within its plane in sweep order: lines of another plane are
        // no neighbours of this one (3D) and are neither staged nor waited for
        const long long vin = G.d == 3 ? v % n1 : v;
        const bool prev_exists = G.d >= 2 && vin >= 1;
        bits_t *ybits = reinterpret_cast<bits_t *>(sy);
        for (int e = threadIdx.x; e < Lo.rows * RS; e += blockDim.x) {
            const int r = e / RS, c = e - r * RS - PADL;
            ybits[e] = (prev_exists && r == own - 1 && c >= 0 && c < n1) ? FB::v : bits_t(0);
        }
        for (int e = threadIdx.x; e < L1_DT; e += blockDim.x) reinterpret_cast<bits_t *>(sT)[e] = FB::v;
        if (live)
            for (int q = threadIdx.x; q < n1; q += blockDim.x) srhs[q] = rhs[q + (long long)n1 * line];
        if (G.d == 3) {
            // the line's slot table: each slot of the stale part that can be in the grid
            // for some position, with the offset of its value from position i (in the
            // output relative to this line, or in the row buffers) and dx for the one
            // check that depends on the position; window slots and slots whose line
            // is outside the grid are dropped (x = dx + 64 < 0 marks them)
            const int lj = (int)(line % n1), lk = (int)(line / n1);
            int2 *tab = reinterpret_cast<int2 *>(smem + Lo.tab);
            for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
                const unsigned m = meta[t];
                const int dx = (int)(m & 255u) - 128, dy = (int)((m >> 8) & 255u) - 128, dz = (int)((m >> 16) & 255u) - 128;
                const int om = -DIR * dx, oj = w - DIR * dx;
                const bool win = dz == 0 && ((dy == 0 && om >= 1 && om <= K) || (dy == -DIR && oj >= 0 && oj < K));
                const int cj = lj + dy, ck = lk + dz;
                int2 e;
                if (win || cj < 0 || cj >= n1 || ck < 0 || ck >= n1) {
                    e = make_int2(0, -1);
                } else if (dz == 0) {
                    e = make_int2((own + DIR * dy) * RS + PADL + dx, (dx + 64) | (1 << 8));
                } else {
                    e = make_int2(dx + n1 * (dy + n1 * dz), dx + 64);
                }
                tab[t] = e;
            }
        }
        if (threadIdx.x == 0) {
            // lines before the first one, and lines of 1D problems, do not exist
            if (G.d < 2 || vin < 1) s_near = n1;
            if (G.d < 2 || vin < 2) s_near2 = n1;
            if (G.d < 2 || vin < 3 || w < 3) s_far = n1;
        }
        // cluster mode: every row is filled before a neighbour stores into it
        if (clu)
            cluster_sync_all();
        else
            __syncthreads();
        bool ok = true;

        if (!live) {
            // past the last line (cluster mode): nothing to do in this group
        } else if (role == R_FIN) {
            // ---------------------------------------------------------------- finisher
            const int j = lane;
            const int fo_t = j < K ? s_fown[j] : -1, fp_t = j < K ? s_fprev[j] : -1;
            const int myrow = own * RS + PADL;
            const int prevoff = G.d >= 2 ? (own - 1) * RS + PADL + DIR * w : 0;
            // lane j holds Gw, the fresh part of position s+j so far; yb = y_{s-1}.  The
            // window starts K-1 steps before position 0 so that every position receives
            // its K newest previous-line values here (steps s < 0 only apply those).
            AT Gw = 0, yb = 0;
            const int s0 = -(K - 1);
            if (n1 > 0) ok = wait_chunk(it, 0);
            // operands of the next step, loaded at the end of the previous one so that
            // their latency overlaps the shuffles: the window's factors, the stale part
            // and the previous line's value (zero past the line's ends; both are final
            // once they differ from the fill)
            AT fo = 0, fp = 0, ri = 1;
            // shared addresses: this lane's factor slots in ring row 0, the stale ring,
            // the previous line's row (at position 0) and the own row
            const unsigned a_ring = smem_u32(ring) + (unsigned)((DIR > 0 ? 0 : 1) * (int)sizeof(V));
            const unsigned a_fo = a_ring + (unsigned)(max(fo_t, 0) * (int)sizeof(V));
            const unsigned a_fp = a_ring + (unsigned)(max(fp_t, 0) * (int)sizeof(V));
            const unsigned a_ri = a_ring + (unsigned)((RL - 2) * (int)sizeof(V));
            const unsigned rowb = (unsigned)(RL * (int)sizeof(V));
            const unsigned a_T = smem_u32(sT), a_P = smem_u32(sy + prevoff), a_Y = smem_u32(sy + myrow);
            // cluster mode: the next line's CTA reads this line's values from its own
            // previous-line row, which lane 0 fills as well
            const bool fwd = clu && crank + 1 < csz && v + 1 < G.nlines;
            const unsigned a_next = fwd ? cluster_map(smem_u32(sy + (own - 1) * RS + PADL), crank + 1) : 0u;
            auto load_factors = [&](int s) {
                const int qj = s + j;
                const bool in = j < K && qj >= 0 && qj < n1;
                const unsigned ro = (unsigned)(qj & (D - 1)) * rowb;
                // every lane loads, from a zero word where it has no factor: a conditional
                // inline-asm load would be a divergent branch in the step loop
                fo = (AT)lds_val((in && fo_t >= 0) ? a_fo + ro : smem_u32(&s_zero8), V(0));
                fp = (AT)lds_val((in && fp_t >= 0) ? a_fp + ro : smem_u32(&s_zero8), V(0));
                // 1 / U(i,i), stored by the factorisation (only lane 0's is used, and only at
                // positions in the line)
                if (DIR < 0) ri = (AT)lds_val(a_ri + ro, V(0));
            };
            auto load_T = [&](int s) -> bits_t {
                return s >= 0 ? lds_vol(a_T + (unsigned)((s % L1_DT) * (int)sizeof(AT)), bits_t(0)) : bits_t(0);
            };
            auto load_P = [&](int s) -> bits_t {
                return (G.d >= 2 && s + w >= 0)
                           ? lds_vol(a_P + (unsigned)((DIR > 0 ? s : n1 - 1 - s) * (int)sizeof(AT)), bits_t(0))
                           : bits_t(0);
            };
            bits_t tb = 0, pb = 0;
            auto next_operands = [&](int s) {  // the window's factors, the stale part, the previous line's value
                load_factors(s);
                tb = load_T(s);
                pb = load_P(s);
            };
            // ring chunks the finisher has waited for: rows [0, rows_ok) have landed
            int rows_ok = 0;
            auto need_rows = [&](int upto) -> bool {  // wait for the chunks of rows < upto
                upto = min(upto, n1);
                bool good = true;
                while (good && rows_ok < upto) {
                    good = wait_chunk(it, rows_ok);
                    rows_ok += L1_CH;
                }
                return good;
            };
            // steps before position 0: previous-line values only
            ok = ok && need_rows(K);
            if (ok) next_operands(s0);
            for (int s = s0; s < 0 && ok; ++s) {
                AT yp = FB::val(pb);
                if (pb == FB::v) ok = poll_value(&sy[prevoff + (DIR > 0 ? s : n1 - 1 - s)], yp, &s_abort, A.err, A.budget);
                if (!ok) break;
                const AT r = fma(-fp, yp, Gw);
                Gw = __shfl_down_sync(FULL, r, 1);
                if (j >= K - 1) Gw = AT(0);
                next_operands(s + 1);
            }
            // Bv: the stale part and the previous line's value of the step (lane 0 adds
            // T_s), computed from operands read one step ahead, off the loop-carried chain;
            // an operand that is not final yet (rare) is polled outside the hot loop's code
            AT Bv = 0;
            auto make_B = [&](int s) -> bool {
                if (__any_sync(FULL, tb == FB::v || pb == FB::v)) {
                    const FinOps<AT> o =
                        poll_operands(&sT[s % L1_DT], G.d >= 2 ? &sy[prevoff + (DIR > 0 ? s : n1 - 1 - s)] : nullptr,
                                      FinOps<AT>{tb, pb, 1}, &s_abort, A.err, A.budget);
                    if (!o.good) return false;
                    tb = o.t;
                    pb = o.p;
                }
                Bv = fma(-fp, FB::val(pb), (j == 0) ? FB::val(tb) : AT(0));
                return true;
            };
            if (ok && n1 > 0) ok = make_B(0);
            // blocks of fb steps: the ring chunks a block reads (its windows and the next
            // step's operands: rows < sb + fb + K) are waited for at its start, so that the
            // steps themselves carry no such branch; the ring holds rows up to D-1 past the
            // finisher's position, hence fb <= D - K
            const int fb = min(L1_FB, D - K);
            for (int sb = 0; sb < n1 && ok; sb += fb) {
                ok = need_rows(sb + fb + K);
                const int se = min(sb + fb, n1);
                for (int s = sb; s < se && ok; ++s) {
                    const int i = DIR > 0 ? s : n1 - 1 - s;
                    // the chain: add, multiply-add by y_{s-1}; the next step's operands are
                    // read while it completes
                    const AT r = fma(-fo, yb, Gw + Bv);
                    const AT val = DIR < 0 ? r * ri : r;
                    const bool more = s + 1 < n1;
                    if (more) next_operands(s + 1);
                    yb = __shfl_sync(FULL, val, 0);
                    Gw = __shfl_down_sync(FULL, r, 1);
                    if (j >= K - 1) Gw = AT(0);
                    // every lane has read this step's stale slot (the shuffle synchronises
                    // the warp): refill it, then publish y_s (all lanes store the same value)
                    sts_vol(a_T + (unsigned)((s % L1_DT) * (int)sizeof(AT)), FB::v);
                    sts_val(a_Y + (unsigned)(i * (int)sizeof(AT)), yb);
                    st_release_cta(&s_prog, s + 1);
                    // and to the next line's CTA and the output (after the release: its fence
                    // does not wait for these stores); every lane stores the same value, one
                    // transaction each, with no divergent branch
                    if (fwd) st_cluster(a_next + (unsigned)(i * (int)sizeof(AT)), yb);
                    st_final(out + i + (long long)n1 * line, yb);
                    if (more) ok = make_B(s + 1);
                }
            }
        } else if (role == R_STALE) {
            // ---------------------------------------------------------------- stale warps
            // T_q = r_q - S_q, S_q every term of row q but the window's: own-line
            // positions < q-K and previous-line positions <= q+w-K are final once the
            // finisher has done q-K positions and line v-1 is staged that far
            for (int q = sw; q < n1 && ok; q += ns) {
                ok = wait_ge(&s_prog, q - K, &s_abort, A.err, A.budget) &&
                     wait_ge(&s_near, min(max(0, q + w - K + 1), n1), &s_abort, A.err, A.budget) &&
                     wait_ge(&s_near2, min(q + w + 1, n1), &s_abort, A.err, A.budget) &&
                     wait_ge(&s_far, min(q + w + 1, n1), &s_abort, A.err, A.budget) && wait_chunk(it, q);
                if (!ok) break;
                const int i = DIR > 0 ? q : n1 - 1 - q;
                const V *row = ring + (size_t)(q % D) * RL + (DIR > 0 ? 0 : 1);
                const unsigned fm = freshmask;
                AT acc0 = lane == 0 ? -srhs[i] : AT(0);
                if (G.d == 3) {
                    // same-plane neighbours from the row buffers, the other planes' values
                    // straight from the output through L1 (a value is read by 2w+1
                    // consecutive positions; it is final once it differs from the fill, and
                    // one that is not yet -- or whose L1 copy predates it -- is polled from
                    // L2), G3 slots per lane at a time, offsets from the line's slot table
                    constexpr int G3 = sizeof(AT) == 8 ? 8 : 12;
                    const int2 *tab = reinterpret_cast<const int2 *>(smem + Lo.tab);
                    const AT *obase = out + (long long)n1 * line + i;
                    for (int t0 = lane; t0 - lane < nslot; t0 += 32 * G3) {
                        AT yv[G3];
                        V fv[G3];
                        unsigned pend = 0;
#pragma unroll
                        for (int u = 0; u < G3; ++u) {
                            yv[u] = AT(0);
                            fv[u] = V(0);
                            if ((t0 - lane) + 32 * u >= nslot) break;  // warp-uniform
                            const int t = t0 + 32 * u;
                            if (t >= nslot) continue;
                            const int2 e = tab[t];
                            const int ci = i + (e.y & 255) - 64;
                            if (e.y < 0 || ci < 0 || ci >= n1) continue;
                            fv[u] = row[t];
                            if (e.y >> 8) {
                                yv[u] = sy[e.x + i];
                            } else {
                                const bits_t bb = ld_cached(obase + e.x);
                                if (bb == FB::v) pend |= 1u << u;
                                yv[u] = FB::val(bb);
                            }
                        }
                        if (__any_sync(FULL, pend != 0)) {
                            bool good = true;
#pragma unroll
                            for (int u = 0; u < G3; ++u)
                                if (good && (pend >> u & 1u))
                                    good = poll_global(obase + tab[t0 + 32 * u].x, yv[u], &s_abort, A.err, A.budget);
                            if (!__all_sync(FULL, good)) {
                                ok = false;
                                break;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < G3; ++u) {
                            if ((t0 - lane) + 32 * u >= nslot) break;  // warp-uniform: no idle FP64 issue
                            acc0 += (AT)fv[u] * yv[u];
                        }
                    }
                    if (!ok) break;
                } else if (nk <= 8) {
                    // every load is issued before the first multiply-add; the
                    // multiply-adds stop at a warp-uniform trip count
                    V fv[8];
                    AT yv[8];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int t0 = lane + 32 * kk;
                        const bool use = kk < nk && t0 < nslot && !(fm >> kk & 1u);
                        fv[kk] = use ? row[t0] : V(0);
                        yv[kk] = use ? sy[off[kk] + i] : AT(0);
                    }
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        if (kk >= nk) break;
                        acc0 += (AT)fv[kk] * yv[kk];
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < SW_KS; ++kk) {
                        if (kk >= nk) break;
                        const int t0 = lane + 32 * kk;
                        if (t0 < nslot && !(fm >> kk & 1u)) acc0 += (AT)row[t0] * sy[off[kk] + i];
                    }
                }
                const AT T = -warp_sum(acc0);
                if (lane == 0) *reinterpret_cast<volatile AT *>(&sT[q % L1_DT]) = T;
            }
        } else if (role == R_PROD) {
            // ---------------------------------------------------------------- TMA producer
            // chunk c goes to its ring rows once the finisher has done the chunk that
            // held them (c - NB; the stale warps are done with it by then too); rows
            // up to 2D ahead are prefetched to L2, so a ring copy rarely waits for HBM
            if (lane == 0) {
                const unsigned rowbytes = (unsigned)(RL * sizeof(V));
                auto grow = [&](int q) { return F + ((DIR > 0 ? q : n1 - 1 - q) + (long long)n1 * line) * RL; };
                for (int pq = D; pq < 2 * D && pq < n1; ++pq) prefetch_l2(grow(pq), rowbytes);
                int c = 0;
                const long long t0 = clock64();
                for (int itp = 0; c < nch; ++itp) {
                    if (s_abort) break;
                    const int fin = s_prog;
                    __threadfence_block();
                    bool any = false;
                    while (c < nch && L1_CH * c - D + L1_CH <= fin) {
                        if (!any) fence_proxy_async();
                        any = true;
                        const int q0 = L1_CH * c, q1 = min(q0 + L1_CH, n1);
                        uint64_t *bar = &mbar[c % NB];
                        mbar_expect_tx(bar, (unsigned)(q1 - q0) * rowbytes);
                        for (int q = q0; q < q1; ++q) {
                            tma_load(ring + (size_t)(q % D) * RL, grow(q), rowbytes, bar);
                            if (q + 2 * D < n1) prefetch_l2(grow(q + 2 * D), rowbytes);
                        }
                        ++c;
                    }
                    if (!any) {
                        if (itp > 64) __nanosleep(32);
                        if (clock64() - t0 > 4 * A.budget) {
                            set_err(A.err, DERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
                s_issued = c;
            }
        } else if (role == R_NEAR) {
            // ---------------------------------------------------------------- loader: lines v-1, v-2
            // 32 positions of each line per poll; the staged prefix is what differs from the fill
            int b1 = s_near, b2 = s_near2;
            const long long l1 = DIR > 0 ? v - 1 : G.nlines - v;
            const long long l2 = DIR > 0 ? v - 2 : G.nlines + 1 - v;
            AT *r1 = sy + (own - 1) * RS + PADL, *r2 = sy + (own - 2) * RS + PADL;
            // cluster mode, rank > 0: line v-1's CTA stores its values into row r1 itself;
            // the loader only follows how far it is final (for the stale warps)
            const bool local1 = clu && crank > 0;
            const long long t0 = clock64();
            for (int itp = 0; b1 < n1 || b2 < n1; ++itp) {
                const int p1 = b1 + lane, p2 = b2 + lane;
                const int i1 = DIR > 0 ? p1 : n1 - 1 - p1, i2 = DIR > 0 ? p2 : n1 - 1 - p2;
                bits_t x1 = FB::v, x2 = FB::v;
                if (p1 < n1) x1 = local1 ? lds_vol(smem_u32(r1 + i1), bits_t(0)) : ld_poll(out + l1 * n1 + i1);
                if (p2 < n1) x2 = ld_poll(out + l2 * n1 + i2);
                const unsigned m1 = __ballot_sync(FULL, p1 < n1 && x1 != FB::v);
                const unsigned m2 = __ballot_sync(FULL, p2 < n1 && x2 != FB::v);
                const int c1 = m1 == FULL ? 32 : __ffs(~m1) - 1;
                const int c2 = m2 == FULL ? 32 : __ffs(~m2) - 1;
                if (lane < c1 && !local1) r1[i1] = FB::val(x1);
                if (lane < c2) r2[i2] = FB::val(x2);
                if (c1 + c2 > 0) {
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        if (c2) st_release_cta(&s_near2, b2 + c2);
                        if (c1) st_release_cta(&s_near, b1 + c1);
                    }
                    b1 += c1;
                    b2 += c2;
                } else {
                    if (itp > 64) __nanosleep(32);
                    if ((itp & 15) == 15) {
                        bool stop = s_abort != 0 || *(volatile int *)A.err != 0;
                        if (clock64() - t0 > 4 * A.budget) {
                            if (lane == 0) set_err(A.err, DERR_TIMEOUT);
                            stop = true;
                        }
                        if (__any_sync(FULL, stop)) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        } else if (role == R_FAR) {
            // ---------------------------------------------------------------- loader: lines v-3 .. v-w
            // lane h holds how far line v-h is staged
            int my = (G.d >= 2 && lane >= 3 && lane <= w && vin - lane >= 0) ? 0 : n1;
            const long long t0 = clock64();
            for (int itp = 0;; ++itp) {
                if ((int)__reduce_min_sync(FULL, (unsigned)my) >= n1) break;
                bool moved = false;
                for (int h0 = 3; h0 <= w; h0 += 8) {
                    bits_t x[8];
                    int st[8], ii[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int h = h0 + u;
                        st[u] = __shfl_sync(FULL, my, h & 31);
                        if (h > w) st[u] = n1;
                        const int p = st[u] + lane;
                        ii[u] = DIR > 0 ? p : n1 - 1 - p;
                        x[u] = FB::v;
                        if (p < n1) {
                            const long long hl = DIR > 0 ? v - h : G.nlines - 1 - (v - h);
                            x[u] = ld_poll(out + hl * n1 + ii[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int h = h0 + u;
                        const int p = st[u] + lane;
                        const unsigned m = __ballot_sync(FULL, p < n1 && x[u] != FB::v);
                        const int c = m == FULL ? 32 : __ffs(~m) - 1;
                        if (c > 0) {
                            if (lane < c) sy[(own - h) * RS + PADL + ii[u]] = FB::val(x[u]);
                            moved = true;
                            if (lane == h) my = st[u] + c;
                        }
                    }
                }
                if (moved) {
                    __syncwarp();
                    const int far = (int)__reduce_min_sync(FULL, (unsigned)my);
                    if (lane == 0) {
                        __threadfence_block();
                        st_release_cta(&s_far, far);
                    }
                } else {
                    if (itp > 64) __nanosleep(32);
                    if ((itp & 15) == 15) {
                        bool stop = s_abort != 0 || *(volatile int *)A.err != 0;
                        if (clock64() - t0 > 4 * A.budget) {
                            if (lane == 0) set_err(A.err, DERR_TIMEOUT);
                            stop = true;
                        }
                        if (__any_sync(FULL, stop)) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) s_abort = 1;
        __syncthreads();
        if (live && s_abort) {
            // the last chunk issued on each ring barrier must land before the CTA exits
            if (threadIdx.x == 0) {
                const int iss = s_issued;
                for (int b = 0; b < NB && b < iss; ++b) {
                    const int cl = b + ((iss - 1 - b) / NB) * NB;
                    mbar_wait(&mbar[b], parity(it, cl * L1_CH), A.err);
                }
                // cluster mode: the next claim stops every cluster (an abort follows a
                // recorded error; this keeps the first one)
                if (clu) set_err(A.err, DERR_TIMEOUT);
            }
            if (!clu) return;
        }
        if (live) ++it;  // the ring barriers' phases count the lines this CTA swept
    }
}

template <typename V, typename AT, int DIR, int D>
static int launch_sweep(const SweepArgs &A, size_t smem, unsigned grid, cudaStream_t s)
{
    static size_t attr = 0;  // benign race: setting the attribute twice is harmless
    if (smem > attr) {
        LSG_CK(cudaFuncSetAttribute(k_sweep<V, AT, DIR, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    ::lsg::count_launch();
    k_sweep<V, AT, DIR, D><<<grid, 32 * (A.B + SW_HELP), smem, s>>>(A);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

template <typename V, typename AT, int DIR>
static int launch_sweep_d(const SweepArgs &A, int D, size_t smem, unsigned grid, cudaStream_t s)
{
    if (D == 6) return launch_sweep<V, AT, DIR, 6>(A, smem, grid, s);
    return launch_sweep<V, AT, DIR, 4>(A, smem, grid, s);
}

template <typename V, typename AT, int DIR, int D, int NW>
static int line_smem_attr(size_t smem)
{
    static size_t attr = 0;  // benign race: setting the attribute twice is harmless
    if (smem > attr) {
        LSG_CK(cudaFuncSetAttribute(k_sweep_line<V, AT, DIR, D, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
        attr = smem;
    }
    return LSG_OK;
}

static cudaLaunchConfig_t line_config(unsigned grid, int nw, size_t smem, int csz, cudaStream_t s,
                                      cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * nw);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csz;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Clusters of csz line CTAs that can be resident at once (0: none, or the query failed).
template <typename V, typename AT, int DIR, int D>
static int line_clusters(size_t smem, int csz)
{
    if (line_smem_attr<V, AT, DIR, D, L1_WARPS2>(smem) != LSG_OK) return 0;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = line_config((unsigned)csz, L1_WARPS2, smem, csz, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_sweep_line<V, AT, DIR, D, L1_WARPS2>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

// csz > 1: launched in clusters of csz CTAs (grid a multiple of csz; 2D only, NW = L1_WARPS2).
template <typename V, typename AT, int DIR, int D, int NW>
static int launch_line(const SweepArgs &A, size_t smem, unsigned grid, int csz, cudaStream_t s)
{
    LSG_TRY((line_smem_attr<V, AT, DIR, D, NW>(smem)));
    ::lsg::count_launch();
    if (csz <= 1) {
        k_sweep_line<V, AT, DIR, D, NW><<<grid, 32 * NW, smem, s>>>(A);
    } else {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = line_config(grid, NW, smem, csz, s, at);
        LSG_CK(cudaLaunchKernelEx(&cfg, k_sweep_line<V, AT, DIR, D, NW>, A));
    }
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

template <typename V, typename AT, int DIR, int NW>
static int launch_line_dw(const SweepArgs &A, int D, size_t smem, unsigned grid, int csz, cudaStream_t s)
{
    if (D == L1_D) return launch_line<V, AT, DIR, L1_D, NW>(A, smem, grid, csz, s);
    if (D == L1_DM) return launch_line<V, AT, DIR, L1_DM, NW>(A, smem, grid, csz, s);
    return launch_line<V, AT, DIR, L1_DS, NW>(A, smem, grid, csz, s);
}
// 3D: 16 warps (nine stale); 1D/2D: 12
template <typename V, typename AT, int DIR>
static int launch_line_d(const SweepArgs &A, int D, size_t smem, unsigned grid, int csz, cudaStream_t s)
{
    if (A.G.d == 3) return launch_line_dw<V, AT, DIR, L1_WARPS3>(A, D, smem, grid, csz, s);
    return launch_line_dw<V, AT, DIR, L1_WARPS2>(A, D, smem, grid, csz, s);
}

template <typename V, typename AT, int DIR>
static int line_clusters_d(int D, size_t smem, int csz)
{
    if (D == L1_D) return line_clusters<V, AT, DIR, L1_D>(smem, csz);
    if (D == L1_DM) return line_clusters<V, AT, DIR, L1_DM>(smem, csz);
    return line_clusters<V, AT, DIR, L1_DS>(smem, csz);
}

template <typename AT>
static int launch_fill(AT *out, long long n, unsigned *counter, const int *done, int nsm, cudaStream_t s)
{
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4LL * nsm));
    ::lsg::count_launch();
    k_line_fill<AT><<<grid, 256, 0, s>>>(out, n, counter, done);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

// CTAs a sweep needs (lines per CTA: B).  In 1D and 2D the wavefront keeps
// about n1 / (w+1) lines busy at a time: line v may finish position q once line
// v-1 has finished q+w, so a line starts w+1 positions after the previous one
// and takes n1 positions plus a hand-off.  A CTA that finishes its line claims the
// next free one, so that many CTAs (and a margin) keep the sweep at full speed;
// more would only wait, holding SMs that other solves running at the same time
// (batched and served problems) can use.  In 3D the planes are pipelined as
// well and every SM finds work.
static long long wavefront_ctas(const Geom &g, int B)
{
    const long long bands = (g.nlines + B - 1) / B;
    if (g.d == 3) return bands;
    const long long busy = (g.n1 + 16 + g.w) / (g.w + 1) + 2;
    return std::min(bands, (busy + B - 1) / B + 1);
}

// Both sweeps with the line-parallel kernel (1D and 2D).
template <typename V, typename AT>
static int sweeps_line(lsg_ctx *c, const AT *r, AT *z, AT *ytmp, const int *done, cudaStream_t s, int D, size_t smf,
                       size_t smb)
{
    const Geom &g = c->g;
    SweepArgs A{};
    A.G = sgeo(g);
    A.done = done;
    A.err = c->err;
    A.budget = c->wait_budget;
    A.B = 1;
    // fresh window: the stale part of a row may start K positions before the row
    // is finished, which covers its ~1 us FP64 reduction at a few hundred ns per position;
    // the ring must hold the window's rows and K more (K <= D - 4)
    A.K = D >= 16 ? 8 : 4;
    int dev = 0, nsm = 0;
    LSG_CK(cudaGetDevice(&dev));
    LSG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    unsigned grid = (unsigned)std::min<long long>(wavefront_ctas(g, 1), nsm);
    // 2D: clusters of line CTAs hand the values of each line to the next through
    // distributed shared memory (one cluster group of csz lines at a time; rank 0 of a
    // group still reads the previous group's last line from the output); enough
    // clusters for the wavefront's busy lines plus one group
    int csz = 1;
    if (g.d == 2) {
        for (int cs : {L1_CLUSTER, 4}) {
            const long long ncl = (wavefront_ctas(g, 1) + cs - 1) / cs + 1;
            if (g.nlines < 2LL * cs || ncl * cs > nsm) continue;
            const int mf = line_clusters_d<V, AT, 1>(D, smf, cs), mb = line_clusters_d<V, AT, -1>(D, smb, cs);
            if (std::min(mf, mb) >= ncl) {
                csz = cs;
                grid = (unsigned)(ncl * cs);
                break;
            }
        }
    }
    int slot;
    // forward: L y = r
    A.F = c->Lv;
    A.RL = g.SL;
    A.rhs = r;
    A.out = ytmp;
    A.counter = c->counters + 1;
    LSG_TRY(prof_begin(c, PROF_SWEEP_L, s, &slot));
    LSG_TRY(launch_fill<AT>(ytmp, g.n, c->counters + 1, done, nsm, s));
    LSG_TRY((launch_line_d<V, AT, 1>(A, D, smf, grid, csz, s)));
    LSG_TRY(prof_end(c, slot, s));
    // backward: U z = y (z is filled only now: it may be the same vector as r)
    A.F = c->Uv;
    A.RL = g.SU;
    A.rhs = ytmp;
    A.out = z;
    A.counter = c->counters + 2;
    LSG_TRY(prof_begin(c, PROF_SWEEP_U, s, &slot));
    LSG_TRY(launch_fill<AT>(z, g.n, c->counters + 2, done, nsm, s));
    LSG_TRY((launch_line_d<V, AT, -1>(A, D, smb, grid, csz, s)));
    LSG_TRY(prof_end(c, slot, s));
    return LSG_OK;
}

template <typename V, typename AT>
static int sweeps(lsg_ctx *c, const AT *r, AT *z, AT *ytmp, const int *done, cudaStream_t s)
{
    const Geom &g = c->g;
    const size_t budget = 210 * 1024;
    if ((g.d == 3 || g.Sc <= 32 * SW_KS) && g.w <= 31) {
        const int vs = (int)sizeof(V), as = (int)sizeof(AT);
        // the deepest ring that fits: the finisher's window (K = 8 from 16 rows, 4 from 8)
        // is the slack the stale warps have to finish a row
        for (int D : {L1_D, L1_DM, L1_DS}) {
            const size_t smf = line_layout(g.d, g.n1, g.w, D, g.SL, vs, g.Sc, as).total;
            const size_t smb = line_layout(g.d, g.n1, g.w, D, g.SU, vs, g.Sc, as).total;
            if (std::max(smf, smb) <= budget) return sweeps_line<V, AT>(c, r, z, ytmp, done, s, D, smf, smb);
        }
    }
    SweepArgs A{};
    A.G = sgeo(g);
    A.done = done;
    A.err = c->err;
    A.budget = c->wait_budget;
    // lines per CTA: one per SM sub-partition (an FP64 warp instruction occupies its
    // sub-partition's FP64 unit for ~64 clocks; in FP32 a second line per
    // sub-partition measured slower too); fewer if shared memory runs out
    const int RLmax = std::max(g.SL, g.SU);
    const int vs = (int)sizeof(V), as = (int)sizeof(AT);
    int B = 4;
    while (B > 1 && sweep_layout(g.n1, g.w, B, 4, RLmax, vs, g.Sc, as).total > budget) B /= 2;
    if (sweep_layout(g.n1, g.w, B, 4, RLmax, vs, g.Sc, as).total > budget) return LSG_ERR_ARG;
    // factor ring: six rows in flight per line where they fit, else four
    const int D = sweep_layout(g.n1, g.w, B, 6, RLmax, vs, g.Sc, as).total <= budget ? 6 : 4;
    if (g.w > 31) return LSG_ERR_ARG;  // one halo lane per previous line
    if (B > g.nlines) B = (int)std::max<long long>(1, g.nlines);
    A.B = B;
    int dev = 0, nsm = 0;
    LSG_CK(cudaGetDevice(&dev));
    LSG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    unsigned grid = (unsigned)std::min<long long>(wavefront_ctas(g, B), nsm);
    LSG_CK(cudaMemsetAsync(c->prog, 0, sizeof(unsigned) * 2 * (size_t)g.nlines, s));
    LSG_CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(unsigned) * 2, s));
    // forward: L y = r
    A.F = c->Lv;
    A.RL = g.SL;
    A.rhs = r;
    A.out = ytmp;
    A.gprog = c->prog;
    A.counter = c->counters + 1;
    size_t smf = sweep_layout(g.n1, g.w, B, D, g.SL, vs, g.Sc, as).total;
    int slot;
    LSG_TRY(prof_begin(c, PROF_SWEEP_L, s, &slot));
    LSG_TRY((launch_sweep_d<V, AT, 1>(A, D, smf, grid, s)));
    LSG_TRY(prof_end(c, slot, s));
    // backward: U z = y
    A.F = c->Uv;
    A.RL = g.SU;
    A.rhs = ytmp;
    A.out = z;
    A.gprog = c->prog + g.nlines;
    A.counter = c->counters + 2;
    size_t smb = sweep_layout(g.n1, g.w, B, D, g.SU, vs, g.Sc, as).total;
    LSG_TRY(prof_begin(c, PROF_SWEEP_U, s, &slot));
    LSG_TRY((launch_sweep_d<V, AT, -1>(A, D, smb, grid, s)));
    LSG_TRY(prof_end(c, slot, s));
    return LSG_OK;
}

// FP64 vectors: FP64 factors with FP64 accumulation, or (mixed contexts) FP32
// factors with FP64 accumulation.
int apply_Minv(lsg_ctx *c, const double *r, double *z, const int *done, cudaStream_t s)
{
    if (c->precond == 1) {  // PCG-I: the constant-coefficient preconditioner, solved directly
        int slot;
        LSG_TRY(prof_begin(c, PROF_CONST, s, &slot));
        LSG_TRY(apply_const_precond(c, r, z, done, s));
        return prof_end(c, slot, s);
    }
    if (c->precision == LSG_FP64) return sweeps<double, double>(c, r, z, c->ys, done, s);
    return sweeps<float, double>(c, r, z, c->ys, done, s);
}

// FP32 vectors (inner solve of the mixed form): FP32 factors, FP32 accumulation.
int apply_Minv32(lsg_ctx *c, const float *r, float *z, const int *done, cudaStream_t s)
{
    if (c->precision == LSG_FP64) return LSG_ERR_ARG;
    return sweeps<float, float>(c, r, z, c->y32, done, s);
}

}  // namespace lsg
