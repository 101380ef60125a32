// tc_transform.cu -- the mixed form's matrix-free product on the fifth-generation
// tensor cores.  Every sum-factorised contraction of K x (Sec. 4.3, steps 1-4;
// see transform.cu for the FP64 form) is a batched GEMM
//     D[m][n] = sum_t sum_k A_t[m][k] X_t[n][k]        (one or two terms t)
// with A a basis table (phi or phi' at the Gauss nodes, or its transpose) and
// X the current field, both K-major.  Operands are TF32 or BF16 in shared
// memory, the accumulator is FP32 in tensor memory: tcgen05.mma issued by one
// thread, completion tracked with tcgen05.commit on an mbarrier, the tile read
// back with tcgen05.ld for the epilogue (optional pointwise factor W a or W b).
//
// Each FP32 operand v is split into two pieces of the operand type, v = hi + lo
// (TF32: hi = v with the 13 low mantissa bits cleared, lo = v - hi exactly;
// BF16: hi = bf16(v), lo = bf16(v - hi)), and a product is taken as
// hi*hi + hi*lo + lo*hi: three MMAs that bring the operand error from 2^-11
// (TF32) or 2^-8 (BF16) down to about 2^-21 or 2^-16, so the FP64 refinement
// around the inner solve needs no extra steps.  Tables are unfolded (no parity
// folding): the tensor cores have flops to spare and a contraction is bound by
// moving the fields, not by the multiply-adds.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "lsg_internal.cuh"

namespace lsg {

constexpr int TC_BM = 128;      // rows of D per CTA (tensor-memory lanes); rows of a stored tile
constexpr int TC_BN = 64;       // columns of D per CTA (tensor-memory columns): half a stored tile of B
constexpr int TC_BK = 32;       // K elements per pipeline stage
constexpr int TC_THREADS = 128;
// pipeline stages of A and B (hi and lo pieces each): 4 x 48 KB for TF32, 7 x 24 KB
// for BF16 (one CTA per SM either way)
template <typename OP>
constexpr int tc_stages() { return sizeof(OP) == 4 ? 4 : 7; }
template <typename OP>
constexpr size_t tc_smem() { return (size_t)tc_stages<OP>() * 2 * (TC_BM + TC_BN) * TC_BK * sizeof(OP) + 128; }

// Operand arrays (the tables and the split fields) are stored tile by tile: each
// tile of 128 rows x TC_BK columns is contiguous and already in the core-matrix order
// the MMA reads from shared memory (8 rows x 16 bytes per core matrix, K-adjacent core
// matrices 128 bytes apart, 8-row groups TC_BK * ES * 8 bytes apart), so that one bulk
// copy moves a tile.  Element (r, k) of an array with nkb tiles per 128-row block:
template <int ES>
__host__ __device__ inline long long tc_tile_off(long long r, int k, int nkb)
{
    constexpr int EPC = 16 / ES, KC = TC_BK / EPC;  // elements per 16 bytes; 16-byte chunks per row
    const int rr = (int)(r & 127), kk = k % TC_BK;
    return ((r >> 7) * nkb + k / TC_BK) * (long long)(128 * TC_BK) + ((rr >> 3) * KC + kk / EPC) * (8 * EPC) +
           (rr & 7) * EPC + kk % EPC;
}

template <typename OP>
struct TcOp;
template <>
struct TcOp<float> {  // TF32: .kind::tf32, K = 8 per instruction
    static constexpr uint32_t fmt = 2;
    static constexpr int kmma = 8;
};
template <>
struct TcOp<__nv_bfloat16> {  // BF16: .kind::f16, K = 16 per instruction
    static constexpr uint32_t fmt = 1;
    static constexpr int kmma = 16;
};

// Operands between contractions are kept split, as the next contraction reads B: a
// field of L values is an array of L / Kn rows of Kn values (Kn = the next
// contraction's K) padded to rup(Kn, TC_BK) columns and whole 128-row blocks, tiled as
// above, hi pieces then lo pieces; padding is zero (the workspace is cleared once, and a
// contraction writes a padding slot only with zero).
struct TcTerm {
    const void *A;    // [Mp][Kp] table (hi pieces, tiled) in the operand type, zero padded; lo pieces follow
    const void *B;    // [Np][Kp] field (hi pieces, tiled) in the operand type; lo pieces `blo` elements on
    long long blo;
};
struct TcOut {
    float *y;            // FP32 [M][N] output (the last contraction), or null
    void *ys;            // else the split output, for a next contraction with K = Kn
    long long ylo;       // elements from its hi pieces to its lo pieces
    int Kn, Kpn;         // the next contraction's K and its padded row length
    const float *scale;  // optional [M][N] pointwise factor
    int nterm;
    TcTerm t[2];
};
struct TcJob {
    int M, K, Kp;
    long long lo;     // elements from a table's hi pieces to its lo pieces (Mp * Kp)
    long long N;
    int nout;
    TcOut o[4];
    const int *done;
    int *err;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t tc_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8
// rows x 16 bytes (rows 16 bytes apart), `lbo` bytes between core matrices
// adjacent in K, `sbo` bytes between 8-row groups.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the fifth-generation tensor cores
    return d;                // base offset 0, relative LBO, no swizzle
}
// Instruction descriptor: FP32 accumulator, A and B of format `fmt`, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt, int M, int N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <typename OP>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    if constexpr (sizeof(OP) == 4) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(bar)) : "memory");
}
// Bounded wait for phase `parity` of an mbarrier.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, int *err)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(tc_saddr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kSpinBudgetCycles) {
            set_err(err, DERR_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <typename OP>
__device__ __forceinline__ void tc_split(float v, OP &hi, OP &lo);
template <>
__device__ __forceinline__ void tc_split<float>(float v, float &hi, float &lo)
{
    hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);  // exactly representable in TF32
    lo = v - hi;                                              // exact in FP32
}
template <>
__device__ __forceinline__ void tc_split<__nv_bfloat16>(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ void tc_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_saddr(bar)), "r"(bytes) : "memory");
}
// one bulk copy global -> shared, completing on `bar` (both addresses 16-byte aligned)
__device__ __forceinline__ void tc_bulk(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(tc_saddr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(tc_saddr(bar))
        : "memory");
}

// One 128 x 128 tile of D per CTA.  One thread runs the pipeline: per K step it
// moves the four tiles (A hi and lo, B hi and lo; both already split and tiled) into
// a stage with bulk copies completing on the stage's `full` barrier, issues the
// step's MMAs once they have landed, and refills the stage of the previous step once
// that step's MMAs are done (tcgen05.commit on the stage's `mdone` barrier).
template <typename OP>
__global__ void __launch_bounds__(TC_THREADS) k_tc_gemm(const __grid_constant__ TcJob J)
{
    if (J.done && *J.done) return;
    const TcOut &O = J.o[blockIdx.z];
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int S = tc_stages<OP>();
    constexpr int ES = (int)sizeof(OP);
    constexpr int KC = TC_BK * ES / 16;            // 16-byte chunks per row and stage
    constexpr int TB = TC_BM * TC_BK * ES;         // bytes of a stored tile (A)
    constexpr int TBB = TC_BN * TC_BK * ES;        // bytes of a B tile: the first or second half of a stored one
    constexpr int STAGE = 2 * (TB + TBB);          // A hi, A lo, B hi, B lo
    constexpr uint32_t IDESC = tc_idesc(TcOp<OP>::fmt, TC_BM, TC_BN);
    static_assert(TC_BM % TC_BN == 0, "B tiles are equal parts of a stored tile");
    uint64_t *full = (uint64_t *)(smem + S * STAGE), *mdone = full + S;
    uint32_t *tslot = (uint32_t *)(mdone + S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mb = blockIdx.x, nbk = blockIdx.y;
    const int m0 = mb * TC_BM;
    const long long n0 = (long long)nbk * TC_BN;

    if (tid == 0) {
        for (int i = 0; i < 2 * S; ++i) tc_mbar_init(&full[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(tslot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int nkt = J.Kp / TC_BK;  // K tiles
    const int total = nkt * O.nterm;
    bool ok = true;
    if (tid == 0) {
        int issued = 0, consumed = 0, last = -1;
        auto issue = [&](int k) {
            const int st = k % S;
            unsigned char *sp = smem + st * STAGE;
            const TcTerm tm = O.t[k / nkt];
            const int kb = k % nkt;
            // B rows n0.. are part nbk % (TC_BM / TC_BN) of the stored tile of row block
            // n0 / TC_BM: a contiguous run of the tile (its 8-row groups are in row order)
            constexpr int NP = TC_BM / TC_BN;
            const OP *A = (const OP *)tm.A + ((long long)mb * nkt + kb) * (TC_BM * TC_BK);
            const OP *B = (const OP *)tm.B + ((long long)(nbk / NP) * nkt + kb) * (TC_BM * TC_BK) +
                          (nbk % NP) * (TC_BN * TC_BK);
            tc_expect_tx(&full[st], 2u * (TB + TBB));
            tc_bulk(sp, A, TB, &full[st]);
            tc_bulk(sp + TB, A + J.lo, TB, &full[st]);
            tc_bulk(sp + 2 * TB, B, TBB, &full[st]);
            tc_bulk(sp + 2 * TB + TBB, B + tm.blo, TBB, &full[st]);
            ++issued;
        };
        for (int k = 0; k < S - 1 && k < total; ++k) issue(k);
        for (int it = 0; it < total && ok; ++it) {
            const int st = it % S;
            ok = tc_wait(&full[st], (uint32_t)((it / S) & 1), J.err);
            if (!ok) break;
            consumed = it + 1;
            tc_fence_after();
            const uint32_t sa = tc_saddr(smem + st * STAGE), sbo = (uint32_t)KC * 128u;
#pragma unroll
            for (int j = 0; j < TC_BK / TcOp<OP>::kmma; ++j) {
                const uint64_t ah = tc_desc(sa + 256u * j, 128u, sbo);
                const uint64_t al = tc_desc(sa + TB + 256u * j, 128u, sbo);
                const uint64_t bh = tc_desc(sa + 2 * TB + 256u * j, 128u, sbo);
                const uint64_t bl = tc_desc(sa + 2 * TB + TBB + 256u * j, 128u, sbo);
                tc_mma<OP>(tmem, ah, bh, IDESC, (it > 0 || j > 0) ? 1u : 0u);  // hi * hi
                tc_mma<OP>(tmem, ah, bl, IDESC, 1u);                            // hi * lo
                tc_mma<OP>(tmem, al, bh, IDESC, 1u);                            // lo * hi
            }
            tc_commit(&mdone[st]);
            last = it;
            // refill the stage of step it - 1 with step it + S - 1, once its MMAs are done
            const int nx = it + S - 1;
            if (nx < total) {
                if (it >= 1) ok = tc_wait(&mdone[(it - 1) % S], (uint32_t)(((it - 1) / S) & 1), J.err);
                if (ok) issue(nx);
            }
        }
        // every MMA must be complete before the tile is read or its memory reused (on an
        // error too: the last commit covers every MMA issued before it), and so must every
        // bulk copy issued
        if (last >= 0 && !tc_wait(&mdone[last % S], (uint32_t)((last / S) & 1), J.err)) ok = false;
        for (int k = consumed; k < issued; ++k) (void)tc_wait(&full[k % S], (uint32_t)((k / S) & 1), J.err);
        if (last < total - 1) ok = false;
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();
    // epilogue: warp w owns tensor-memory lanes 32w..32w+31 = rows m0+32w+lane; the tile
    // goes through shared memory (free now) so that the stores, and the reads of the
    // pointwise factor, run along memory
    float *tile = (float *)smem;  // [TC_BM][TC_BN + 1], the pointwise factor applied
    constexpr int TP = TC_BN + 1;
    const int mrow = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        uint32_t r[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            float v = __uint_as_float(r[jj]);
            const long long n = n0 + c0 + jj;
            if (O.scale && mrow < J.M && n < J.N) v *= O.scale[(size_t)mrow * J.N + n];
            tile[(32 * warp + lane) * TP + c0 + jj] = v;
        }
    }
    __syncthreads();
    OP *yh = (OP *)O.ys, *yl = yh + O.ylo;
    const int nkbn = O.Kpn / TC_BK;  // K tiles of the next contraction
    if (!ok) {
    } else if (!O.y && J.N == O.Kn) {
        // the output's rows are the next B's rows and its columns the next K: this tile
        // fills whole next-B tiles (row block mb, K tiles n0 / TC_BK ..), written 16 bytes
        // per thread in memory order, zero outside the field
        constexpr int EPC = 16 / ES, PPT = TC_BM * TC_BK / EPC;
        for (int t = 0; t < TC_BN / TC_BK; ++t) {
            const int kb = (int)(n0 / TC_BK) + t;
            if (kb >= nkbn) break;
            const long long tb = ((long long)mb * nkbn + kb) * (TC_BM * TC_BK);
            for (int p = tid; p < PPT; p += TC_THREADS) {
                const int chunk = p >> 3, rr = ((chunk / KC) << 3) | (p & 7), cl = t * TC_BK + (chunk % KC) * EPC;
                const int m = m0 + rr;
                OP h[EPC], l[EPC];
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const long long n = n0 + cl + e;
                    float v = 0.0f;
                    if (m < J.M && n < J.N) v = tile[rr * TP + cl + e];
                    tc_split<OP>(v, h[e], l[e]);
                }
                uint4 vh, vl;
                memcpy(&vh, h, 16);
                memcpy(&vl, l, 16);
                *(uint4 *)(yh + tb + (long long)p * EPC) = vh;
                *(uint4 *)(yl + tb + (long long)p * EPC) = vl;
            }
        }
    } else {
        // RS threads per column, on alternate rows
        constexpr int RS = TC_THREADS / TC_BN;
        const int r0 = tid / TC_BN;
        const long long n = n0 + tid % TC_BN;
        if (n < J.N) {
            // general layout: flat index o = m N + n is row o / Kn, column o % Kn of the
            // next B; from one of this thread's rows to the next o grows by RS N
            const long long Kn = O.Kn, qN = RS * J.N / Kn, rN = RS * J.N % Kn;
            const long long o0 = (long long)(m0 + r0) * J.N + n;
            long long row = o0 / Kn, col = o0 - (o0 / Kn) * Kn;
            for (int rr = r0; rr < TC_BM; rr += RS) {
                const int m = m0 + rr;
                if (m >= J.M) break;
                const size_t o = (size_t)m * J.N + n;
                const float v = tile[rr * TP + (int)(n - n0)];
                if (O.y) {
                    O.y[o] = v;
                } else {
                    const long long so = tc_tile_off<ES>(row, (int)col, nkbn);
                    OP hi, lo;
                    tc_split<OP>(v, hi, lo);
                    yh[so] = hi;
                    yl[so] = lo;
                }
                row += qN;
                col += rN;
                if (col >= Kn) {
                    col -= Kn;
                    ++row;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// The product's input field, split into the operand type in the layout the first
// contraction reads (L values as L / Kn rows of Kn, tiled).
template <typename OP>
__global__ void k_tc_split(const float *x, long long L, int Kn, int Kpn, OP *hi, long long lo, const int *done)
{
    if (done && *done) return;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < L; f += (long long)gridDim.x * blockDim.x) {
        const long long row = f / Kn;
        const long long o = tc_tile_off<(int)sizeof(OP)>(row, (int)(f - row * Kn), Kpn / TC_BK);
        OP h, l;
        tc_split<OP>(x[f], h, l);
        hi[o] = h;
        hi[lo + o] = l;
    }
}

// ---- unfolded tables in the operand type -------------------------------------
// Forward tables Fphi/Fdphi [2][MpF][KpF] (hi, lo; tiled): row q (node), column k
// (basis index); backward tables Bphi/Bdphi [2][MpB][KpB]: their transposes.  Built from the
// parity-folded FP64 tables (first half of the nodes): for the mirrored node,
// phi_k(-x) = (-1)^k phi_k(x) and phi'_k(-x) = (-1)^(k+1) phi'_k(x).
template <typename OP>
__global__ void k_tc_tables(int Q, int n1, int Qh, int QhP, int KP, const double *tab, int MpF, int KpF, int MpB,
                            int KpB, OP *Fphi, OP *Fdphi, OP *Bphi, OP *Bdphi)
{
    const long long nF = (long long)MpF * KpF, nB = (long long)MpB * KpB;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nF + nB) return;
    int q, k;
    const bool fwd = idx < nF;
    if (fwd) {
        q = (int)(idx / KpF);
        k = (int)(idx % KpF);
    } else {
        const long long e = idx - nF;
        k = (int)(e / KpB);
        q = (int)(e % KpB);
    }
    double phi = 0.0, dphi = 0.0;
    if (q < Q && k < n1) {
        const size_t blk = (size_t)QhP * KP;
        const bool mirror = q >= Qh;
        const int qq = mirror ? Q - 1 - q : q;
        const size_t o = (size_t)qq * KP + (k >> 1);
        phi = (k & 1) ? tab[blk + o] : tab[o];
        dphi = (k & 1) ? tab[3 * blk + o] : tab[2 * blk + o];
        if (mirror) {
            if (k & 1) phi = -phi;
            else dphi = -dphi;
        }
    }
    // hi pieces, then lo pieces of the same table (the FP64 value is split as its FP32 rounding)
    OP ph, pl, dh, dl;
    tc_split<OP>((float)phi, ph, pl);
    tc_split<OP>((float)dphi, dh, dl);
    // stored tiled (row q and column k forward, row k and column q backward)
    constexpr int ES = (int)sizeof(OP);
    if (fwd) {
        const long long o = tc_tile_off<ES>(q, k, KpF / TC_BK);
        Fphi[o] = ph;
        Fphi[nF + o] = pl;
        Fdphi[o] = dh;
        Fdphi[nF + o] = dl;
    } else {
        const long long o = tc_tile_off<ES>(k, q, KpB / TC_BK);
        Bphi[o] = ph;
        Bphi[nB + o] = pl;
        Bdphi[o] = dh;
        Bdphi[nB + o] = dl;
    }
}

static inline int rup(int v, int m) { return (v + m - 1) / m * m; }

size_t tc_table_bytes(const Geom &g, int precision)
{
    if (precision == LSG_FP64) return 0;
    const size_t es = precision == LSG_MIXED_TF32 ? 4 : 2;
    const size_t MpF = rup(g.Q, TC_BM), KpF = rup(g.n1, TC_BK), MpB = rup(g.n1, TC_BM), KpB = rup(g.Q, TC_BK);
    return es * 4 * (MpF * KpF + MpB * KpB);  // two tables per direction, hi and lo pieces
}

template <typename OP>
static int tc_tables_t(lsg_ctx *c, cudaStream_t s)
{
    const Geom &g = c->g;
    c->tcMpF = rup(g.Q, TC_BM);
    c->tcKpF = rup(g.n1, TC_BK);
    c->tcMpB = rup(g.n1, TC_BM);
    c->tcKpB = rup(g.Q, TC_BK);
    const long long nF = (long long)c->tcMpF * c->tcKpF, nB = (long long)c->tcMpB * c->tcKpB;
    OP *Fphi = (OP *)c->tct, *Fdphi = Fphi + 2 * nF, *Bphi = Fdphi + 2 * nF, *Bdphi = Bphi + 2 * nB;
    ::lsg::count_launch();
    k_tc_tables<OP><<<(unsigned)((nF + nB + 255) / 256), 256, 0, s>>>(g.Q, g.n1, g.Qh, g.QhP, g.KP, c->tab, c->tcMpF,
                                                                    c->tcKpF, c->tcMpB, c->tcKpB, Fphi, Fdphi, Bphi,
                                                                    Bdphi);
    LSG_CK(cudaGetLastError());
    return LSG_OK;
}

int build_tc_tables(lsg_ctx *c, cudaStream_t s)
{
    if (!c->tct) return LSG_OK;
    if (c->precision == LSG_MIXED_TF32) return tc_tables_t<float>(c, s);
    return tc_tables_t<__nv_bfloat16>(c, s);
}

// ---- K x as a chain of tensor-core contractions -------------------------------
// The split fields of the chain: (L, Kn) per buffer, L values as L / Kn rows of Kn.
struct TcBufSpec {
    long long L;
    int Kn;
};
static int tc_buffers(const Geom &g, TcBufSpec *b)
{
    const long long Q = g.Q, n1 = g.n1;
    const int q = (int)Q, n = (int)n1;
    int k = 0;
    if (g.d == 1) {
        b[k++] = {n1, n};                        // x
        b[k++] = {Q, q}, b[k++] = {Q, q};        // H, Gx
    } else if (g.d == 2) {
        b[k++] = {n1 * n1, n};                   // x
        b[k++] = {Q * n1, n}, b[k++] = {Q * n1, n};                              // AP, AD
        b[k++] = {Q * Q, q}, b[k++] = {Q * Q, q}, b[k++] = {Q * Q, q};           // H, Gy, Gx
        b[k++] = {n1 * Q, q}, b[k++] = {n1 * Q, q};                              // P1, P2
    } else {
        b[k++] = {n1 * n1 * n1, n};                                              // x
        b[k++] = {Q * n1 * n1, n}, b[k++] = {Q * n1 * n1, n};                    // A0, A1
        for (int i = 0; i < 3; ++i) b[k++] = {Q * Q * n1, n};                    // B0, B1, B2
        for (int i = 0; i < 4; ++i) b[k++] = {Q * Q * Q, q};                     // H, Gz, Gy, Gx
        for (int i = 0; i < 3; ++i) b[k++] = {n1 * Q * Q, q};                    // Pa, Pb, Pc
        b[k++] = {n1 * n1 * Q, q}, b[k++] = {n1 * n1 * Q, q};                    // Ra, Rc
    }
    return k;
}
// elements of one piece (hi or lo) of a split field: rows padded for the B tiles,
// rows padded for the K steps, rounded to 256 bytes
static long long tc_piece(const TcBufSpec &b, int es)
{
    const long long rows = rup((int)((b.L + b.Kn - 1) / b.Kn), TC_BM);
    const long long e = rows * rup(b.Kn, TC_BK);
    return (e * es + 255) / 256 * 256 / es;
}

size_t tc_ws_bytes(const Geom &g, int precision)
{
    if (precision == LSG_FP64) return 0;
    const int es = precision == LSG_MIXED_TF32 ? 4 : 2;
    TcBufSpec b[16];
    const int nb = tc_buffers(g, b);
    size_t t = 0;
    for (int i = 0; i < nb; ++i) t += 2 * (size_t)tc_piece(b[i], es) * es;
    return t;
}

template <typename OP>
struct TcBuf {
    OP *p;
    long long lo;
    int Kn, Kpn;
};

template <typename OP>
struct TcBuilder {
    lsg_ctx *c;
    TcJob j;
    bool isfwd;
    const OP *tabF(int t) const
    {
        const long long nF = (long long)c->tcMpF * c->tcKpF;
        return (const OP *)c->tct + (t ? 2 * nF : 0);
    }
    const OP *tabB(int t) const
    {
        const long long nF = (long long)c->tcMpF * c->tcKpF, nB = (long long)c->tcMpB * c->tcKpB;
        return (const OP *)c->tct + 4 * nF + (t ? 2 * nB : 0);
    }
    // forward contraction: out[q][b] = sum_k T[q][k] x[b][k]  (M = Q, K = n1)
    void fwd(long long B, const int *done)
    {
        j = TcJob{};
        isfwd = true;
        j.M = c->g.Q;
        j.K = c->g.n1;
        j.Kp = c->tcKpF;
        j.lo = (long long)c->tcMpF * c->tcKpF;
        j.N = B;
        j.done = done;
        j.err = c->err;
    }
    // backward contraction: out[k][b] = sum_q T[q][k] x[b][q]  (M = n1, K = Q)
    void bwd(long long B, const int *done)
    {
        j = TcJob{};
        isfwd = false;
        j.M = c->g.n1;
        j.K = c->g.Q;
        j.Kp = c->tcKpB;
        j.lo = (long long)c->tcMpB * c->tcKpB;
        j.N = B;
        j.done = done;
        j.err = c->err;
    }
    // one output: a split field for the next contraction (y null) or the FP32 result
    void out(const TcBuf<OP> &dst, float *y, const float *scale, const TcBuf<OP> &x0, int t0,
             const TcBuf<OP> *x1 = nullptr, int t1 = 0)
    {
        const bool f = isfwd;
        TcOut &o = j.o[j.nout++];
        o.y = y;
        o.ys = y ? nullptr : (void *)dst.p;
        o.ylo = dst.lo;
        o.Kn = dst.Kn;
        o.Kpn = dst.Kpn;
        o.scale = scale;
        o.nterm = x1 ? 2 : 1;
        o.t[0] = TcTerm{f ? (const void *)tabF(t0) : (const void *)tabB(t0), x0.p, x0.lo};
        o.t[1] = TcTerm{x1 ? (f ? (const void *)tabF(t1) : (const void *)tabB(t1)) : nullptr, x1 ? x1->p : nullptr,
                        x1 ? x1->lo : 0};
    }
    int launch(cudaStream_t s)
    {
        static bool attr_set = false;  // benign race: setting the attribute twice is harmless
        if (!attr_set) {
            LSG_CK(cudaFuncSetAttribute(k_tc_gemm<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<OP>()));
            attr_set = true;
        }
        dim3 grid((unsigned)((j.M + TC_BM - 1) / TC_BM), (unsigned)((j.N + TC_BN - 1) / TC_BN), (unsigned)j.nout);
        ::lsg::count_launch();
        k_tc_gemm<OP><<<grid, TC_THREADS, tc_smem<OP>(), s>>>(j);
        LSG_CK(cudaGetLastError());
        return LSG_OK;
    }
};

template <typename OP>
static int apply_K_tc_t(lsg_ctx *c, const float *x, float *y, const int *done, cudaStream_t s)
{
    const Geom &g = c->g;
    const long long Q = g.Q, n1 = g.n1;
    const float *Wa = c->Wa32, *Way = c->Wa32y, *Waz = c->Wa32z, *Wb = c->Wb32;  // W a_j per gradient term
    TcBufSpec spec[16];
    const int nb = tc_buffers(g, spec);
    TcBuf<OP> B[16];
    OP *p = (OP *)c->ws32;
    for (int i = 0; i < nb; ++i) {
        const long long e = tc_piece(spec[i], (int)sizeof(OP));
        B[i] = TcBuf<OP>{p, e, spec[i].Kn, rup(spec[i].Kn, TC_BK)};
        p += 2 * e;
    }
    const TcBuf<OP> none{nullptr, 0, 1, 1};
    // the input field, split
    {
        const long long L = spec[0].L;
        const unsigned blocks = (unsigned)std::min<long long>((L + 255) / 256, 4096);
        ::lsg::count_launch();
        k_tc_split<OP><<<blocks, 256, 0, s>>>(x, L, B[0].Kn, B[0].Kpn, B[0].p, B[0].lo, done);
        LSG_CK(cudaGetLastError());
    }
    TcBuilder<OP> T{c, {}, true};
    if (g.d == 1) {
        const TcBuf<OP> &X = B[0], &H = B[1], &Gx = B[2];
        T.fwd(1, done);
        T.out(H, nullptr, Wb, X, 0);
        T.out(Gx, nullptr, Wa, X, 1);
        LSG_TRY(T.launch(s));
        T.bwd(1, done);
        T.out(none, y, nullptr, H, 0, &Gx, 1);
        return T.launch(s);
    }
    if (g.d == 2) {
        const TcBuf<OP> &X = B[0], &AP = B[1], &AD = B[2], &H = B[3], &Gy = B[4], &Gx = B[5], &P1 = B[6], &P2 = B[7];
        T.fwd(n1, done);  // contract x
        T.out(AP, nullptr, nullptr, X, 0);
        T.out(AD, nullptr, nullptr, X, 1);
        LSG_TRY(T.launch(s));
        T.fwd(Q, done);  // contract y, pointwise W a / W b
        T.out(H, nullptr, Wb, AP, 0);
        T.out(Gy, nullptr, Way, AP, 1);
        T.out(Gx, nullptr, Wa, AD, 0);
        LSG_TRY(T.launch(s));
        T.bwd(Q, done);  // back over x nodes
        T.out(P1, nullptr, nullptr, H, 0, &Gx, 1);
        T.out(P2, nullptr, nullptr, Gy, 0);
        LSG_TRY(T.launch(s));
        T.bwd(n1, done);  // back over y nodes
        T.out(none, y, nullptr, P1, 0, &P2, 1);
        return T.launch(s);
    }
    const TcBuf<OP> &X = B[0], &A0 = B[1], &A1 = B[2], &B0 = B[3], &B1 = B[4], &B2 = B[5];
    const TcBuf<OP> &H = B[6], &Gz = B[7], &Gy = B[8], &Gx = B[9], &Pa = B[10], &Pb = B[11], &Pc = B[12];
    const TcBuf<OP> &Ra = B[13], &Rc = B[14];
    T.fwd(n1 * n1, done);
    T.out(A0, nullptr, nullptr, X, 0);
    T.out(A1, nullptr, nullptr, X, 1);
    LSG_TRY(T.launch(s));
    T.fwd(Q * n1, done);
    T.out(B0, nullptr, nullptr, A0, 0);
    T.out(B1, nullptr, nullptr, A0, 1);
    T.out(B2, nullptr, nullptr, A1, 0);
    LSG_TRY(T.launch(s));
    T.fwd(Q * Q, done);
    T.out(H, nullptr, Wb, B0, 0);
    T.out(Gz, nullptr, Waz, B0, 1);
    T.out(Gy, nullptr, Way, B1, 0);
    T.out(Gx, nullptr, Wa, B2, 0);
    LSG_TRY(T.launch(s));
    T.bwd(Q * Q, done);
    T.out(Pa, nullptr, nullptr, H, 0, &Gx, 1);
    T.out(Pb, nullptr, nullptr, Gy, 0);
    T.out(Pc, nullptr, nullptr, Gz, 0);
    LSG_TRY(T.launch(s));
    T.bwd(n1 * Q, done);
    T.out(Ra, nullptr, nullptr, Pa, 0, &Pb, 1);
    T.out(Rc, nullptr, nullptr, Pc, 0);
    LSG_TRY(T.launch(s));
    T.bwd(n1 * n1, done);
    T.out(none, y, nullptr, Ra, 0, &Rc, 1);
    return T.launch(s);
}

// y = K x with TF32 or BF16 tensor-core contractions (FP32 fields and accumulation).
int apply_K_tc(lsg_ctx *c, const float *x, float *y, const int *done, cudaStream_t s)
{
    if (!c->tct) return LSG_ERR_ARG;
    if (c->precision == LSG_MIXED_TF32) return apply_K_tc_t<float>(c, x, y, done, s);
    return apply_K_tc_t<__nv_bfloat16>(c, x, y, done, s);
}

}  // namespace lsg
