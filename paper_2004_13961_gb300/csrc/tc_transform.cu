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

#include "lsg_internal.cuh"

namespace lsg {

constexpr int TC_BM = 128;      // rows of D per CTA (tensor-memory lanes)
constexpr int TC_BN = 128;      // columns of D per CTA (tensor-memory columns)
constexpr int TC_BK = 32;       // K elements per pipeline stage
constexpr int TC_THREADS = 128;
// two stages of A and B (hi and lo pieces each): 128 KB for TF32, 64 KB for
// BF16, so at most three CTAs (3 x 128 tensor-memory columns) share an SM
template <typename OP>
constexpr size_t tc_smem() { return (size_t)2 * 4 * TC_BM * TC_BK * sizeof(OP) + 128; }

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

struct TcTerm {
    const void *A;    // [Mp][Kp] table (hi pieces) in the operand type, zero padded; lo pieces follow
    const float *X;   // [N][K] FP32 field
};
struct TcOut {
    float *y;            // [M][N]
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

// One 128 x 128 tile of D per CTA, K streamed through two shared-memory stages.
template <typename OP>
__global__ void __launch_bounds__(TC_THREADS) k_tc_gemm(const __grid_constant__ TcJob J)
{
    if (J.done && *J.done) return;
    const TcOut &O = J.o[blockIdx.z];
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int ES = (int)sizeof(OP);
    constexpr int KC = TC_BK * ES / 16;             // 16-byte chunks per row and stage
    constexpr int ABYTES = TC_BM * TC_BK * ES, BBYTES = TC_BN * TC_BK * ES;
    constexpr int STAGE = 2 * (ABYTES + BBYTES);  // A hi, A lo, B hi, B lo
    constexpr uint32_t IDESC = tc_idesc(TcOp<OP>::fmt, TC_BM, TC_BN);
    uint64_t *mbar = (uint64_t *)(smem + 2 * STAGE);
    uint32_t *tslot = (uint32_t *)(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM;
    const long long n0 = (long long)blockIdx.y * TC_BN;

    if (tid == 0) {
        tc_mbar_init(&mbar[0]);
        tc_mbar_init(&mbar[1]);
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

    const int nkt = (J.K + TC_BK - 1) / TC_BK;
    const int total = nkt * O.nterm;
    bool ok = true;
    for (int it = 0; it < total; ++it) {
        const int s = it & 1;
        unsigned char *sA = smem + s * STAGE, *sAl = sA + ABYTES, *sB = sAl + ABYTES, *sBl = sB + BBYTES;
        // the MMAs that read this stage two iterations ago must be complete
        if (it >= 2 && ok) ok = tc_wait(&mbar[s], (uint32_t)(((it >> 1) - 1) & 1), J.err);
        const TcTerm tm = O.t[it / nkt];
        const int k0 = (it % nkt) * TC_BK;
        // A: rows m0.., K columns k0.. of the padded table, 16-byte chunks
        const unsigned char *Ag = (const unsigned char *)tm.A;
        const unsigned char *Agl = Ag + J.lo * ES;
        for (int c = tid; c < TC_BM * KC; c += TC_THREADS) {
            const int r = c / KC, kc = c % KC;
            const size_t go = ((size_t)(m0 + r) * J.Kp + k0) * ES + kc * 16;
            const int so = ((r >> 3) * KC + kc) * 128 + (r & 7) * 16;
            *(uint4 *)(sA + so) = *(const uint4 *)(Ag + go);
            *(uint4 *)(sAl + so) = *(const uint4 *)(Agl + go);
        }
        // B: rows n0.. of the field, converted to the operand type (zero outside)
        for (int e = tid; e < TC_BN * TC_BK; e += TC_THREADS) {
            const int r = e / TC_BK, k = e % TC_BK;
            const long long n = n0 + r;
            const int kk = k0 + k;
            const float v = (n < J.N && kk < J.K) ? tm.X[n * J.K + kk] : 0.0f;
            OP hi, lo;
            tc_split<OP>(v, hi, lo);
            const int so = ((r >> 3) * KC + ((k * ES) >> 4)) * 128 + (r & 7) * 16 + ((k * ES) & 15);
            *(OP *)(sB + so) = hi;
            *(OP *)(sBl + so) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        ok = __syncthreads_and(ok);
        if (tid == 0 && ok) {
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < TC_BK / TcOp<OP>::kmma; ++j) {
                const uint32_t sbo = (uint32_t)KC * 128u;
                const uint64_t ah = tc_desc(tc_saddr(sA) + 256u * j, 128u, sbo);
                const uint64_t al = tc_desc(tc_saddr(sAl) + 256u * j, 128u, sbo);
                const uint64_t bh = tc_desc(tc_saddr(sB) + 256u * j, 128u, sbo);
                const uint64_t bl = tc_desc(tc_saddr(sBl) + 256u * j, 128u, sbo);
                tc_mma<OP>(tmem, ah, bh, IDESC, (it > 0 || j > 0) ? 1u : 0u);  // hi * hi
                tc_mma<OP>(tmem, ah, bl, IDESC, 1u);                            // hi * lo
                tc_mma<OP>(tmem, al, bh, IDESC, 1u);                            // lo * hi
            }
            tc_commit(&mbar[s]);
        }
    }
    // the last commit covers every MMA issued before it
    if (ok) ok = tc_wait(&mbar[(total - 1) & 1], (uint32_t)(((total - 1) >> 1) & 1), J.err);
    tc_fence_after();
    // epilogue: warp w owns tensor-memory lanes 32w..32w+31 = rows m0+32w+lane
    const int m = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        uint32_t r[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
        if (!ok || m >= J.M) continue;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const long long n = n0 + c0 + jj;
            if (n >= J.N) break;
            float v = __uint_as_float(r[jj]);
            const size_t o = (size_t)m * J.N + n;
            if (O.scale) v *= O.scale[o];
            O.y[o] = v;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// ---- unfolded tables in the operand type -------------------------------------
// Forward tables Fphi/Fdphi [2][MpF][KpF] (hi, lo): row q (node), column k
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
    if (fwd) {
        Fphi[idx] = ph;
        Fphi[nF + idx] = pl;
        Fdphi[idx] = dh;
        Fdphi[nF + idx] = dl;
    } else {
        const long long e = idx - nF;
        Bphi[e] = ph;
        Bphi[nB + e] = pl;
        Bdphi[e] = dh;
        Bdphi[nB + e] = dl;
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
    void out(float *y, const float *scale, const float *x0, int t0, const float *x1 = nullptr, int t1 = 0)
    {
        const bool f = isfwd;
        TcOut &o = j.o[j.nout++];
        o.y = y;
        o.scale = scale;
        o.nterm = x1 ? 2 : 1;
        o.t[0] = TcTerm{f ? (const void *)tabF(t0) : (const void *)tabB(t0), x0};
        o.t[1] = TcTerm{x1 ? (f ? (const void *)tabF(t1) : (const void *)tabB(t1)) : nullptr, x1};
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
    float *ws = c->ws32;
    const float *Wa = c->Wa32, *Way = c->Wa32y, *Waz = c->Wa32z, *Wb = c->Wb32;  // W a_j per gradient term
    TcBuilder<OP> T{c, {}, true};
    if (g.d == 1) {
        float *H = ws, *Gx = ws + Q;
        T.fwd(1, done);
        T.out(H, Wb, x, 0);
        T.out(Gx, Wa, x, 1);
        LSG_TRY(T.launch(s));
        T.bwd(1, done);
        T.out(y, nullptr, H, 0, Gx, 1);
        return T.launch(s);
    }
    if (g.d == 2) {
        float *AP = ws, *AD = ws + Q * n1;                              // [Q][n1]
        float *H = ws + 2 * Q * n1, *Gy = H + Q * Q, *Gx = Gy + Q * Q;  // [Q][Q]
        float *P1 = AP, *P2 = AD;                                       // [n1][Q]
        T.fwd(n1, done);  // contract x
        T.out(AP, nullptr, x, 0);
        T.out(AD, nullptr, x, 1);
        LSG_TRY(T.launch(s));
        T.fwd(Q, done);  // contract y, pointwise W a / W b
        T.out(H, Wb, AP, 0);
        T.out(Gy, Way, AP, 1);
        T.out(Gx, Wa, AD, 0);
        LSG_TRY(T.launch(s));
        T.bwd(Q, done);  // back over x nodes
        T.out(P1, nullptr, H, 0, Gx, 1);
        T.out(P2, nullptr, Gy, 0);
        LSG_TRY(T.launch(s));
        T.bwd(n1, done);  // back over y nodes
        T.out(y, nullptr, P1, 0, P2, 1);
        return T.launch(s);
    }
    float *A0 = ws, *A1 = ws + Q * n1 * n1;
    float *B0 = ws + 2 * Q * n1 * n1, *B1 = B0 + Q * Q * n1, *B2 = B1 + Q * Q * n1;
    float *F0 = B2 + Q * Q * n1, *F1 = F0 + Q * Q * Q, *F2 = F1 + Q * Q * Q, *F3 = F2 + Q * Q * Q;
    float *H = F0, *Gz = F1, *Gy = F2, *Gx = F3;
    T.fwd(n1 * n1, done);
    T.out(A0, nullptr, x, 0);
    T.out(A1, nullptr, x, 1);
    LSG_TRY(T.launch(s));
    T.fwd(Q * n1, done);
    T.out(B0, nullptr, A0, 0);
    T.out(B1, nullptr, A0, 1);
    T.out(B2, nullptr, A1, 0);
    LSG_TRY(T.launch(s));
    T.fwd(Q * Q, done);
    T.out(H, Wb, B0, 0);
    T.out(Gz, Waz, B0, 1);
    T.out(Gy, Way, B1, 0);
    T.out(Gx, Wa, B2, 0);
    LSG_TRY(T.launch(s));
    float *Pa = B0, *Pb = B1, *Pc = B2;
    T.bwd(Q * Q, done);
    T.out(Pa, nullptr, H, 0, Gx, 1);
    T.out(Pb, nullptr, Gy, 0);
    T.out(Pc, nullptr, Gz, 0);
    LSG_TRY(T.launch(s));
    float *Ra = A0, *Rc = A1;
    T.bwd(n1 * Q, done);
    T.out(Ra, nullptr, Pa, 0, Pb, 1);
    T.out(Rc, nullptr, Pc, 0);
    LSG_TRY(T.launch(s));
    T.bwd(n1 * n1, done);
    T.out(y, nullptr, Ra, 0, Rc, 1);
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
