// stencil.cuh -- geometry of the stencil storage of M and its ILU(0) factors.
//
// Row r = (i, j, k) (i fastest) has S = (2w+1)^d slots, one per offset
// (dx, dy, dz) in the box |d*| <= w = T+2, ordered lexicographically with dx
// fastest, so slot order is column order; slot Sc is the diagonal.
#pragma once

#include "lsg_internal.cuh"

namespace lsg {

struct StencilGeo {
    int d, n1, w, W1, S, Sc, SL, SU, T, has_b;
    long long n, nlines;
    signed char ta[9], tb[3];  // truncation degrees: ta[3 j + i] of a_j in direction i, tb[i] of b
};

static inline StencilGeo sgeo(const Geom &g)
{
    StencilGeo G{g.d, g.n1, g.w, g.W1, g.S, g.Sc, g.SL, g.SU, g.T, g.has_b, g.n, g.nlines, {}, {}};
    for (int j = 0; j < 3; ++j) {
        G.tb[j] = (signed char)g.tb[j];
        for (int i = 0; i < 3; ++i) G.ta[3 * j + i] = (signed char)g.ta[j][i];
    }
    return G;
}

__device__ __forceinline__ void slot_offsets(const StencilGeo &G, int s, int &dx, int &dy, int &dz)
{
    dx = s % G.W1 - G.w;
    dy = (G.d >= 2) ? (s / G.W1) % G.W1 - G.w : 0;
    dz = (G.d == 3) ? s / (G.W1 * G.W1) - G.w : 0;
}
__device__ __forceinline__ int slot_index(const StencilGeo &G, int dx, int dy, int dz)
{
    return (dx + G.w) + G.W1 * ((G.d >= 2 ? dy + G.w : 0) + G.W1 * (G.d == 3 ? dz + G.w : 0));
}

// Structural pattern of M (reading of NZ(M) in Sec. 4.2): union over the
// Kronecker terms of their band supports.  Term j (stiffness in direction j, the
// series of a_j) has a stiffness band (|o| <= degree) in direction j and mass
// bands (|o| <= degree + 2; only even offsets for degree 0) in the others, each
// with a_j's degree in that direction; the reaction term, when present, has mass
// bands of b's degrees in every direction.
__device__ __forceinline__ bool stiff_band(int o, int T) { return o <= T && o >= -T; }
__device__ __forceinline__ bool mass_band(int o, int T)
{
    int a = o < 0 ? -o : o;
    return a <= T + 2 && (T > 0 || (a & 1) == 0);
}
__device__ inline bool structural(const StencilGeo &G, int dx, int dy, int dz)
{
    int o[3] = {dx, dy, dz};
    for (int j = 0; j < G.d; ++j) {
        bool ok = stiff_band(o[j], G.ta[3 * j + j]);
        for (int i = 0; i < G.d && ok; ++i)
            if (i != j) ok = mass_band(o[i], G.ta[3 * j + i]);
        if (ok) return true;
    }
    if (G.has_b) {
        bool mm = true;
        for (int i = 0; i < G.d; ++i) mm = mm && mass_band(o[i], G.tb[i]);
        if (mm) return true;
    }
    return false;
}

// Bounded spin on a completion word (all lanes poll; returns false on timeout
// or when another warp already reported an error).
__device__ __forceinline__ bool wait_flag(const unsigned *flag, unsigned need, int *err)
{
    long long t0 = 0;
    for (int it = 0;; ++it) {
        if (ld_acquire(flag) >= need) return true;
        if (it == 0) t0 = clock64();
        if ((it & 15) == 15 && *(volatile int *)err != 0) return false;
        if (clock64() - t0 > kSpinBudgetCycles) {
            set_err(err, DERR_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
}

// Like wait_flag, but remembers the last value seen in *seen, so that a caller
// that polls the same word row after row only goes to memory when the cached
// value is not enough.
__device__ __forceinline__ bool wait_flag_cached(const unsigned *flag, unsigned need, int *err, unsigned *seen,
                                                 long long budget)
{
    if (*seen >= need) return true;
    long long t0 = 0;
    for (int it = 0;; ++it) {
        unsigned v = ld_acquire(flag);
        if (v >= need) {
            *seen = v;
            return true;
        }
        if (it == 0) t0 = clock64();
        if ((it & 15) == 15 && *(volatile int *)err != 0) return false;
        if (clock64() - t0 > budget) {
            set_err(err, DERR_TIMEOUT);
            return false;
        }
    }
}

}  // namespace lsg
