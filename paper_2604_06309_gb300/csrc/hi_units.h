// Work distribution shared by the history-integral kernels.
//
// A unit is (output index j, part p): the summation range of i is split into
// hi_parts(L, chunk) chunks of `chunk` indices (the last chunk takes the remainder).
// Each CTA takes a contiguous block of units and its
// warps take the block's units round-robin, so every SM gets the same number of units
// within one. A warp reduces its part with a fixed butterfly and writes the partial
// sums; the part that finishes last for a given j (a per-j counter, incremented after a
// memory fence) adds the partials in part order and writes S -- deterministic, and no
// unit ever waits for another.
#pragma once

#include "dmfe_internal.h"

__host__ __device__ __forceinline__ int hi_parts(int L, int chunk) { return L / chunk > 1 ? L / chunk : 1; }

__device__ __forceinline__ void hi_unit_block(int L, int chunk, int* ub, int* ue) {
    const long long U = (long long)hi_parts(L, chunk) * L;
    *ub = (int)(U * blockIdx.x / gridDim.x);
    *ue = (int)(U * (blockIdx.x + 1) / gridDim.x);
}

// Units are ordered chunk-major, so the warps of a CTA work on neighbouring output
// indices over the same i-chunk: their B2 reads follow nearby paths through the
// history and share L1 lines.
__device__ __forceinline__ void hi_unit_range(int u, int L, int chunk, int* j, int* i0, int* i1) {
    const int P = hi_parts(L, chunk);
    *j = u % L;
    const int p = u / L;
    *i0 = p * chunk;
    *i1 = p == P - 1 ? L : (p + 1) * chunk;
}

// Sum over the warp of a double-float value (fixed butterfly, FP32 pipes only).
__device__ __forceinline__ df df_warp_sum(df x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
        x = df_add(x, y);
    }
    return x;
}

// Called by one lane per unit with the reduced sums of that part.
__device__ __forceinline__ void hi_finish_unit(const double (&sums)[9], double c_at_0, int u, int L, int chunk,
                                               double* Spart, int* jcount, double* S) {
    const int P = hi_parts(L, chunk);
    const int j = u % L, p = u / L;
#pragma unroll
    for (int r = 0; r < 9; ++r) Spart[((size_t)p * 9 + r) * L + j] = sums[r];
    if (p == 0) S[(size_t)9 * L + j] = c_at_0;
    __threadfence();
    const int prev = atomicAdd(&jcount[j], 1);
    if (prev == P - 1) {
        __threadfence();
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            double a = 0.0;
            for (int q = 0; q < P; ++q) a += __ldcg(&Spart[((size_t)q * 9 + r) * L + j]);
            S[(size_t)r * L + j] = a;
        }
        jcount[j] = 0;
    }
}

// Copy a slot's view into shared memory (the batched kernels read it for every pair;
// from shared memory those reads are broadcasts instead of global loads).
__device__ __forceinline__ void load_view(SolverView& dst, const SolverView& src) {
    static_assert(sizeof(SolverView) % 4 == 0, "view size");
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int q = threadIdx.x; q < (int)(sizeof(SolverView) / 4); q += blockDim.x) d[q] = s[q];
}

// Work-balanced share of a batch for this CTA: the pairs of all slots are split evenly
// over the CTAs and each slot's share is mapped to its units in proportion (a slot's
// units carry nearly equal work). Calls f(k, lb, le) for every slot k with units [lb, le).
// Stages beyond the Dormand-Prince ones split only the slots that run them (woff_late).
template <typename F>
__device__ __forceinline__ void batch_for_my_units(const BatchTable* bt, int stg, F&& f) {
    const long long* woff = stg > kDP5Stages ? bt->woff_late : bt->woff;
    const long long W = woff[bt->count];
    const long long g0 = W * blockIdx.x / gridDim.x, g1 = W * (blockIdx.x + 1) / gridDim.x;
    int k = 0;
    while (k < bt->count && woff[k + 1] <= g0) ++k;
    for (; k < bt->count && woff[k] < g1; ++k) {
        const long long o = woff[k], Wk = woff[k + 1] - o;
        if (Wk <= 0) continue;
        const long long Uk = bt->uoff[k + 1] - bt->uoff[k];
        const long long a = (g0 > o ? g0 : o) - o, e = (g1 < o + Wk ? g1 : o + Wk) - o;
        const int lb = (int)(a * Uk / Wk), le = (int)(e * Uk / Wk);
        if (le > lb) f(k, lb, le);
    }
}
