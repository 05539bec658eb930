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

#include <vector>

#include "dmfe_internal.h"

// Work-unit size value that selects the flat split (single solves only): the L^2 pairs in
// row-major order (output index j, then summation index i) are cut into one equal segment
// per warp of the launch, and a warp takes its segment row by row. The pieces of one row are
// that output index's parts, in order. Every warp gets the same number of pairs, so all SMs
// and warp slots finish together.
constexpr int kFlatSplit = -1;

__host__ __device__ __forceinline__ int hi_parts(int L, int chunk) {
    return (chunk > 0 && L / chunk > 1) ? L / chunk : 1;
}

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

// The flat split needs at least 256 pairs per warp (8 per lane), which also keeps every
// segment non-empty and a row's parts within the partial-sum buffer (L / 32 parts).
__host__ __device__ __forceinline__ bool flat_split_fits(int L, long long warps) {
    return warps > 0 && (long long)L * L >= 256 * warps && L >= 512;
}

// Calls f(j, i0, i1, part, nparts) for each piece of work of this warp: the units [ub, ue)
// of its CTA round-robin over the CTA's warps, or under the flat split the rows of the
// warp's segment, read from the split's tables (flat_split_tables): seg[g] = {first pair, its
// row} of segment g (seg[G] = {L^2, L}), row[j] = {first segment, segments} of row j.
template <typename F>
__device__ __forceinline__ void hi_for_items(int L, int chunk, int ub, int ue, const int2* __restrict__ seg,
                                             const int2* __restrict__ row, F&& f) {
    if (chunk == kFlatSplit) {
        const int g = (int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
        const int2 a = seg[g], b = seg[g + 1];
        int j = a.y;
        for (int q = a.x; q < b.x; ++j) {
            const int rb = j * L;
            const int qe = b.x < rb + L ? b.x : rb + L;
            const int2 r = row[j];
            f(j, q - rb, qe - rb, g - r.x, r.y);
            q = qe;
        }
        return;
    }
    const int P = hi_parts(L, chunk);
    for (int u = ub + (threadIdx.x >> 5); u < ue; u += (int)(blockDim.x >> 5)) {
        int j, i0, i1;
        hi_unit_range(u, L, chunk, &j, &i0, &i1);
        f(j, i0, i1, u / L, P);
    }
}

// Host: the tables of the flat split over G warps. Segment g covers the pairs
// [g L^2 / G, (g + 1) L^2 / G) in row-major order; pair q lies in segment
// ((q + 1) G - 1) / L^2, so row j's parts are the segments from that of its first pair to
// that of its last. seg has G + 1 entries, row L.
inline void flat_split_tables(int L, int G, std::vector<int2>& seg, std::vector<int2>& row) {
    const long long LL = (long long)L * L;
    seg.resize((size_t)G + 1);
    for (int g = 0; g <= G; ++g) {
        const long long q = (long long)g * LL / G;
        seg[g] = make_int2((int)q, (int)(q / L));
    }
    row.resize(L);
    for (int j = 0; j < L; ++j) {
        const long long rb = (long long)j * L;
        const long long s0 = ((rb + 1) * G - 1) / LL, s1 = ((rb + L) * G - 1) / LL;
        row[j] = make_int2((int)s0, (int)(s1 - s0 + 1));
    }
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

// Called by one lane per piece of work with the reduced sums of part p (of P) of output
// index j.
__device__ __forceinline__ void hi_finish_part(const double (&sums)[9], double c_at_0, int j, int p, int P, int L,
                                               double* Spart, int* jcount, double* S) {
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
