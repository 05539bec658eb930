// History integrals of one Runge-Kutta stage (Secs. 3.3, 3.4, Eq. int).
//
// For every output index j (t' = theta_j t) and summation index i the kernel forms
//   A   the current stage row at phi1 = theta_i theta_j and phi2 = theta_j + (1 - theta_j) theta_i
//       (index-space Lagrange stencil, rows K = f''(C) R, D = f'(C), C, R in shared memory),
//   B1  (C, R)(theta_j t, theta_i): on-grid in theta, cubic Hermite in t between the two
//       stored slices around theta_j t,
//   B2  (C, R)(phi2 t, theta_j / phi2): Lagrange stencil in theta on the two slices around
//       phi2 t, then cubic Hermite in t,
// and accumulates the nine nu-weighted products S[0..8] of dmfe.h plus S[9] = C(theta_j t, 0).
// Times in (t_last, t] come from the quadratic through the last slice and the stage row.
//
// Mapping (hi_units.h): a warp takes a unit (j, chunk of 256 i), lanes stride over
// i (coalesced table and B1 rows); each lane sums its terms in i order, the warp reduces
// with a fixed butterfly and the last chunk to finish adds the chunks in a fixed
// order, so results are deterministic. The slice containing phi2 t is found from a
// per-stage table cell -> slice (phi2 lies in grid cell floor(x2)) and a short walk.
//
// Precision variants:
//   FP64: every value in FP64, stencil positions from FP64 tables.
//   FP32: stage row, history replica and interpolation in FP32, stencil positions from
//         fixed-point tables (19 fraction bits), per-lane Kahan-compensated sums, slice
//         times handled as complements v_n = (t - t_n)/t so that 1 - phi2 = omega_j omega_i
//         keeps its relative precision near the diagonal; per-j quantities, the warp
//         reduction and the output stay FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dmfe_internal.h"
#include "hi_units.h"

namespace {

constexpr int HI_THREADS = 512;
constexpr int HI_WARPS = HI_THREADS / 32;

// 1 / prod_{m != k} (k - m) = (-1)^{SW-1-k} / (k! (SW-1-k)!), evaluated by the compiler.
__host__ __device__ constexpr double lagrange_denom(int k, int sw) {
    double c = 1.0;
    for (int m = 0; m < sw; ++m)
        if (m != k) c /= double(k - m);
    return c;
}

template <int SW>
struct LagrangeDenoms {
    float v[SW];
    __host__ __device__ constexpr LagrangeDenoms() : v() {
        for (int k = 0; k < SW; ++k) v[k] = (float)lagrange_denom(k, SW);
    }
};

// Lagrange weights on nodes 0..SW-1 at u (FP32): w_k = prod_{m != k} (u - m) / (k - m), the
// products as prefix and suffix products, the denominators compile-time constants.
template <int SW>
__device__ __forceinline__ void lagrange(float u, float (&w)[SW]) {
    constexpr LagrangeDenoms<SW> den{};
    float pre[SW], suf[SW];
    pre[0] = 1.f;
#pragma unroll
    for (int k = 1; k < SW; ++k) pre[k] = pre[k - 1] * (u - float(k - 1));
    suf[SW - 1] = 1.f;
#pragma unroll
    for (int k = SW - 2; k >= 0; --k) suf[k] = suf[k + 1] * (u - float(k + 1));
#pragma unroll
    for (int k = 0; k < SW; ++k) w[k] = pre[k] * suf[k] * den.v[k];
}

template <int SW>
__device__ __forceinline__ int stencil_base(int fl, int L) {
    int b = fl - SW / 2 + 1;
    b = b < 0 ? 0 : b;
    return b > L - SW ? L - SW : b;
}

// Fixed-point position p (FIX_FRAC_BITS fraction bits) -> stencil base b and the offset
// u = x - b. m = p - b 2^19 < 2^23, so the float with bit pattern 0x4B000000 + m is 2^23 + m
// exactly and the subtraction gives float(m) exactly: the same value as a conversion, from
// the integer and FP32 pipes (GB300 issues conversions on its FP64 unit).
template <int SW>
__device__ __forceinline__ int fix_stencil(uint32_t p, int L, float& u) {
    const int b = stencil_base<SW>((int)(p >> FIX_FRAC_BITS), L);
    const uint32_t m = p - ((uint32_t)b << FIX_FRAC_BITS);
    u = (__int_as_float(0x4B000000u | m) - 8388608.0f) * (1.0f / (float)(1u << FIX_FRAC_BITS));
    return b;
}

// Time weights: value = w0 Y[a0] + w1 dY[a0] + w2 Y[a1] + w3 dY[a1]; a1 < 0 means the
// stage row (only its value is used, w3 = 0). FP64, shared by both variants (per j).
struct TimeW {
    int a0, a1;
    double w0, w1, w2, w3;
};

// Slice times are non-negative, so their IEEE bit patterns order like the values: the slice
// walk compares 64-bit integers (integer pipe) instead of doubles (the FP64 pipe, GB300's
// bottleneck here).
__device__ __forceinline__ long long tbits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ FP64 variant
// Body shared by the single-instance and batched kernels: processes units [ub, ue) of
// solver v with the warps of this CTA (shared memory is reloaded for v).
// LOGR: compiled with the log-R reads (taken where the solver has log-R tables); without
// it the default kernel carries none of that code.
template <int SW, bool LOGR>
__device__ __forceinline__ void hi_f64_body(const SolverView& v, const double* __restrict__ row, double t_arg,
                                            int from_state, double* __restrict__ S, int ub, int ue) {
    extern __shared__ __align__(32) unsigned char smraw[];
    const DevState* st = v.st;
    if (stage_off(st, from_state)) return;
    const int L = v.L;
    const int n = st->n;
    const int act = st->active;
    const double t = from_state ? st->t_stage : t_arg;
    const dbl4* __restrict__ H = v.hist[act];
    const dbl8* __restrict__ HC = v.hcoef[act];
    const dbl4* __restrict__ LC = LOGR ? v.lcoef[act] : nullptr;  // log-R mode only
    const double* __restrict__ ht = v.ht[act];
    // Slice times with the stage time appended when the stage lies beyond the last slice:
    // the quadratic extension is then the virtual interval n-1 = [t_last, t], whose
    // monomial coefficients the prep kernel wrote into row n-1 of HC, and every pair takes
    // the same Horner path (no divergence near theta = 1).
    const double tl = ht[n - 1];
    const bool ext = t > tl;
    const double hx = t - tl;
    dbl4* srow = reinterpret_cast<dbl4*>(smraw);            // [L] {K, D, C, R}
    double* sht = reinterpret_cast<double*>(srow + L);              // [cap + 1] slice times
    double* sinvh = sht + v.cap + 1;                                // [cap + 1] 1/(t_{k+1} - t_k)
    int* scell = reinterpret_cast<int*>(sinvh + v.cap + 1);         // [L]
    // the stage row {K, D, C, R} and the reciprocal interval widths, prepared once per stage
    // by the prep kernel
    for (int i = threadIdx.x; i < L; i += blockDim.x) srow[i] = v.row64[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sht[i] = ht[i];
        sinvh[i] = v.slice64[i];
    }
    if (threadIdx.x == 0) sht[n] = t;
    for (int m = threadIdx.x; m < L; m += blockDim.x) scell[m] = v.cell[m];
    __syncthreads();
    const int kmax = ext ? n - 1 : n - 2;  // last interval a B2 point can fall in
    const int lane = threadIdx.x & 31;
    const double* __restrict__ theta = v.theta;
    const double* __restrict__ omega = v.omega;
    const double* __restrict__ nu = v.nu;
    const int chunk = v.hi_chunk;

    hi_for_items(L, chunk, ub, ue, v.flat_seg, v.flat_row, [&](int j, int i0, int i1, int part, int nparts) {
        // the stage time of B2, tau2 = phi2 t = theta_j t + (omega_j t) theta_i, by one FMA
        const double thj_t = theta[j] * t, omj_t = omega[j] * t;
        TimeW b1;
        double s1;
        {
            const B1Desc d = v.b1[j];
            b1.a0 = d.a0; b1.a1 = d.a1;
            b1.w0 = d.w[0]; b1.w1 = d.w[1]; b1.w2 = d.w[2]; b1.w3 = d.w[3];
            s1 = d.s;
        }
        // an interval of the history or the virtual extension interval (a1 < 0); else a
        // single stored slice at the stage time t = 0
        const bool b1_interior = b1.a1 == b1.a0 + 1 || b1.a1 < 0;
        const bool b1ok = DMFE_IN_BOUNDS(v.st, b1.a0 >= 0 && b1.a0 < n && b1.a1 < n, 1);
        constexpr size_t WTS = 8 + 8 * SW;  // bytes per stencil entry
        const unsigned char* __restrict__ w1r = v.wt1 + (size_t)j * L * WTS;
        const unsigned char* __restrict__ w2r = v.wt2 + (size_t)j * L * WTS;
        const unsigned char* __restrict__ w3r = v.wt3 + (size_t)j * L * WTS;
        double acc[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) acc[r] = 0.0;
        double c_at_0 = 0.0;
        for (int i = i0 + lane; i < i1; i += 32) {
            // ---- B1: on-grid column i at time theta_j t
            double CB1 = 0.0, RB1 = 0.0;
            if (!b1ok) {
            } else if (b1_interior) {
                const dbl8 c = HC[(size_t)b1.a0 * L + i];
                CB1 = c.c0 + s1 * (c.c1 + s1 * (c.c2 + s1 * c.c3));
                RB1 = c.r0 + s1 * (c.r1 + s1 * (c.r2 + s1 * c.r3));
                if (LC) {
                    const dbl4 l = LC[(size_t)b1.a0 * L + i];
                    if (!isnan(l.x)) RB1 = exp(l.x + s1 * (l.y + s1 * (l.z + s1 * l.w)));
                }
            } else {
                dbl4 h0 = H[(size_t)b1.a0 * L + i];
                CB1 = b1.w0 * h0.x + b1.w1 * h0.y;
                RB1 = b1.w0 * h0.z + b1.w1 * h0.w;
                if (b1.a1 >= 0) {
                    dbl4 h1 = H[(size_t)b1.a1 * L + i];
                    CB1 += b1.w2 * h1.x + b1.w3 * h1.y;
                    RB1 += b1.w2 * h1.z + b1.w3 * h1.w;
                } else {
                    dbl4 r1 = srow[i];
                    CB1 += b1.w2 * r1.z;
                    RB1 += b1.w2 * r1.w;
                }
            }
            // ---- A1: current row at phi1
            double KA1 = 0, DA1 = 0, CA1 = 0, RA1 = 0;
            {
                const unsigned char* e = w1r + (size_t)i * WTS;
                const int b = *reinterpret_cast<const int*>(e);
                double w[SW];
#pragma unroll
                for (int k = 0; k < SW; ++k) w[k] = reinterpret_cast<const double*>(e + 8)[k];
                if (DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 2)) {
#pragma unroll
                    for (int k = 0; k < SW; ++k) {
                        dbl4 q = srow[b + k];
                        KA1 += w[k] * q.x; DA1 += w[k] * q.y; CA1 += w[k] * q.z; RA1 += w[k] * q.w;
                    }
                }
            }
            // ---- A2: current row at phi2
            double KA2 = 0, RA2 = 0;
            int base2;
            {
                const unsigned char* e = w2r + (size_t)i * WTS;
                const int b = *reinterpret_cast<const int*>(e);
                base2 = b;
                double w[SW];
#pragma unroll
                for (int k = 0; k < SW; ++k) w[k] = reinterpret_cast<const double*>(e + 8)[k];
                if (DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 3)) {
#pragma unroll
                    for (int k = 0; k < SW; ++k) {
                        dbl4 q = srow[b + k];
                        KA2 += w[k] * q.x; RA2 += w[k] * q.w;
                    }
                }
            }
            // ---- B2: theta position psi on the slices around phi2 t
            double CB2, RB2;
            {
                const double tau2 = fma(omj_t, theta[i], thj_t);
                const long long taub = tbits(tau2);
                const unsigned char* e = w3r + (size_t)i * WTS;
                const int b = *reinterpret_cast<const int*>(e);
                double w[SW];
#pragma unroll
                for (int k = 0; k < SW; ++k) w[k] = reinterpret_cast<const double*>(e + 8)[k];
                if (kmax >= 0) {
                    // the slice interval (or the virtual extension interval) by a short walk
                    // from the cell hint; each stencil node's interpolant by Horner's rule
                    // in s (6 FMAs), then the theta stencil (2 FMAs)
                    int cell = base2 + SW / 2 - 1;  // the grid cell of phi2 (the walk corrects)
                    cell = cell < 0 ? 0 : (cell > L - 1 ? L - 1 : cell);
                    int k = scell[cell];
                    while (k < kmax && tbits(sht[k + 1]) <= taub) ++k;
                    while (k > 0 && tbits(sht[k]) > taub) --k;
                    const double sg = (tau2 - sht[k]) * sinvh[k];
                    const dbl8* __restrict__ P = HC + (size_t)k * L + b;
                    CB2 = 0.0;
                    RB2 = 0.0;
                    const bool ok2 = DMFE_IN_BOUNDS(v.st, k >= 0 && k <= kmax && b >= 0 && b <= L - SW, 4);
#pragma unroll
                    for (int m = 0; m < (ok2 ? SW : 0); ++m) {
                        const dbl8 c = P[m];
                        CB2 += w[m] * (c.c0 + sg * (c.c1 + sg * (c.c2 + sg * c.c3)));
                        RB2 += w[m] * (c.r0 + sg * (c.r1 + sg * (c.r2 + sg * c.r3)));
                    }
                    if (LC && ok2) {
                        // log-R mode: the same interpolant on log R; a NaN (some node's R not
                        // positive) propagates through the sum and keeps the linear value
                        const dbl4* __restrict__ Q = LC + (size_t)k * L + b;
                        double lr = 0.0;
#pragma unroll
                        for (int m = 0; m < SW; ++m) {
                            const dbl4 l = Q[m];
                            lr += w[m] * (l.x + sg * (l.y + sg * (l.z + sg * l.w)));
                        }
                        if (!isnan(lr)) RB2 = exp(lr);
                    }
                } else {
                    // a single stored slice and the stage at its time
                    CB2 = 0.0;
                    RB2 = 0.0;
                    bool pos = true;
                    double lr = 0.0;
                    const bool ok1 = DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 5);
#pragma unroll
                    for (int m = 0; m < (ok1 ? SW : 0); ++m) {
                        const dbl4 q = H[b + m];
                        CB2 += w[m] * q.x;
                        RB2 += w[m] * q.z;
                        pos = pos && q.z > 0.0;
                        lr += w[m] * (q.z > 0.0 ? log(q.z) : 0.0);
                    }
                    if (LC && pos) RB2 = exp(lr);
                }
            }
            const double f1a = fp1(v.poly, CB1), f2a = fp2(v.poly, CB1);
            const double f1b = fp1(v.poly, CB2), f2b = fp2(v.poly, CB2);
            // the weight nu_i is in the A1 and A2 stencil weights (KA1, DA1, CA1, RA1, KA2,
            // RA2 carry it); only the last sum, which has no A factor, multiplies by it
            acc[0] += KA1 * CB1;
            acc[1] += KA2 * CB2;
            acc[2] += DA1 * RB1;
            acc[3] += KA2 * RB2;
            acc[4] += (f2a * CA1) * RB1;
            acc[5] += f1a * RA1;
            acc[6] += f1b * RA2;
            acc[7] += (f2b * RB2) * RA2;
            acc[8] += (f2a * CB1 + f1a) * (nu[i] * RB1);
            if (i == 0) c_at_0 = CB1;
        }
        double sums[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) sums[r] = warp_sum(acc[r]);
        if (lane == 0) hi_finish_part(sums, c_at_0, j, part, nparts, L, v.Spart, v.jcount, S);
    });
}

// ------------------------------------------------------------------ FP32 variant
struct Kahan {
    float s, c;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <int SW>
__device__ __forceinline__ void hi_f32_body(const SolverView& v, const double* __restrict__ row, double t_arg,
                                            int from_state, double* __restrict__ S, int ub, int ue) {
    extern __shared__ __align__(32) unsigned char smraw[];
    const DevState* st = v.st;
    if (stage_off(st, from_state)) return;
    const int L = v.L;
    const int n = st->n;
    const int act = st->active;
    const double t = from_state ? st->t_stage : t_arg;
    const float4* __restrict__ H = v.hist32[act];
    const double* __restrict__ ht = v.ht[act];
    // slices, and for a stage beyond the last slice the virtual slice n at the stage time
    // (the prep kernel's quadratic extension in Hermite form): all pairs take one path
    const bool ext = t > ht[n - 1];
    const int nsl = ext ? n + 1 : n;
    const int kmax = nsl - 2;
    const float4* __restrict__ VR = v.vrow32;
    float4* srow = reinterpret_cast<float4*>(smraw);               // [L] {K, D, C, R}
    float* sv = reinterpret_cast<float*>(srow + L);                 // [cap + 1] (t - t_k)/t
    float* sinv = sv + v.cap + 1;                                   // [cap + 1] 1/(v_k - v_{k+1})
    float* sdt = sinv + v.cap + 1;                                  // [cap + 1] t_{k+1} - t_k
    int* scell = reinterpret_cast<int*>(sdt + v.cap + 1);           // [L]
    // the stage row in FP32 and the slice constants, prepared once per stage by the prep kernel
    for (int i = threadIdx.x; i < L; i += blockDim.x) srow[i] = v.row32f[i];
    for (int i = threadIdx.x; i < nsl; i += blockDim.x) {
        const float4 e = v.slice32[i];
        sv[i] = e.x;
        sinv[i] = e.y;
        sdt[i] = e.z;
    }
    for (int m = threadIdx.x; m < L; m += blockDim.x) scell[m] = v.cell[m];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float* __restrict__ om32 = v.omega32;
    const float* __restrict__ nu32 = v.nu32;
    const int chunk = v.hi_chunk;

    hi_for_items(L, chunk, ub, ue, v.flat_seg, v.flat_row, [&](int j, int i0, int i1, int part, int nparts) {
        const float omj = om32[j];
        TimeW b1d;
        float bw0, bw1, bw2, bw3;
        {
            const B1Desc d = v.b1[j];
            b1d.a0 = d.a0; b1d.a1 = d.a1;
            bw0 = d.wd[0].hi; bw1 = d.wd[1].hi; bw2 = d.wd[2].hi; bw3 = d.wd[3].hi;
        }
        const uint32_t* __restrict__ p1r = v.p1 + (size_t)j * L;
        const uint32_t* __restrict__ p2r = v.p2 + (size_t)j * L;
        const uint32_t* __restrict__ p3r = v.p3 + (size_t)j * L;
        const bool b1ok = DMFE_IN_BOUNDS(v.st, b1d.a0 >= 0 && b1d.a0 < n && b1d.a1 < n, 11);
        const float4* __restrict__ H0 = H + (size_t)(b1ok ? b1d.a0 : 0) * L;
        const float4* __restrict__ H1 = (b1d.a1 >= 0 && b1ok) ? H + (size_t)b1d.a1 * L : nullptr;
        Kahan acc[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) { acc[r].s = 0.f; acc[r].c = 0.f; }
        float c_at_0 = 0.f;
        // software pipeline: the loads that head each pair's dependence chains (positions,
        // omega_i, nu_i and the B1 history entries) are issued one index ahead
        int i = i0 + lane;
        uint32_t n1 = 0, n2 = 0, n3 = 0;
        float nom = 0.f, nnu = 0.f;
        float4 nh0 = make_float4(0.f, 0.f, 0.f, 0.f), nh1 = nh0;
        if (i < i1) {
            n1 = p1r[i]; n2 = p2r[i]; n3 = p3r[i]; nom = om32[i]; nnu = nu32[i];
            nh0 = H0[i];
            nh1 = H1 ? H1[i] : srow[i];
        }
        for (; i < i1; i += 32) {
            const uint32_t pp1 = n1, pp2 = n2, pp3 = n3;
            const float omi = nom, nui = nnu;
            const float4 h0 = nh0, h1 = nh1;
            const int in = i + 32;
            if (in < i1) {
                n1 = p1r[in]; n2 = p2r[in]; n3 = p3r[in]; nom = om32[in]; nnu = nu32[in];
                nh0 = H0[in];
                nh1 = H1 ? H1[in] : srow[in];
            }
            // ---- B2 slice walk and stencil base. Up to stencil width 6 the gathers are
            // issued here, first, so that the A and B1 arithmetic below covers their
            // latency; wider stencils load them where they are used (holding 2 x SW gathered
            // entries across that arithmetic would spill registers)
            constexpr bool kEarly = SW <= 6;
            int a0 = 0, a1 = -1, b3 = 0;
            float sg = 0.f, hh = 0.f, ub = 0.f;
            bool ok3 = true;
            float4 g0[kEarly ? SW : 1], g1[kEarly ? SW : 1];
            auto walk = [&]() {
                // complement of phi2: 1 - phi2 = omega_j omega_i; slice k holds v_k = (t - t_k)/t
                const float uc = omj * omi;
                if (kmax >= 0) {
                    const int cell = (int)(pp2 >> FIX_FRAC_BITS);
                    int k = DMFE_IN_BOUNDS(v.st, cell < L, 14) ? scell[cell] : 0;
                    while (k < kmax && sv[k + 1] >= uc) ++k;
                    while (k > 0 && sv[k] < uc) --k;
                    sg = (sv[k] - uc) * sinv[k];
                    hh = sdt[k];
                    a0 = k; a1 = k + 1;
                }
                b3 = fix_stencil<SW>(pp3, L, ub);
                ok3 = DMFE_IN_BOUNDS(v.st, a0 >= 0 && a0 < n && a1 < nsl && b3 >= 0 && b3 <= L - SW, 15);
            };
            if constexpr (kEarly) {
                walk();
                const float4* __restrict__ s0 = H + (size_t)(ok3 ? a0 : 0) * L + (ok3 ? b3 : 0);
#pragma unroll
                for (int k = 0; k < SW; ++k) g0[k] = s0[k];
                if (a1 >= 0 && ok3) {
                    const float4* __restrict__ s1 = (a1 < n ? H + (size_t)a1 * L : VR) + b3;
#pragma unroll
                    for (int k = 0; k < SW; ++k) g1[k] = s1[k];
                } else {
#pragma unroll
                    for (int k = 0; k < SW; ++k) g1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            // ---- B1 (h1 is the stage row's entry when a1 < 0; only its value is used)
            float CB1 = bw0 * h0.x + bw1 * h0.y;
            float RB1 = bw0 * h0.z + bw1 * h0.w;
            if (H1) {
                CB1 += bw2 * h1.x + bw3 * h1.y;
                RB1 += bw2 * h1.z + bw3 * h1.w;
            } else {
                CB1 += bw2 * h1.z;
                RB1 += bw2 * h1.w;
            }
            // ---- A1, A2: the stage row at phi1 and phi2
            float KA1 = 0.f, DA1 = 0.f, CA1 = 0.f, RA1 = 0.f;
            {
                float uu;
                const int b = fix_stencil<SW>(pp1, L, uu);
                float w[SW];
                lagrange<SW>(uu, w);
                const bool ok = DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 12);
#pragma unroll
                for (int k = 0; k < (ok ? SW : 0); ++k) {
                    float4 q = srow[b + k];
                    KA1 += w[k] * q.x; DA1 += w[k] * q.y; CA1 += w[k] * q.z; RA1 += w[k] * q.w;
                }
            }
            float KA2 = 0.f, RA2 = 0.f;
            {
                float uu;
                const int b = fix_stencil<SW>(pp2, L, uu);
                float w[SW];
                lagrange<SW>(uu, w);
                const bool ok = DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 13);
#pragma unroll
                for (int k = 0; k < (ok ? SW : 0); ++k) {
                    float4 q = srow[b + k];
                    KA2 += w[k] * q.x; RA2 += w[k] * q.w;
                }
            }
            if constexpr (!kEarly) walk();
            // ---- B2: the theta stencil at psi on both slices, then cubic Hermite in time
            float CB2, RB2;
            {
                float w0 = 1.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;  // a single slice: its value
                if (kmax >= 0) {
                    const float om = 1.f - sg;
                    w0 = (1.f + 2.f * sg) * om * om;
                    w1 = sg * om * om * hh;
                    w2 = sg * sg * (3.f - 2.f * sg);
                    w3 = sg * sg * (sg - 1.f) * hh;
                }
                float w[SW];
                lagrange<SW>(ub, w);
                float c0 = 0.f, dc0 = 0.f, r0 = 0.f, dr0 = 0.f, c1 = 0.f, dc1 = 0.f, r1 = 0.f, dr1 = 0.f;
                const float4* __restrict__ s0 = H + (size_t)a0 * L + b3;
#pragma unroll
                for (int k = 0; k < (ok3 ? SW : 0); ++k) {
                    const float4 q = kEarly ? g0[kEarly ? k : 0] : s0[k];
                    c0 += w[k] * q.x; dc0 += w[k] * q.y; r0 += w[k] * q.z; dr0 += w[k] * q.w;
                }
                if (a1 >= 0 && ok3) {
                    const float4* __restrict__ s1 = (a1 < n ? H + (size_t)a1 * L : VR) + b3;
#pragma unroll
                    for (int k = 0; k < SW; ++k) {
                        const float4 q = kEarly ? g1[kEarly ? k : 0] : s1[k];
                        c1 += w[k] * q.x; dc1 += w[k] * q.y; r1 += w[k] * q.z; dr1 += w[k] * q.w;
                    }
                }
                CB2 = w0 * c0 + w1 * dc0 + w2 * c1 + w3 * dc1;
                RB2 = w0 * r0 + w1 * dr0 + w2 * r1 + w3 * dr1;
            }
            float f1a, f2a, f1b, f2b;
            fp12_pair(v.poly, CB1, CB2, f1a, f2a, f1b, f2b);
            acc[0].add(nui * (KA1 * CB1));
            acc[1].add(nui * (KA2 * CB2));
            acc[2].add(nui * (DA1 * RB1));
            acc[3].add(nui * (KA2 * RB2));
            acc[4].add(nui * (f2a * RB1 * CA1));
            acc[5].add(nui * (f1a * RA1));
            acc[6].add(nui * (f1b * RA2));
            acc[7].add(nui * (f2b * RB2 * RA2));
            acc[8].add(nui * ((f2a * CB1 + f1a) * RB1));
            if (i == 0) c_at_0 = CB1;
        }
        double sums[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            // the compensated pair (s, -c) reduced as a double-float on the FP32 pipes
            const df x = df_warp_sum(fast_two_sum(acc[r].s, -acc[r].c));
            sums[r] = lane == 0 ? df_to_d(x) : 0.0;
        }
        if (lane == 0) hi_finish_part(sums, (double)c_at_0, j, part, nparts, L, v.Spart, v.jcount, S);
    });
}

template <int SW, bool LOGR>
__global__ void __launch_bounds__(HI_THREADS, 1) k_hi_f64(SolverView v, const double* __restrict__ row,
                                                       double t_arg, int from_state, double* __restrict__ S) {
    int ub, ue;
    hi_unit_block(v.L, v.hi_chunk, &ub, &ue);
    hi_f64_body<SW, LOGR>(v, row, t_arg, from_state, S, ub, ue);
}

template <int SW>
__global__ void __launch_bounds__(HI_THREADS, 1) k_hi_f32(SolverView v, const double* __restrict__ row,
                                                       double t_arg, int from_state, double* __restrict__ S) {
    int ub, ue;
    hi_unit_block(v.L, v.hi_chunk, &ub, &ue);
    hi_f32_body<SW>(v, row, t_arg, from_state, S, ub, ue);
}

// Batched: one persistent launch per stage over the units of every slot of the batch
// table; each CTA takes an equal share of the batch's pairs (batch_for_my_units). The slot
// loop's state stays live around the body, so the batched kernels run 384-thread CTAs
// (up to 168 registers a thread): with 512 threads (128 registers) they spilled.
constexpr int BATCH_THREADS = 384;

template <int SW, int PREC>
__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batch_hi(const BatchTable* __restrict__ bt, int stg) {
    __shared__ __align__(16) SolverView sview;
    batch_for_my_units(bt, stg, [&](int k, int lb, int le) {
        __syncthreads();  // the previous slot's shared-memory data are no longer read
        load_view(sview, bt->views[k]);
        __syncthreads();
        const SolverView& v = sview;
        const double* row = v.Y + (size_t)(stg & 1) * 2 * v.L;
        // (batch slots have no log-R mode: dmfe_batch_add refuses it)
        if (PREC == DMFE_FP64) hi_f64_body<SW, false>(v, row, 0.0, stg, v.S, lb, le);
        else hi_f32_body<SW>(v, row, 0.0, stg, v.S, lb, le);
    });
}

size_t hi_smem_bytes(const SolverView& v) {
    if (v.precision == DMFE_FP64)
        return (size_t)v.L * sizeof(dbl4) + (size_t)(v.cap + 1) * 2 * sizeof(double) + (size_t)v.L * sizeof(int);
    return (size_t)v.L * sizeof(float4) + (size_t)(v.cap + 1) * 3 * sizeof(float) + (size_t)v.L * sizeof(int);
}

template <int SW>
void* hi_kernel(int precision, bool log_r) {
    if (precision != DMFE_FP64) return (void*)k_hi_f32<SW>;
    return log_r ? (void*)k_hi_f64<SW, true> : (void*)k_hi_f64<SW, false>;
}

void* hi_kernel_for(const SolverView& v) {
    const bool lr = v.log_r != 0;
    switch (v.s) {
        case 4: return hi_kernel<4>(v.precision, lr);
        case 6: return hi_kernel<6>(v.precision, lr);
        case 8: return hi_kernel<8>(v.precision, lr);
        case 10: return hi_kernel<10>(v.precision, lr);
    }
    return nullptr;
}

}  // namespace

// Block size and grid of a single solve's history-integral launch: enough warps per CTA
// that the units of one stage cover every SM once (at least 4 and at most 16 warps), and
// at most the CTAs that can be resident (the kernel is persistent over its unit blocks).
int hi_launch_shape(long long units, int nsm, int max_warps, int* warps) {
    long long w = (units + nsm - 1) / nsm;
    w = w < 4 ? 4 : (w > max_warps ? max_warps : w);
    *warps = (int)w;
    return (int)((units + w - 1) / w);
}

int hi_config(SolverView& v, int* grid_ctas, size_t* smem) {
    if (v.precision == DMFE_DOUBLE_FLOAT) return hi_config_df(v, grid_ctas, smem);
    void* fn = hi_kernel_for(v);
    if (!fn) return DMFE_ERR_UNSUPPORTED;
    size_t sm = hi_smem_bytes(v);
    int dev = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    int max_optin = 0, nsm = 0;
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (sm > (size_t)max_optin) return DMFE_ERR_UNSUPPORTED;
    DMFE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int warps = 0;
    const bool flat = v.hi_chunk == kFlatSplit;
    const int want = flat ? 0 : hi_launch_shape((long long)hi_parts(v.L, v.hi_chunk) * v.L, nsm, HI_WARPS, &warps);
    if (flat) warps = HI_WARPS;
    int per_sm = 0;
    DMFE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, sm));
    if (per_sm < 1) return DMFE_ERR_UNSUPPORTED;
    const int cap = nsm * per_sm;
    // the flat split: every resident warp slot takes one equal segment of the pairs
    *grid_ctas = flat ? cap : (want < cap ? want : cap);
    if (flat && !flat_split_fits(v.L, (long long)cap * warps)) return DMFE_ERR_UNSUPPORTED;
    v.hi_threads = warps * 32;
    *smem = sm;
    return DMFE_OK;
}

int launch_history_integrals(const SolverView& v, const double* row_dev, double t, int stage,
                             double* S_dev, int grid_ctas, cudaStream_t s) {
    if (v.precision == DMFE_DOUBLE_FLOAT)
        return launch_history_integrals_df(v, row_dev, t, stage, S_dev, grid_ctas, s);
    void* fn = hi_kernel_for(v);
    if (!fn) return DMFE_ERR_UNSUPPORTED;
    int rc = launch_stage_prep(v, row_dev, t, stage, s);
    if (rc) return rc;
    size_t sm = hi_smem_bytes(v);
    int fs = stage;
    void* args[] = {(void*)&v, (void*)&row_dev, (void*)&t, (void*)&fs, (void*)&S_dev};
    DMFE_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid_ctas), dim3(v.hi_threads > 0 ? v.hi_threads : HI_THREADS), args,
                                   sm, s));
    return DMFE_OK;
}

// ---- batched launchers
int batch_hi_config(int precision, int sw, int max_L, int max_cap, int* grid_ctas, size_t* smem) {
    if (precision == DMFE_DOUBLE_FLOAT) return batch_hi_config_df(sw, max_L, max_cap, grid_ctas, smem);
    SolverView v{};
    v.L = max_L;
    v.cap = max_cap;
    v.precision = precision;
    v.s = sw;
    const size_t sm = hi_smem_bytes(v);
    void* fn = nullptr;
    switch (sw) {
        case 4: fn = precision == DMFE_FP64 ? (void*)k_batch_hi<4, DMFE_FP64> : (void*)k_batch_hi<4, DMFE_FP32_COMPENSATED>; break;
        case 6: fn = precision == DMFE_FP64 ? (void*)k_batch_hi<6, DMFE_FP64> : (void*)k_batch_hi<6, DMFE_FP32_COMPENSATED>; break;
        case 8: fn = precision == DMFE_FP64 ? (void*)k_batch_hi<8, DMFE_FP64> : (void*)k_batch_hi<8, DMFE_FP32_COMPENSATED>; break;
        case 10: fn = precision == DMFE_FP64 ? (void*)k_batch_hi<10, DMFE_FP64> : (void*)k_batch_hi<10, DMFE_FP32_COMPENSATED>; break;
        default: return DMFE_ERR_UNSUPPORTED;
    }
    int dev = 0, max_optin = 0, nsm = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (sm > (size_t)max_optin) return DMFE_ERR_UNSUPPORTED;
    DMFE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    DMFE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BATCH_THREADS, sm));
    if (per_sm < 1) return DMFE_ERR_UNSUPPORTED;
    *grid_ctas = nsm * per_sm;
    *smem = sm;
    return DMFE_OK;
}

int launch_batch_hi(const BatchTable* bt, int precision, int sw, int stg, int grid, size_t smem, cudaStream_t s) {
    if (precision == DMFE_DOUBLE_FLOAT) return launch_batch_hi_df(bt, sw, stg, grid, smem, s);
    const bool f64 = precision == DMFE_FP64;
    switch (sw) {
        case 4: if (f64) k_batch_hi<4, DMFE_FP64><<<grid, BATCH_THREADS, smem, s>>>(bt, stg);
                else k_batch_hi<4, DMFE_FP32_COMPENSATED><<<grid, BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 6: if (f64) k_batch_hi<6, DMFE_FP64><<<grid, BATCH_THREADS, smem, s>>>(bt, stg);
                else k_batch_hi<6, DMFE_FP32_COMPENSATED><<<grid, BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 8: if (f64) k_batch_hi<8, DMFE_FP64><<<grid, BATCH_THREADS, smem, s>>>(bt, stg);
                else k_batch_hi<8, DMFE_FP32_COMPENSATED><<<grid, BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 10: if (f64) k_batch_hi<10, DMFE_FP64><<<grid, BATCH_THREADS, smem, s>>>(bt, stg);
                 else k_batch_hi<10, DMFE_FP32_COMPENSATED><<<grid, BATCH_THREADS, smem, s>>>(bt, stg); break;
        default: return DMFE_ERR_UNSUPPORTED;
    }
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}
