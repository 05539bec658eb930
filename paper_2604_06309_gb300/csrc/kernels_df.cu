// History integrals in double-float arithmetic (Secs. 3.3, 3.4, Eq. int).
//
// Same quantities, mapping and reduction order as kernels_hi.cu (units of (j, chunk of
// the i-range), lanes stride over i, fixed butterflies), but every interpolation, product and
// sum runs in double-float (df64.h): FP64-class accuracy (~1e-13 relative) on the FP32
// pipes, which on this part issue 64 times the FP64 rate. Inputs are a double-float
// replica of the history and double-float stencil positions.
//
// k_stage_prep does the per-stage FP64 work once, spread over many SMs: the table
// cell -> slice of time theta_m t, the B1 time weights of every output index, and for
// this path the stage row {K = f''(C) R, D = f'(C), C, R} and the per-slice
// complements v_k = (t - t_k)/t with their reciprocal widths.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dmfe_internal.h"
#include "hi_units.h"

namespace {

constexpr int DF_THREADS = 512;
constexpr int DF_WARPS = DF_THREADS / 32;

__device__ __forceinline__ int find_slice_g(const double* ht, int n, double tau) {
    if (n <= 2) return 0;
    int lo = 0, hi = n - 2;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ht[mid] <= tau) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-stage preparation (all precisions): the cell -> slice table, the B1 time weights of
// every output index, and for the double-float path the stage row and slice constants.
__device__ __forceinline__ void stage_prep_body(const SolverView& v, const double* __restrict__ row, double t_arg,
                                                int from_state) {
    const DevState* st = v.st;
    if (stage_off(st, from_state)) return;
    const int L = v.L, n = st->n, act = st->active;
    const double t = from_state ? st->t_stage : t_arg;
    const double* ht = v.ht[act];
    const double tl = ht[n - 1];
    const bool ext = t > tl;
    const double hx = t - tl;
    const int tot = L > n + 1 ? L : n + 1;
    __shared__ double red_m[kPrepThreads], red_e[kPrepThreads];
    double pm = 0.0, pe = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += gridDim.x * blockDim.x) {
        if (q < L) {
            // integrands of mu and E on the stage row (Sec. 2.1), summed per block below
            const double Cq = row[q], Rq = row[L + q];
            const double Dq = fp1(v.poly, Cq);
            pm += v.nu[q] * (fp2(v.poly, Cq) * Rq * Cq + Dq * Rq);
            pe += v.nu[q] * (Dq * Rq);
            // the stage row as the FP64 and FP32 kernels read it (once per stage here instead
            // of once per CTA there; the same operations)
            if (v.row64) v.row64[q] = dbl4{fp2(v.poly, Cq) * Rq, Dq, Cq, Rq};
            if (v.row32f) v.row32f[q] = make_float4((float)(fp2(v.poly, Cq) * Rq), (float)Dq, (float)Cq, (float)Rq);
            const double tau = v.theta[q] * t;
            const int c = find_slice_g(ht, n, tau);
            v.cell[q] = c;
            B1Desc d;
            d.s = 0.0;
            if (ext && tau > tl) {
                const double s = tau - tl, qq = s / hx;
                d.a0 = n - 1; d.a1 = -1;
                d.s = qq;
                d.w[0] = 1.0 - qq * qq; d.w[1] = s - s * qq; d.w[2] = qq * qq; d.w[3] = 0.0;
            } else if (n == 1) {
                d.a0 = 0; d.a1 = 0;
                d.w[0] = 1.0; d.w[1] = 0.0; d.w[2] = 0.0; d.w[3] = 0.0;
            } else {
                const double hh = ht[c + 1] - ht[c];
                const double sg = (tau - ht[c]) / hh, om = 1.0 - sg;
                d.a0 = c; d.a1 = c + 1;
                d.s = sg;
                d.w[0] = (1.0 + 2.0 * sg) * om * om;
                d.w[1] = sg * om * om * hh;
                d.w[2] = sg * sg * (3.0 - 2.0 * sg);
                d.w[3] = sg * sg * (sg - 1.0) * hh;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) d.wd[k] = df_from_d(d.w[k]);
            v.b1[q] = d;
            if (v.vrow32 && ext) {
                // FP32 path: the extension as a virtual slice, as for double-float below
                const dbl4 e = v.hist[act][(size_t)(n - 1) * L + q];
                v.vrow32[q] = make_float4((float)Cq, (float)(2.0 * (Cq - e.x) / hx - e.y), (float)Rq,
                                          (float)(2.0 * (Rq - e.z) / hx - e.w));
            }
            if (v.hcoef[act] && ext) {
                // FP64 path: the quadratic extension through the last slice and this stage
                // row as a virtual interval n-1 = [t_last, t] in monomial form (c3 = 0)
                const dbl4 e = v.hist[act][(size_t)(n - 1) * L + q];
                dbl8 c;
                c.c0 = e.x; c.c1 = hx * e.y; c.c2 = Cq - e.x - hx * e.y; c.c3 = 0.0;
                c.r0 = e.z; c.r1 = hx * e.w; c.r2 = Rq - e.z - hx * e.w; c.r3 = 0.0;
                v.hcoef[act][(size_t)(n - 1) * L + q] = c;
                if (v.lcoef[act]) {
                    // log-R mode: the quadratic in log R through (log R_last, R'_last/R_last)
                    // and log of the stage row, where both are positive
                    dbl4 l{nan(""), 0.0, 0.0, 0.0};
                    if (e.z > 0.0 && Rq > 0.0) {
                        const double l0 = log(e.z), l1 = hx * e.w / e.z;
                        l = dbl4{l0, l1, log(Rq) - l0 - l1, 0.0};
                    }
                    v.lcoef[act][(size_t)(n - 1) * L + q] = l;
                }
            }
            if (v.rowdf) {
                const double C = row[q], R = row[L + q];
                v.rowdf[q] = dfrow{df_from_d(fp2(v.poly, C) * R), df_from_d(fp1(v.poly, C)), df_from_d(C), df_from_d(R)};
                if (ext) {
                    // double-float path: the quadratic extension through the last slice and
                    // this stage row equals the cubic Hermite interpolant to a virtual slice
                    // (t, Y, 2 (Y - y_last) / hx - y'_last); the kernel reads it as slice n
                    const dbl4 e = v.hist[act][(size_t)(n - 1) * L + q];
                    const double dCv = 2.0 * (C - e.x) / hx - e.y, dRv = 2.0 * (R - e.z) / hx - e.w;
                    v.vrowdf[q] = df8{df_from_d(C), df_from_d(dCv), df_from_d(R), df_from_d(dRv)};
                }
            }
        }
        if (q < n && v.slice64) v.slice64[q] = q + 1 < n ? 1.0 / (ht[q + 1] - ht[q]) : (ext ? 1.0 / hx : 0.0);
        if (v.slice32 && q < (ext ? n + 1 : n)) {
            // FP32 path: slice q (q = n: the stage time itself, the virtual slice of an
            // extension) as complements, reciprocal widths and widths
            const int nsl = ext ? n + 1 : n;
            const double tk = q < n ? ht[q] : t;
            float4 e = make_float4((float)((t - tk) / t), 0.f, 0.f, 0.f);
            if (q + 1 < nsl) {
                const double tk1 = q + 1 < n ? ht[q + 1] : t;
                e.y = (float)(t / (tk1 - tk));
                e.z = (float)(tk1 - tk);
            }
            v.slice32[q] = e;
        }
        if (q <= n && v.slicedf) {
            // slice q (q = n: the stage time itself, the virtual slice of an extension)
            const double tk = q < n ? ht[q] : t;
            const double tn = q + 1 < n ? ht[q + 1] : t;
            dfslice e;
            e.v = df_from_d((t - tk) / t);
            if (q + 1 < n || (q + 1 == n && ext)) {
                const double w = tn - tk;
                e.inv = df_from_d(t / w);
                e.h = (float)w;
            } else {
                e.inv = df{0.f, 0.f};
                e.h = 0.f;
            }
            e.pad = 0.f;
            v.slicedf[q] = e;
        }
    }
    // deterministic block reduction: each block owns one fixed range of q
    red_m[threadIdx.x] = pm;
    red_e[threadIdx.x] = pe;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red_m[threadIdx.x] += red_m[threadIdx.x + w];
            red_e[threadIdx.x] += red_e[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        v.mupart[blockIdx.x] = red_m[0];
        v.mupart[kMaxPrepBlocks + blockIdx.x] = red_e[0];
    }
}

// Lagrange weights on nodes 0..SW-1 at the double-float position u, 0 <= u <= SW - 1 (the
// stencil base is clamped so that the position lies on the stencil). The differences u - m
// are formed exactly as pairs (df_add_exact_const: m >= u.hi, or u.hi > m >= 1 with an
// exactly representable difference).
template <int SW>
__device__ __forceinline__ void lagrange_df(df u, df (&w)[SW]);

// Width 4: w0 = -(u-1)(u-2)(u-3)/6, w1 = u(u-2)(u-3)/2, w2 = -u(u-1)(u-3)/2,
// w3 = u(u-1)(u-2)/6, with the shared products u(u-1) and (u-2)(u-3).
template <>
__device__ __forceinline__ void lagrange_df<4>(df u, df (&w)[4]) {
    const df u1 = df_add_exact_const(u, -1.f), u2 = df_add_exact_const(u, -2.f), u3 = df_add_exact_const(u, -3.f);
    const df ab = df_mul_raw(u, u1), cd = df_mul_raw(u2, u3);
    const df sixth = df{0.16666667163372040f, -4.9670538e-09f};  // 1/6 as a double-float
    w[0] = df_neg(df_mul_raw(df_mul_raw(u1, cd), sixth));
    const df h1 = df_mul_raw(u, cd);
    w[1] = df{h1.hi * 0.5f, h1.lo * 0.5f};
    const df h2 = df_mul_raw(ab, u3);
    w[2] = df{h2.hi * -0.5f, h2.lo * -0.5f};
    w[3] = df_mul_raw(df_mul_raw(ab, u2), sixth);
}

template <int SW>
__device__ __forceinline__ void lagrange_df(df u, df (&w)[SW]) {
    df um[SW];
#pragma unroll
    for (int k = 0; k < SW; ++k) um[k] = df_add_exact_const(u, -(float)k);
    df pre[SW], suf[SW];
    pre[0] = df{1.f, 0.f};
#pragma unroll
    for (int k = 1; k < SW; ++k) pre[k] = df_mul_raw(pre[k - 1], um[k - 1]);
    suf[SW - 1] = df{1.f, 0.f};
#pragma unroll
    for (int k = SW - 2; k >= 0; --k) suf[k] = df_mul_raw(suf[k + 1], um[k + 1]);
#pragma unroll
    for (int k = 0; k < SW; ++k) {
        // 1 / prod_{m != k} (k - m) as a double-float constant
        double c = 1.0;
#pragma unroll
        for (int m = 0; m < SW; ++m)
            if (m != k) c /= (double)(k - m);
        const float ch = (float)c;
        const float cl = (float)(c - (double)ch);
        w[k] = df_mul_raw(df_mul_raw(pre[k], suf[k]), df{ch, cl});
    }
}

// floor(x) for 0 <= x < 2^23, as a float: adding 2^23 rounded down keeps the integer part
// (the float spacing there is 1). Integer <-> float conversions are avoided on this path:
// GB300 issues them on its FP64 unit.
__device__ __forceinline__ float floor_nonneg(float x) { return __fsub_rn(__fadd_rd(x, 8388608.f), 8388608.f); }
// an integer-valued float 0 <= f < 2^23 as an int (its bit pattern above 2^23)
__device__ __forceinline__ int int_of(float f) { return __float_as_int(__fadd_rn(f, 8388608.f)) - 0x4B000000; }

// Stencil position x (double-float, 0 <= x <= L - 1) -> base b = clamp(floor(x.hi) - SW/2 + 1,
// 0, L - SW) and the weights; *fl receives floor(x.hi). bmax = L - SW as a float.
template <int SW>
__device__ __forceinline__ int stencil_df(df x, float bmax, df (&w)[SW], float* fl = nullptr) {
    const float f = floor_nonneg(x.hi);
    if (fl) *fl = f;
    const float bf = fminf(fmaxf(__fsub_rn(f, (float)(SW / 2 - 1)), 0.f), bmax);
    // x.hi - b is exact (b is an integer within a few units of x.hi)
    const df u = fast_two_sum(__fsub_rn(x.hi, bf), x.lo);
    lagrange_df<SW>(u, w);
    return int_of(bf);
}

// f'(q) and f''(q) in double-float at two points in one loop: the same Horner steps, in
// the same order, as evaluating each polynomial alone (f'' has degree deg1 - 1, so f' takes
// one step more, peeled in front), with a quarter of the loop overhead and loads.
__device__ __forceinline__ void poly12_df_pair(const Poly& P, df qa, df qb, df& f1a, df& f2a, df& f1b, df& f2b) {
    const int d1 = P.deg1;
    f1a = f1b = df{P.f1[d1], P.g1[d1]};
    if (d1 == 0) {
        f2a = f2b = df{P.f2[0], P.g2[0]};
        return;
    }
    f2a = f2b = df{P.f2[d1 - 1], P.g2[d1 - 1]};
    const df c = df{P.f1[d1 - 1], P.g1[d1 - 1]};
    f1a = df_fma(f1a, qa, c);
    f1b = df_fma(f1b, qb, c);
    for (int m = d1 - 2; m >= 0; --m) {
        const df c1 = df{P.f1[m], P.g1[m]}, c2 = df{P.f2[m], P.g2[m]};
        f1a = df_fma(f1a, qa, c1);
        f2a = df_fma(f2a, qa, c2);
        f1b = df_fma(f1b, qb, c1);
        f2b = df_fma(f2b, qb, c2);
    }
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int SW>
__device__ __forceinline__ void hi_df_body(const SolverView& v, double t_arg, int from_state, double* __restrict__ S,
                                           int ub, int ue) {
    extern __shared__ __align__(32) unsigned char smraw[];
    const DevState* st = v.st;
    if (stage_off(st, from_state)) return;
    const int L = v.L, n = st->n, act = st->active;
    const double t = from_state ? st->t_stage : t_arg;
    const df8* __restrict__ H = v.histdf[act];
    const double* __restrict__ ht = v.ht[act];
    const double tl = ht[n - 1];
    const bool ext = t > tl;
    // slices, and for a stage beyond the last slice the virtual slice n at the stage time
    // (the prep kernel's quadratic extension in Hermite form): all pairs take one path
    const int nsl = ext ? n + 1 : n;
    const int kmax = nsl - 2;
    dfrow* srow = reinterpret_cast<dfrow*>(smraw);                   // [L]
    df* sv = reinterpret_cast<df*>(srow + L);                         // [cap + 1] v_k
    df* sinv = sv + v.cap + 1;                                        // [cap + 1] t/(t_{k+1} - t_k)
    float* sh = reinterpret_cast<float*>(sinv + v.cap + 1);           // [cap + 1] t_{k+1} - t_k
    uint16_t* scell = reinterpret_cast<uint16_t*>(sh + v.cap + 1);    // [L]
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        srow[i] = v.rowdf[i];
        scell[i] = (uint16_t)v.cell[i];
    }
    for (int i = threadIdx.x; i < nsl; i += blockDim.x) {
        const dfslice e = v.slicedf[i];
        sv[i] = e.v;
        sinv[i] = e.inv;
        sh[i] = e.h;
    }
    __syncthreads();
    const df8* __restrict__ VR = v.vrowdf;
    const df hx_df = df_from_d(t - tl);
    const int lane = threadIdx.x & 31;
    const df* __restrict__ omdf = v.omega_df;
    const df* __restrict__ nudf = v.nu_df;
    const float bmax = (float)(L - SW);

    const int chunk = v.hi_chunk;
    hi_for_items(L, chunk, ub, ue, v.flat_seg, v.flat_row, [&](int j, int i0, int i1, int part, int nparts) {
        // ---- per unit: B1 time weights prepared once per stage
        const df omj = omdf[j];
        int a0, a1;
        df bw0, bw1, bw2, bw3;
        {
            const B1Desc d = v.b1[j];
            a0 = d.a0; a1 = d.a1;
            if (!DMFE_IN_BOUNDS(v.st, a0 >= 0 && a0 < n && a1 < n, 21)) { a0 = 0; a1 = -1; }
            bw0 = d.wd[0]; bw1 = d.wd[1]; bw2 = d.wd[2]; bw3 = d.wd[3];
        }
        // double-float positions (8 B per pair and stencil); the weights are formed here:
        // a third of the table traffic and a fifth of the footprint of stored weights,
        // which matters for batches of many solves (measured: 12 % faster batched)
        const df* __restrict__ q1r = v.q1 + (size_t)j * L;
        const df* __restrict__ q2r = v.q2 + (size_t)j * L;
        const df* __restrict__ q3r = v.q3 + (size_t)j * L;
        dacc acc[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) acc[r] = dacc{0.f, 0.f};
        df c_at_0 = df{0.f, 0.f};
        // software pipeline: the three positions, omega_i and nu_i of the next index are
        // loaded before this index's arithmetic
        int i = i0 + lane;
        df n1{0.f, 0.f}, n2{0.f, 0.f}, n3{0.f, 0.f}, nom{0.f, 0.f}, nnu{0.f, 0.f};
        if (i < i1) { n1 = q1r[i]; n2 = q2r[i]; n3 = q3r[i]; nom = omdf[i]; nnu = nudf[i]; }
        for (; i < i1; i += 32) {
            const df x1 = n1, x2 = n2, x3 = n3, omi = nom, nui = nnu;
            if (i + 32 < i1) {
                const int in = i + 32;
                n1 = q1r[in]; n2 = q2r[in]; n3 = q3r[in]; nom = omdf[in]; nnu = nudf[in];
            }
            // ---- B1: on-grid column i at time theta_j t
            df CB1, RB1;
            {
                const df8 h0 = H[(size_t)a0 * L + i];
                dacc c = dacc_prod(bw0, h0.C), r = dacc_prod(bw0, h0.R);
                dacc_add(c, bw1, h0.dC);
                dacc_add(r, bw1, h0.dR);
                if (a1 >= 0) {
                    const df8 h1 = H[(size_t)a1 * L + i];
                    dacc_add(c, bw2, h1.C);
                    dacc_add(c, bw3, h1.dC);
                    dacc_add(r, bw2, h1.R);
                    dacc_add(r, bw3, h1.dR);
                } else {
                    const dfrow r1 = srow[i];
                    dacc_add(c, bw2, r1.C);
                    dacc_add(r, bw2, r1.R);
                }
                CB1 = dacc_raw(c);
                RB1 = dacc_raw(r);
            }
            // ---- A1: current row at phi1
            df KA1, DA1, CA1, RA1;
            {
                df w[SW];
                int b = stencil_df<SW>(x1, bmax, w);
                if (!DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 22)) b = 0;
                const dfrow q0 = srow[b];
                dacc k = dacc_prod(w[0], q0.K), d = dacc_prod(w[0], q0.D);
                dacc c = dacc_prod(w[0], q0.C), r = dacc_prod(w[0], q0.R);
#pragma unroll
                for (int m = 1; m < SW; ++m) {
                    const dfrow q = srow[b + m];
                    dacc_add(k, w[m], q.K);
                    dacc_add(d, w[m], q.D);
                    dacc_add(c, w[m], q.C);
                    dacc_add(r, w[m], q.R);
                }
                KA1 = dacc_raw(k); DA1 = dacc_raw(d); CA1 = dacc_raw(c); RA1 = dacc_raw(r);
            }
            // ---- A2: current row at phi2
            df KA2, RA2;
            float fl2;  // floor of the phi2 position: its grid cell
            {
                df w[SW];
                int b = stencil_df<SW>(x2, bmax, w, &fl2);
                if (!DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW, 23)) b = 0;
                const dfrow q0 = srow[b];
                dacc k = dacc_prod(w[0], q0.K), r = dacc_prod(w[0], q0.R);
#pragma unroll
                for (int m = 1; m < SW; ++m) {
                    const dfrow q = srow[b + m];
                    dacc_add(k, w[m], q.K);
                    dacc_add(r, w[m], q.R);
                }
                KA2 = dacc_raw(k); RA2 = dacc_raw(r);
            }
            // ---- B2: theta position psi on the slices around phi2 t (complement form)
            df CB2, RB2;
            {
                const df u = df_mul(omj, omi);  // 1 - phi2 = omega_j omega_i
                int s0, s1;
                df tw0, tw1, tw2, tw3;
                if (kmax < 0) {
                    // a single stored slice and the stage at its time
                    s0 = 0; s1 = -1;
                    tw0 = df{1.f, 0.f}; tw1 = df{0.f, 0.f}; tw2 = df{0.f, 0.f}; tw3 = df{0.f, 0.f};
                } else {
                    const int c2 = int_of(fl2);
                    int k = scell[c2 < L ? c2 : L - 1];
                    while (k < kmax && df_ge(sv[k + 1], u)) ++k;
                    while (k > 0 && df_lt(sv[k], u)) --k;
                    const df sg = df_mul_raw(df_sub(sv[k], u), sinv[k]);
                    // 1 - sg, 3 - 2 sg and 1 - h01 exactly as pairs: 0 <= sg <= 1 up to
                    // rounding, so each constant dominates (or Sterbenz applies)
                    const df om = df_add_exact_const(df_neg(sg), 1.f);
                    const df om2 = df_mul_raw(om, om), sg2 = df_mul_raw(sg, sg);
                    s0 = k; s1 = k + 1;
                    // h01 = sg^2 (3 - 2 sg) and h00 = 1 - h01 (the value weights sum to one);
                    // the doubling of sg is exact
                    tw2 = df_mul_raw(sg2, df_add_exact_const(df{-2.f * sg.hi, -2.f * sg.lo}, 3.f));
                    tw0 = df_add_exact_const(df_neg(tw2), 1.f);
                    // sg^2 (sg - 1) = -(sg^2 (1 - sg))
                    const df a1 = df_mul_raw(sg, om2), a3 = df_neg(df_mul_raw(sg2, om));
                    if (k < n - 1) {
                        // a stored interval: its width in FP32 (the derivative terms are
                        // O(h) corrections)
                        tw1 = df_mul_f_raw(a1, sh[k]);
                        tw3 = df_mul_f_raw(a3, sh[k]);
                    } else {
                        // the virtual interval: the width in full double-float, since the
                        // virtual slice's derivative need not be small
                        tw1 = df_mul_raw(a1, hx_df);
                        tw3 = df_mul_raw(a3, hx_df);
                    }
                }
                df w[SW];
                int b = stencil_df<SW>(x3, bmax, w);
                if (!DMFE_IN_BOUNDS(v.st, b >= 0 && b <= L - SW && s0 >= 0 && s0 < n && s1 < nsl, 24)) {
                    b = 0; s0 = 0; s1 = -1;
                }
                const df8* __restrict__ p0 = H + (size_t)s0 * L + b;
                df c0, dc0, r0, dr0;
                {
                    const df8 e0 = p0[0];
                    dacc ac = dacc_prod(w[0], e0.C), adc = dacc_prod(w[0], e0.dC);
                    dacc ar = dacc_prod(w[0], e0.R), adr = dacc_prod(w[0], e0.dR);
#pragma unroll
                    for (int m = 1; m < SW; ++m) {
                        const df8 e = p0[m];
                        dacc_add(ac, w[m], e.C);
                        dacc_add(adc, w[m], e.dC);
                        dacc_add(ar, w[m], e.R);
                        dacc_add(adr, w[m], e.dR);
                    }
                    c0 = dacc_raw(ac); dc0 = dacc_raw(adc); r0 = dacc_raw(ar); dr0 = dacc_raw(adr);
                }
                dacc tc = dacc_prod(tw0, c0), tr = dacc_prod(tw0, r0);
                dacc_add(tc, tw1, dc0);
                dacc_add(tr, tw1, dr0);
                if (s1 >= 0) {
                    const df8* __restrict__ p1 = (s1 < n ? H + (size_t)s1 * L : VR) + b;
                    const df8 e0 = p1[0];
                    dacc ac = dacc_prod(w[0], e0.C), adc = dacc_prod(w[0], e0.dC);
                    dacc ar = dacc_prod(w[0], e0.R), adr = dacc_prod(w[0], e0.dR);
#pragma unroll
                    for (int m = 1; m < SW; ++m) {
                        const df8 e = p1[m];
                        dacc_add(ac, w[m], e.C);
                        dacc_add(adc, w[m], e.dC);
                        dacc_add(ar, w[m], e.R);
                        dacc_add(adr, w[m], e.dR);
                    }
                    dacc_add(tc, tw2, dacc_raw(ac));
                    dacc_add(tc, tw3, dacc_raw(adc));
                    dacc_add(tr, tw2, dacc_raw(ar));
                    dacc_add(tr, tw3, dacc_raw(adr));
                }
                CB2 = dacc_raw(tc);
                RB2 = dacc_raw(tr);
            }
            df f1a, f2a, f1b, f2b;
            poly12_df_pair(v.poly, CB1, CB2, f1a, f2a, f1b, f2b);
            const df nRB1 = df_mul_raw(nui, RB1);
            const df nRA2 = df_mul_raw(nui, RA2);
            const df nKA2 = df_mul_raw(nui, KA2);
            dacc_add(acc[0], df_mul_raw(nui, KA1), CB1);
            dacc_add(acc[1], nKA2, CB2);
            dacc_add(acc[2], DA1, nRB1);
            dacc_add(acc[3], nKA2, RB2);
            dacc_add(acc[4], df_mul_raw(f2a, CA1), nRB1);
            dacc_add(acc[5], df_mul_raw(nui, f1a), RA1);
            dacc_add(acc[6], f1b, nRA2);
            dacc_add(acc[7], df_mul_raw(f2b, RB2), nRA2);
            dacc_add(acc[8], df_fma(f2a, CB1, f1a), nRB1);
            if (i == 0) c_at_0 = CB1;
        }
        double sums[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const df x = df_warp_sum(dacc_get(acc[r]));
            sums[r] = lane == 0 ? df_to_d(x) : 0.0;
        }
        if (lane == 0) hi_finish_part(sums, df_to_d(c_at_0), j, part, nparts, L, v.Spart, v.jcount, S);
    });
}

__global__ void k_stage_prep(SolverView v, const double* __restrict__ row, double t_arg, int from_state) {
    stage_prep_body(v, row, t_arg, from_state);
}

template <int SW>
__global__ void __launch_bounds__(DF_THREADS, 1) k_hi_df(SolverView v, double t_arg, int from_state,
                                                         double* __restrict__ S) {
    int ub, ue;
    hi_unit_block(v.L, v.hi_chunk, &ub, &ue);
    hi_df_body<SW>(v, t_arg, from_state, S, ub, ue);
}

// Batched versions (see kernels_hi.cu): prep over (element block, slot), integrals over
// the concatenated unit space of the batch table.
__global__ void k_batch_prep(const BatchTable* __restrict__ bt, int stg) {
    const int k = blockIdx.y;
    if (k >= bt->count || !bt->active[k]) return;
    const SolverView& v = bt->views[k];
    stage_prep_body(v, v.Y + (size_t)(stg & 1) * 2 * v.L, 0.0, stg);
}

// 384-thread CTAs, as for the other batched kernels (with 512 threads the slot loop's live
// state made this kernel spill 148 bytes a thread)
constexpr int DF_BATCH_THREADS = 384;

template <int SW>
__global__ void __launch_bounds__(DF_BATCH_THREADS, 1) k_batch_hi_df(const BatchTable* __restrict__ bt, int stg) {
    __shared__ __align__(16) SolverView sview;
    batch_for_my_units(bt, stg, [&](int k, int lb, int le) {
        __syncthreads();  // the previous slot's shared-memory data are no longer read
        load_view(sview, bt->views[k]);
        __syncthreads();
        hi_df_body<SW>(sview, 0.0, stg, sview.S, lb, le);
    });
}

size_t df_smem_bytes(const SolverView& v) {
    return (size_t)v.L * sizeof(dfrow) + (size_t)(v.cap + 1) * (2 * sizeof(df) + sizeof(float)) +
           (size_t)v.L * sizeof(uint16_t) + 16;
}

void* df_kernel_for(int s) {
    switch (s) {
        case 4: return (void*)k_hi_df<4>;
        case 6: return (void*)k_hi_df<6>;
        case 8: return (void*)k_hi_df<8>;
        case 10: return (void*)k_hi_df<10>;
    }
    return nullptr;
}

}  // namespace

int launch_stage_prep(const SolverView& v, const double* row_dev, double t, int stage, cudaStream_t s) {
    const int tot = v.L > v.cap ? v.L : v.cap;
    k_stage_prep<<<(tot + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, s>>>(v, row_dev, t, stage);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int hi_config_df(SolverView& v, int* grid_ctas, size_t* smem) {
    void* fn = df_kernel_for(v.s);
    if (!fn) return DMFE_ERR_UNSUPPORTED;
    if (v.L > 65535) return DMFE_ERR_UNSUPPORTED;
    const size_t sm = df_smem_bytes(v);
    int dev = 0, max_optin = 0, nsm = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (sm > (size_t)max_optin) return DMFE_ERR_UNSUPPORTED;
    DMFE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int warps = 0;
    const bool flat = v.hi_chunk == kFlatSplit;
    const int want = flat ? 0 : hi_launch_shape((long long)hi_parts(v.L, v.hi_chunk) * v.L, nsm, DF_WARPS, &warps);
    if (flat) warps = DF_WARPS;
    int per_sm = 0;
    DMFE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, sm));
    if (per_sm < 1) return DMFE_ERR_UNSUPPORTED;
    const int cap = nsm * per_sm;
    *grid_ctas = flat ? cap : (want < cap ? want : cap);
    if (flat && !flat_split_fits(v.L, (long long)cap * warps)) return DMFE_ERR_UNSUPPORTED;
    v.hi_threads = warps * 32;
    *smem = sm;
    return DMFE_OK;
}

int launch_history_integrals_df(const SolverView& v, const double* row_dev, double t, int stage,
                                double* S_dev, int grid_ctas, cudaStream_t s) {
    void* fn = df_kernel_for(v.s);
    if (!fn) return DMFE_ERR_UNSUPPORTED;
    const int fs = stage;
    int rc = launch_stage_prep(v, row_dev, t, stage, s);
    if (rc) return rc;
    const size_t sm = df_smem_bytes(v);
    void* args[] = {(void*)&v, (void*)&t, (void*)&fs, (void*)&S_dev};
    DMFE_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid_ctas), dim3(v.hi_threads > 0 ? v.hi_threads : DF_THREADS), args,
                                   sm, s));
    return DMFE_OK;
}

int batch_hi_config_df(int sw, int max_L, int max_cap, int* grid_ctas, size_t* smem) {
    SolverView v{};
    v.L = max_L;
    v.cap = max_cap;
    v.s = sw;
    void* fn = nullptr;
    switch (sw) {
        case 4: fn = (void*)k_batch_hi_df<4>; break;
        case 6: fn = (void*)k_batch_hi_df<6>; break;
        case 8: fn = (void*)k_batch_hi_df<8>; break;
        case 10: fn = (void*)k_batch_hi_df<10>; break;
        default: return DMFE_ERR_UNSUPPORTED;
    }
    if (max_L > 65535) return DMFE_ERR_UNSUPPORTED;
    const size_t sm = df_smem_bytes(v);
    int dev = 0, max_optin = 0, nsm = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (sm > (size_t)max_optin) return DMFE_ERR_UNSUPPORTED;
    DMFE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    DMFE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, DF_BATCH_THREADS, sm));
    if (per_sm < 1) return DMFE_ERR_UNSUPPORTED;
    *grid_ctas = nsm * per_sm;
    *smem = sm;
    return DMFE_OK;
}

int launch_batch_hi_df(const BatchTable* bt, int sw, int stg, int grid, size_t smem, cudaStream_t s) {
    switch (sw) {
        case 4: k_batch_hi_df<4><<<grid, DF_BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 6: k_batch_hi_df<6><<<grid, DF_BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 8: k_batch_hi_df<8><<<grid, DF_BATCH_THREADS, smem, s>>>(bt, stg); break;
        case 10: k_batch_hi_df<10><<<grid, DF_BATCH_THREADS, smem, s>>>(bt, stg); break;
        default: return DMFE_ERR_UNSUPPORTED;
    }
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_batch_prep(const BatchTable* bt, int stg, int max_tot, int slots, cudaStream_t s) {
    k_batch_prep<<<dim3((max_tot + kPrepThreads - 1) / kPrepThreads, slots), kPrepThreads, 0, s>>>(bt, stg);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}
