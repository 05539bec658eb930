// Kernels around the history integrals:
//   (a)  stencil tables: fractional grid index of phi1, phi2 and psi for every (j, i)
//        (Sec. 3.3, the precomputed theta-interpolation positions),
//   RHS assembly: mu(t), E(t) and the total derivatives at fixed theta (Sec. 2.1),
//   (c)  Runge-Kutta stage combination (Dormand-Prince 5(4) or SSPRK(10,4)), error
//        estimate, the step rule with rollback and the switch between the two
//        methods (Sec. 3.5), all decided on the device,
//   (d)  sparsification (Sec. 3.6): residuals of every candidate slice, the greedy
//        "remove n, skip n+1" selection, and compaction into the other history buffer,
//   two-time lookups C(t,t'), R(t,t') for the API.
// Single-CTA kernels use a fixed reduction tree, so every result is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dmfe_internal.h"

namespace {

constexpr int CTL_THREADS = 1024;

// Explicit Runge-Kutta pairs in first-same-as-last form (Sec. 3.5). Stage 0 is the
// stored derivative of the last slice; stage st = 1..n is evaluated at t + c[st] h on
// Y_st = y + h sum_{l < st} a[st][l] k_l. Row a[n] is the propagating weight vector,
// so Y_n is the new slice and k_n its derivative; the error estimate is
// h sum_{l <= n} e[l] k_l.
struct RKTab {
    int n;
    double c[kMaxStages + 1];
    double a[kMaxStages + 1][kMaxStages];
    double e[kMaxStages + 1];
};

// [0] Dormand & Prince (1980) RK5(4)7M, e = b5 - b4.
// [1] SSPRK(10,4) of Ketcheson (2008): in low-storage form five Euler substeps of h/6,
//     registers recombined as q2 = q2/25 + 9 q1/25, q1 = 15 q2 - 5 q1, four more
//     substeps and u = q2 + 3 q1/5 + h/10 f(q1); as a Butcher tableau the rows below,
//     uniform weights 1/10. Embedded estimate: the third-order weights of minimal
//     2-norm on the same stages with a zero last weight,
//     bhat = (3/20, 1/12, 7/120, 3/40, 2/15, 7/120, 3/40, 2/15, 7/30, 0), e = b - bhat.
__constant__ RKTab kRK[2] = {
    {6,
     {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0},
     {{0},
      {1.0 / 5},
      {3.0 / 40, 9.0 / 40},
      {44.0 / 45, -56.0 / 15, 32.0 / 9},
      {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
      {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
      {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}},
     {35.0 / 384 - 5179.0 / 57600, 0.0, 500.0 / 1113 - 7571.0 / 16695, 125.0 / 192 - 393.0 / 640,
      -2187.0 / 6784 + 92097.0 / 339200, 11.0 / 84 - 187.0 / 2100, -1.0 / 40}},
    {10,
     {0.0, 1.0 / 6, 2.0 / 6, 3.0 / 6, 4.0 / 6, 1.0 / 3, 1.0 / 2, 2.0 / 3, 5.0 / 6, 1.0, 1.0},
     {{0},
      {1.0 / 6},
      {1.0 / 6, 1.0 / 6},
      {1.0 / 6, 1.0 / 6, 1.0 / 6},
      {1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6},
      {1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15},
      {1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 6},
      {1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 6, 1.0 / 6},
      {1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 6, 1.0 / 6, 1.0 / 6},
      {1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 15, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6},
      {1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10, 1.0 / 10,
       1.0 / 10}},
     {1.0 / 10 - 3.0 / 20, 1.0 / 10 - 1.0 / 12, 1.0 / 10 - 7.0 / 120, 1.0 / 10 - 3.0 / 40,
      1.0 / 10 - 2.0 / 15, 1.0 / 10 - 7.0 / 120, 1.0 / 10 - 3.0 / 40, 1.0 / 10 - 2.0 / 15,
      1.0 / 10 - 7.0 / 30, 1.0 / 10, 0.0}},
};

// ---------------------------------------------------------------- grid inverse
__device__ double z_of_i_dev(double i, int L, double alpha, double delta) {
    double y = (2.0 * i - 1.0 - L) / (L - 1.0);
    auto g = [delta](double x) {
        double v = cbrt(fabs(x) * x * x + delta * delta * delta) - delta;
        return x < 0 ? -v : v;
    };
    double phi = 0.5 * (L - 1.0) * (g(y) / g(1.0) + 1.0) + 1.0;
    return alpha * phi + (1.0 - alpha) * i;
}

// 0-based fractional index x with theta(x + 1) = th (Eq. theta inverted); om = 1 - th.
__device__ double frac_index_dev(const SolverView& v, double th, double om) {
    const int L = v.L;
    double y = th <= 0.5 ? log(tan(v.ga + th * v.gD)) / v.gamma : -log(tan(v.ga + om * v.gD)) / v.gamma;
    double z = 0.5 * (y * (L - 1.0) + 1.0 + L);
    double i = z;
    if (v.alpha != 0.0 && v.delta != 0.0) {
        double lo = 1.0, hi = (double)L;
        for (int it = 0; it < 80; ++it) {
            double mid = 0.5 * (lo + hi);
            if (z_of_i_dev(mid, L, v.alpha, v.delta) < z) lo = mid; else hi = mid;
        }
        i = 0.5 * (lo + hi);
    }
    double x = i - 1.0;
    return x < 0.0 ? 0.0 : (x > L - 1.0 ? L - 1.0 : x);
}

// Weights of the s-point theta stencil at base b (Sec. 3.3) for the solver's scheme: the
// default Lagrange basis in the index at u = x - b (product form), or Floater-Hormann
// rational interpolation (Floater & Hormann 2007) with blending degree d -- barycentric
// weights beta_k = sum_{i in J_k} (-1)^i prod_{j=i..i+d, j != k} 1/(x_k - x_j), J_k =
// {max(0, k-d) .. min(k, s-1-d)}, w_k proportional to beta_k / (point - x_k) -- on the
// index nodes 0..s-1 or on the complements 1 - theta of the nodes, at the point's
// complement om (theta schemes; d = s - 1 there for Lagrange).
__device__ void stencil_weights(const SolverView& v, int b, double x, double om, double* w) {
    const int s = v.s;
    if (v.interp == DMFE_INTERP_LAGRANGE_INDEX) {
        const double u = x - b;
        for (int k = 0; k < s; ++k) {
            double p = 1.0;
            for (int m = 0; m < s; ++m)
                if (m != k) p *= (u - m) / (double)(k - m);
            w[k] = p;
        }
        return;
    }
    const bool theta_nodes = v.interp == DMFE_INTERP_LAGRANGE_THETA || v.interp == DMFE_INTERP_FH_THETA;
    const int d = (v.interp == DMFE_INTERP_LAGRANGE_THETA) ? s - 1 : v.fh_d;
    double xn[16];
    for (int k = 0; k < s; ++k) xn[k] = theta_nodes ? v.omega[b + k] : (double)k;
    const double pt = theta_nodes ? om : x - b;
    double sum = 0.0;
    int hit = -1;
    for (int k = 0; k < s; ++k) {
        double beta = 0.0;
        const int i0 = k - d > 0 ? k - d : 0, i1 = k < s - 1 - d ? k : s - 1 - d;
        for (int i = i0; i <= i1; ++i) {
            double term = (i & 1) ? -1.0 : 1.0;
            for (int j = i; j <= i + d; ++j)
                if (j != k) term /= (xn[k] - xn[j]);
            beta += term;
        }
        const double diff = pt - xn[k];
        if (diff == 0.0) hit = k;
        w[k] = diff == 0.0 ? 0.0 : beta / diff;
        sum += w[k];
    }
    for (int k = 0; k < s; ++k) w[k] = hit >= 0 ? (k == hit ? 1.0 : 0.0) : w[k] / sum;
}

// Stencil entry of a fractional index x (point complement om): base b = clamp(floor(x) -
// s/2 + 1, 0, L - s) and the s FP64 weights of the solver's scheme, times `scale`.
__device__ void write_entry(const SolverView& v, unsigned char* base, size_t idx, double x, double om,
                            double scale = 1.0) {
    const int L = v.L, s = v.s;
    int b = (int)floor(x) - s / 2 + 1;
    b = b < 0 ? 0 : (b > L - s ? L - s : b);
    unsigned char* e = base + idx * (size_t)(8 + 8 * s);
    reinterpret_cast<int*>(e)[0] = b;
    reinterpret_cast<int*>(e)[1] = 0;
    double* w = reinterpret_cast<double*>(e + 8);
    stencil_weights(v, b, x, om, w);
    if (scale != 1.0)
        for (int k = 0; k < s; ++k) w[k] *= scale;
}

__global__ void k_tables(SolverView v, double* x1, double* x2, double* x3, uint32_t* p1, uint32_t* p2,
                         uint32_t* p3, df* q1, df* q2, df* q3) {
    const long long LL = (long long)v.L * v.L;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < LL;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx / v.L), i = (int)(idx % v.L);
        const double thj = v.theta[j], omj = v.omega[j], thi = v.theta[i], omi = v.omega[i];
        // phi1 = theta_i theta_j, 1 - phi1 = omega_i + theta_i omega_j
        const double ph1 = thj * thi, oph1 = omi + thi * omj;
        // phi2 = theta_j + omega_j theta_i, 1 - phi2 = omega_j omega_i
        const double ph2 = thj + omj * thi, oph2 = omj * omi;
        // psi = theta_j / phi2, 1 - psi = omega_j theta_i / phi2 (psi = 0 where phi2 = 0)
        double ps = 0.0, ops = 1.0;
        if (ph2 > 0.0) { ps = thj / ph2; ops = omj * thi / ph2; }
        const double a = frac_index_dev(v, ph1, oph1);
        const double b = frac_index_dev(v, ph2, oph2);
        const double c = frac_index_dev(v, ps, ops);
        if (x1) { x1[idx] = a; x2[idx] = b; x3[idx] = c; }
        if (q1) {
            q1[idx] = df_from_d(a);
            q2[idx] = df_from_d(b);
            q3[idx] = df_from_d(c);
        }
        if (v.wt1) {
            // the A1 and A2 stencils (current row at phi1, phi2) carry the quadrature weight
            // nu_i of their summation index: every product they enter is weighted by it
            write_entry(v, (unsigned char*)v.wt1, idx, a, oph1, v.nu[i]);
            write_entry(v, (unsigned char*)v.wt2, idx, b, oph2, v.nu[i]);
            write_entry(v, (unsigned char*)v.wt3, idx, c, ops);
        }
        if (p1) {
            const double sc = (double)(1u << FIX_FRAC_BITS);
            p1[idx] = (uint32_t)llrint(a * sc);
            p2[idx] = (uint32_t)llrint(b * sc);
            p3[idx] = (uint32_t)llrint(c * sc);
        }
    }
}

// ---------------------------------------------------------------- reductions
__device__ double block_sum(double x, double* red) {
    const int tid = threadIdx.x;
    red[tid] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// mu, E and the total derivatives (dCf/dt, dRf/dt at fixed theta) of the row (C, R) at
// time t from the history sums S (layout of dmfe_history_integrals). One CTA.
//   d1C = -mu C + t [theta (S0 + S2) + omega S1] + beta0 f'(C(t,0)) C(t',0)
//   d1R = -mu R + t omega S3
//   mu' = mu(t') = T + t theta S8 + beta0 f'(C(t',0)) C(t',0)
//   d2C = -mu' C + t [theta (S4 + S5) + omega S6] + 2 T R + beta0 f'(C(t',0)) C(t,0)
//   d2R =  mu' R - t omega S7
//   dC  = d1C + theta d2C,  dR = d1R + theta d2R,  0 at theta = 1 (pinned diagonal).
__device__ void assemble_core(const SolverView& v, const double* row, const double* S, double t,
                              double* dC, double* dR, double* mu_out, double* E_out, double* red) {
    const int L = v.L;
    double pm = 0.0, pe = 0.0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const double C = row[i], R = row[L + i];
        const double K = fp2(v.poly, C) * R, D = fp1(v.poly, C);
        pm += v.nu[i] * (K * C + D * R);
        pe += v.nu[i] * (D * R);
    }
    const double sm = block_sum(pm, red);
    const double se = block_sum(pe, red);
    const double C0 = row[0];
    const double mu = v.T + t * sm + v.beta0 * fp1(v.poly, C0) * C0;
    const double E = -t * se - v.beta0 * fp0(v.poly, C0);
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        const double th = v.theta[j], om = v.omega[j];
        const double C = row[j], R = row[L + j];
        const double* s = S + j;
        const double S0 = s[0], S1 = s[L], S2 = s[2 * L], S3 = s[3 * L], S4 = s[4 * L];
        const double S5 = s[5 * L], S6 = s[6 * L], S7 = s[7 * L], S8 = s[8 * L], S9 = s[9 * L];
        const double d1C = -mu * C + t * (th * (S0 + S2) + om * S1) + v.beta0 * fp1(v.poly, C0) * S9;
        const double d1R = -mu * R + t * om * S3;
        const double mup = v.T + t * th * S8 + v.beta0 * fp1(v.poly, S9) * S9;
        const double d2C = -mup * C + t * (th * (S4 + S5) + om * S6) + 2.0 * v.T * R +
                           v.beta0 * fp1(v.poly, S9) * C0;
        const double d2R = mup * R - t * om * S7;
        const bool diag = (j == L - 1);
        dC[j] = diag ? 0.0 : d1C + th * d2C;
        dR[j] = diag ? 0.0 : d1R + th * d2R;
    }
    if (mu_out) *mu_out = mu;
    if (E_out) *E_out = E;
}

__global__ void __launch_bounds__(CTL_THREADS) k_assemble(SolverView v, const double* row, const double* S,
                                                          double t, double* dC, double* dR, double* muE) {
    __shared__ double red[CTL_THREADS];
    double mu, E;
    assemble_core(v, row, S, t, dC, dR, &mu, &E, red);
    if (threadIdx.x == 0 && muE) { muE[0] = mu; muE[1] = E; }
}

// The initial slice t = 0, Cf = Rf = 1: every history integral carries a factor t, and
// C(t', 0) = C(0, 0) = 1, so S = 0 except S[9] = 1.
__global__ void __launch_bounds__(CTL_THREADS) k_initial(SolverView v) {
    __shared__ double red[CTL_THREADS];
    const int L = v.L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        v.Y[i] = 1.0;
        v.Y[L + i] = 1.0;
        for (int r = 0; r < DMFE_NS; ++r) v.S[(size_t)r * L + i] = (r == 9) ? 1.0 : 0.0;
    }
    __syncthreads();
    double* dC = v.k;
    double* dR = v.k + L;
    double mu, E;
    assemble_core(v, v.Y, v.S, 0.0, dC, dR, &mu, &E, red);
    __syncthreads();
    const int act = v.st->active;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        v.hist[act][i] = dbl4{1.0, dC[i], 1.0, dR[i]};
        if (v.hist32[act]) v.hist32[act][i] = make_float4(1.f, (float)dC[i], 1.f, (float)dR[i]);
        if (v.histdf[act]) v.histdf[act][i] = df8{df{1.f, 0.f}, df_from_d(dC[i]), df{1.f, 0.f}, df_from_d(dR[i])};
    }
    if (threadIdx.x == 0) {
        v.ht[act][0] = 0.0;
        DevState* st = v.st;
        st->n = 1;
        st->t = 0.0;
        st->mu = mu;
        st->E = E;
    }
}

__device__ __forceinline__ bool gated(const DevState* st) { return st->status != 0 || st->done; }

// Monomial coefficients of the cubic Hermite interpolant between history points a (at t_k)
// and b (at t_k + h), for C (x, y = value, derivative) and R (z, w).
__device__ __forceinline__ dbl8 interval_coef(const dbl4& a, const dbl4& b, double h) {
    const double dC = b.x - a.x, dR = b.z - a.z;
    dbl8 c;
    c.c0 = a.x;
    c.c1 = h * a.y;
    c.c2 = 3.0 * dC - h * (2.0 * a.y + b.y);
    c.c3 = -2.0 * dC + h * (a.y + b.y);
    c.r0 = a.z;
    c.r1 = h * a.w;
    c.r2 = 3.0 * dR - h * (2.0 * a.w + b.w);
    c.r3 = -2.0 * dR + h * (a.w + b.w);
    return c;
}

// Monomial coefficients of the cubic Hermite interpolant of log R between history points a
// and b (log-R mode, App. A): values log R, derivatives R'/R. x = NaN where either R is not
// positive (the kernels then interpolate R itself).
__device__ __forceinline__ dbl4 interval_logcoef(const dbl4& a, const dbl4& b, double h) {
    if (!(a.z > 0.0 && b.z > 0.0)) return dbl4{nan(""), 0.0, 0.0, 0.0};
    const double la = log(a.z), lb = log(b.z), da = a.w / a.z, db = b.w / b.z, dl = lb - la;
    return dbl4{la, h * da, 3.0 * dl - h * (2.0 * da + db), -2.0 * dl + h * (da + db)};
}

// Write slice `slot` = (t, Y, dY) to buffer `act`: FP64 master, the replica of the
// precision, and (FP64 path) the interval coefficients between slots slot-1 and slot.
__device__ void append_slice(const SolverView& v, int act, int slot, double t, const double* Y,
                             const double* dY) {
    const int L = v.L;
    dbl4* H = v.hist[act] + (size_t)slot * L;
    float4* H32 = v.hist32[act] ? v.hist32[act] + (size_t)slot * L : nullptr;
    df8* HD = v.histdf[act] ? v.histdf[act] + (size_t)slot * L : nullptr;
    dbl8* HC = (v.hcoef[act] && slot >= 1) ? v.hcoef[act] + (size_t)(slot - 1) * L : nullptr;
    dbl4* LC = (v.lcoef[act] && slot >= 1) ? v.lcoef[act] + (size_t)(slot - 1) * L : nullptr;
    const double hprev = slot >= 1 ? t - v.ht[act][slot - 1] : 0.0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const dbl4 e{Y[i], dY[i], Y[L + i], dY[L + i]};
        H[i] = e;
        if (H32) H32[i] = make_float4((float)e.x, (float)e.y, (float)e.z, (float)e.w);
        if (HD) HD[i] = df8{df_from_d(e.x), df_from_d(e.y), df_from_d(e.z), df_from_d(e.w)};
        if (HC) HC[i] = interval_coef(H[(long long)i - L], e, hprev);
        if (LC) LC[i] = interval_logcoef(H[(long long)i - L], e, hprev);
    }
    if (threadIdx.x == 0) v.ht[act][slot] = t;
}

__global__ void __launch_bounds__(CTL_THREADS) k_begin_integrate(SolverView v, double t_target, double tol) {
    if (threadIdx.x != 0) return;
    DevState* st = v.st;
    st->t_target = t_target;
    st->tol = tol;
    st->done = (st->t >= t_target) ? 1 : 0;
}

// Start of a trial step (multi-CTA): the method of the step (fixed until the step ends),
// h = min(dt, t_target - t), k_0 = stored derivative of the last slice
// (first-same-as-last), stage-1 row Y_1 = y + h a_10 k_0 into buffer 1.
__device__ __forceinline__ void step_begin_body(const SolverView& v, int cta, int ncta) {
    DevState* st = v.st;
    if (gated(st)) return;
    const int L = v.L;
    const int m = st->method;
    const RKTab& M = kRK[m];
    const dbl4* yrow = v.hist[st->active] + (size_t)(st->n - 1) * L;
    const double t = st->t;
    const double h = fmin(st->dt, st->t_target - t);
    double* Y1 = v.Y + 2 * (size_t)L;
    for (int j = cta * blockDim.x + threadIdx.x; j < L; j += ncta * blockDim.x) {
        const dbl4 e = yrow[j];
        v.k[j] = e.y;
        v.k[L + j] = e.w;
        Y1[j] = __dadd_rn(e.x, __dmul_rn(h, __dmul_rn(M.a[1][0], e.y)));
        Y1[L + j] = __dadd_rn(e.z, __dmul_rn(h, __dmul_rn(M.a[1][0], e.w)));
    }
    if (cta == 0 && threadIdx.x == 0) {
        st->rk = m;
        st->nst = M.n;
        st->h = h;
        st->t_stage = __dadd_rn(t, __dmul_rn(M.c[1], h));
    }
}

// End of stage stg (1..n of the step's method), multi-CTA: k_stg from the sums S and the
// stage row (read from buffer stg & 1); then either the next stage row (written to the
// other buffer) or, after the last stage, the error estimate, whose per-CTA partials
// the last CTA to finish adds in a fixed order before taking the step decision of
// Sec. 3.5 (and the switch to SSPRK(10,4)) and appending the slice. mu and E come from
// the per-block partial sums of the prep kernel.
__device__ __forceinline__ void stage_end_body(const SolverView& v, int stg, int prep_blocks, int cta, int ncta) {
    __shared__ double s_mu, s_E, red[kCtlThreads];
    __shared__ int s_last, s_append;
    DevState* st = v.st;
    if (stage_off(st, stg)) return;
    const RKTab& M = kRK[st->rk];
    const int nst = M.n;
    const int L = v.L;
    const int L2 = 2 * L;
    const int act = st->active;
    const int n = st->n;
    const dbl4* yrow = v.hist[act] + (size_t)(n - 1) * L;
    const double t = st->t, h = st->h;
    const double ts = __dadd_rn(t, __dmul_rn(M.c[stg], h));  // this stage's time
    const double* Yc = v.Y + (size_t)(stg & 1) * L2;
    double* Yn = v.Y + (size_t)((stg + 1) & 1) * L2;
    const double C0 = Yc[0];
    if (threadIdx.x == 0) {
        double sm = 0.0, se = 0.0;
        for (int b = 0; b < prep_blocks; ++b) {
            sm += v.mupart[b];
            se += v.mupart[kMaxPrepBlocks + b];
        }
        s_mu = v.T + ts * sm + v.beta0 * fp1(v.poly, C0) * C0;
        s_E = -ts * se - v.beta0 * fp0(v.poly, C0);
    }
    __syncthreads();
    const double mu = s_mu;
    double* kC = v.k + (size_t)stg * L2;
    double pe = 0.0;
    for (int j = cta * blockDim.x + threadIdx.x; j < L; j += ncta * blockDim.x) {
        const double th = v.theta[j], om = v.omega[j];
        const double C = Yc[j], R = Yc[L + j];
        const double* sj = v.S + j;
        const double S0 = sj[0], S1 = sj[L], S2 = sj[2 * L], S3 = sj[3 * L], S4 = sj[4 * L];
        const double S5 = sj[5 * L], S6 = sj[6 * L], S7 = sj[7 * L], S8 = sj[8 * L], S9 = sj[9 * L];
        const double d1C = -mu * C + ts * (th * (S0 + S2) + om * S1) + v.beta0 * fp1(v.poly, C0) * S9;
        const double d1R = -mu * R + ts * om * S3;
        const double mup = v.T + ts * th * S8 + v.beta0 * fp1(v.poly, S9) * S9;
        const double d2C = -mup * C + ts * (th * (S4 + S5) + om * S6) + 2.0 * v.T * R +
                           v.beta0 * fp1(v.poly, S9) * C0;
        const double d2R = mup * R - ts * om * S7;
        const bool diag = (j == L - 1);
        kC[j] = diag ? 0.0 : d1C + th * d2C;
        kC[L + j] = diag ? 0.0 : d1R + th * d2R;
        if (stg < nst) {
            // next stage row Y = y + h sum_{l <= stg} a[stg+1][l] k_l, rounded like the plain sum
            for (int half = 0; half < 2; ++half) {
                const int q = j + half * L;
                double acc = 0.0;
                for (int l = 0; l <= stg; ++l) acc = __dadd_rn(acc, __dmul_rn(M.a[stg + 1][l], v.k[(size_t)l * L2 + q]));
                const double y = half == 0 ? yrow[j].x : yrow[j].z;
                Yn[q] = __dadd_rn(y, __dmul_rn(h, acc));
            }
        } else {
            // embedded error estimate h sum_l e_l k_l, 1-norm
            for (int half = 0; half < 2; ++half) {
                const int q = j + half * L;
                double acc = 0.0;
                for (int l = 0; l <= nst; ++l) acc = __dadd_rn(acc, __dmul_rn(M.e[l], v.k[(size_t)l * L2 + q]));
                pe += fabs(__dmul_rn(h, acc));
            }
        }
    }
    if (stg < nst) {
        if (cta == 0 && threadIdx.x == 0) {
            st->stages += 1;
            st->t_stage = __dadd_rn(t, __dmul_rn(M.c[stg + 1], h));
        }
        return;
    }
    const double ep = block_sum(pe, red);
    if (threadIdx.x == 0) {
        v.epart[cta] = ep;
        __threadfence();
        s_last = atomicAdd(v.ctl_count, 1) == ncta - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double eps = 0.0;
        for (int b = 0; b < ncta; ++b) eps += __ldcg(&v.epart[b]);
        *v.ctl_count = 0;
        st->stages += 1;
        st->eps = eps;
        st->mu = s_mu;
        st->E = s_E;
        s_append = -1;
        const double tol = st->tol;
        if (!isfinite(eps)) {
            st->status = DMFE_ERR_NONFINITE;
        } else if (eps > 2.0 * tol) {
            // reject: revert the last min(10, n-1) slices and halve the step
            st->steps_rejected += 1;
            const int drop = n - 1 < 10 ? n - 1 : 10;
            st->n = n - drop;
            st->t = v.ht[act][n - drop - 1];
            st->dt *= 0.5;
        } else {
            st->steps_accepted += 1;
            const double tnew = (h < st->t_target - t) ? t + h : st->t_target;
            if (n >= v.cap) {
                // a full store: a sparsification round whose first pass makes room for
                // the new slice (appended when that pass finishes)
                if (v.sparsify) { st->pending = 1; st->t_pending = tnew; st->sp_left = v.sp_passes; }
                else st->status = DMFE_ERR_CAPACITY;
            } else {
                s_append = n;
                st->t_pending = tnew;
                // the periodic round, after this step's append
                if (v.sp_every > 0 && st->steps_accepted % v.sp_every == 0) st->sp_left = v.sp_passes;
            }
            if (eps > tol) st->dt *= 0.9;
            else if (eps < 0.5 * tol) st->dt *= 1.01;
            if (st->rk == 0 && st->dt >= v.rk_switch_dt) {
                // Dormand-Prince has reached its stability limit: SSPRK(10,4) from the
                // next step on, with the step halved
                st->method = 1;
                st->dt *= 0.5;
                st->t_switch = tnew;
            }
        }
        if (st->status == 0 && st->dt < st->dt_min) st->status = DMFE_ERR_STEP_UNDERFLOW;
    }
    __syncthreads();
    if (s_append >= 0) {
        // the new solution Y_n sits in buffer n & 1, its derivative in k[n]
        append_slice(v, act, s_append, st->t_pending, v.Y + (size_t)(nst & 1) * L2, v.k + (size_t)nst * L2);
        __syncthreads();
        if (threadIdx.x == 0) {
            st->n = s_append + 1;
            st->t = st->t_pending;
            if (st->t >= st->t_target) st->done = 1;
        }
    }
}

__device__ __forceinline__ int ctl_grid(int L) {
    const int g = (L + kCtlThreads - 1) / kCtlThreads;
    return g < 1 ? 1 : (g > kCtlGrid ? kCtlGrid : g);
}

// COND: the launch belongs to a step graph whose stages beyond kDP5Stages sit in a
// conditional node with handle `cond`; one thread enables it for a live SSPRK step. (A
// separate instantiation without the call keeps the plain variant visible to profilers,
// which skip kernels that can set graph conditions.)
template <bool COND>
__global__ void __launch_bounds__(kCtlThreads) k_step_begin(SolverView v, cudaGraphConditionalHandle cond) {
    step_begin_body(v, blockIdx.x, gridDim.x);
    if (COND && blockIdx.x == 0 && threadIdx.x == 0 && !gated(v.st) && kRK[v.st->method].n > kDP5Stages)
        cudaGraphSetConditional(cond, 1u);
}

__global__ void __launch_bounds__(kCtlThreads) k_stage_end(SolverView v, int stg, int prep_blocks) {
    stage_end_body(v, stg, prep_blocks, blockIdx.x, gridDim.x);
}

// Batched wrappers: blockIdx.y is the slot; each slot keeps its own CTA partition.
template <bool COND>
__global__ void __launch_bounds__(kCtlThreads) k_batch_step_begin(const BatchTable* __restrict__ bt,
                                                                  cudaGraphConditionalHandle cond) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        // work offsets of the slots whose step has stages beyond the Dormand-Prince ones
        // (their method does not change while the step runs), and the graph condition
        long long* wl = const_cast<BatchTable*>(bt)->woff_late;
        long long w = 0;
        for (int q = 0; q < bt->count; ++q) {
            wl[q] = w;
            if (!bt->active[q]) continue;
            const SolverView& vq = bt->views[q];
            if (!gated(vq.st) && kRK[vq.st->method].n > kDP5Stages) w += (long long)vq.L * vq.L;
        }
        wl[bt->count] = w;
        if (COND) cudaGraphSetConditional(cond, w > 0 ? 1u : 0u);
    }
    const int k = blockIdx.y;
    if (k >= bt->count || !bt->active[k]) return;
    const SolverView& v = bt->views[k];
    const int g = ctl_grid(v.L);
    if ((int)blockIdx.x < g) step_begin_body(v, blockIdx.x, g);
}

__global__ void __launch_bounds__(kCtlThreads) k_batch_stage_end(const BatchTable* __restrict__ bt, int stg) {
    const int k = blockIdx.y;
    if (k >= bt->count || !bt->active[k]) return;
    const SolverView& v = bt->views[k];
    const int g = ctl_grid(v.L);
    const int tot = v.L > v.cap ? v.L : v.cap;
    if ((int)blockIdx.x < g) stage_end_body(v, stg, (tot + kPrepThreads - 1) / kPrepThreads, blockIdx.x, g);
}

// ---------------------------------------------------------------- sparsification


// A pass of the step graph runs while the current round has passes left (a round is set
// by the step decision: on a full store, or after every sp_every-th accepted step); an
// explicit call (dmfe_sparsify) always runs.
__device__ __forceinline__ bool sp_active(const DevState* st, int from_step) {
    return from_step ? (st->sp_left > 0 && st->status == 0) : true;
}

// eps_sparse(n) for candidates n = 1 .. N-12: one CTA per candidate (CTA `cta` takes n =
// cta + 1), its threads striding over the grid index; each thread adds its terms in i
// order, the warps reduce with a fixed butterfly and the first thread adds the warp sums in
// warp order, so the result is deterministic.
constexpr int SP_RES_THREADS = 128;

__device__ __forceinline__ void sp_residual_body(const SolverView& v, int from_step, int cta) {
    const DevState* st = v.st;
    if (!sp_active(st, from_step)) return;
    const int L = v.L;
    const int N = st->n;
    const int n = cta + 1;
    if (n > N - 12) return;
    if (!DMFE_IN_BOUNDS(v.st, n + 1 < N && N <= v.cap, 31)) return;
    const int act = st->active;
    const dbl4* H = v.hist[act];
    const double* ht = v.ht[act];
    const double h1 = ht[n] - ht[n - 1], h2 = ht[n + 1] - ht[n];
    const dbl4* a = H + (size_t)(n - 1) * L;
    const dbl4* b = H + (size_t)n * L;
    const dbl4* c = H + (size_t)(n + 1) * L;
    // Delta_n = (I[t_{n-1}, t_n] + I[t_n, t_{n+1}]) - I[t_{n-1}, t_{n+1}] with the Hermite
    // integral I = h (y0 + y1)/2 + h^2 (y0' - y1')/12 is linear in the six stored values:
    // weights -h2/2, (h1 + h2)/2, -h1/2 on the values and (h1^2 - h^2)/12, (h2^2 - h1^2)/12,
    // (h^2 - h2^2)/12 on the derivatives (h = h1 + h2), formed once per candidate
    const SpWeights wt = sp_weights(h1, h2);
    double acc = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const dbl4 A = a[i], B = b[i], Cc = c[i];
        acc += fabs(sp_delta(wt, A.x, A.y, B.x, B.y, Cc.x, Cc.y)) + fabs(sp_delta(wt, A.z, A.w, B.z, B.w, Cc.z, Cc.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double wsum[SP_RES_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e += wsum[w];
        v.eps_sp[n] = e;
    }
}

// Exclusive scan over the threads of the CTA (Hillis-Steele in shared memory, fixed
// order); *total receives the combination over all threads.
template <typename T, typename Op>
__device__ __forceinline__ T block_exclusive_scan(T x, T identity, Op op, T* buf, T* total) {
    const int t = threadIdx.x, nt = blockDim.x;
    buf[t] = x;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const T y = t >= off ? buf[t - off] : identity;
        __syncthreads();
        buf[t] = op(buf[t], y);
        __syncthreads();
    }
    const T excl = t > 0 ? buf[t - 1] : identity;
    *total = buf[nt - 1];
    __syncthreads();
    return excl;
}

// Selection of a pass (Sec. 3.6) by one CTA. The greedy scan -- remove n if eps(n) < tol/10,
// then skip n+1 -- removes, within each maximal run of consecutive qualifying candidates, the
// run's 1st, 3rd, 5th, ... members, so a candidate's fate depends only on its position in
// its run: an exclusive max-scan gives the last non-qualifying index before each index, and
// an exclusive sum-scan of the kept slices gives the compaction map. A pass that may force a
// removal and finds none removes the candidate with the smallest residual (the first of
// equal ones). Thread t takes the contiguous indices [t P, (t + 1) P) of [0, N),
// P = ceil(N / blockDim).
__device__ __forceinline__ void sp_select_body(const SolverView& v, int from_step, double tol_arg) {
    __shared__ int s_int[CTL_THREADS];
    __shared__ double s_dbl[CTL_THREADS];
    DevState* st = v.st;
    // every thread reads the pass's state before thread 0 changes it
    if (!sp_active(st, from_step)) return;
    // the first pass of a full-store round (and an explicit pass) must free a slot, so it
    // may force a removal; the other passes remove only slices that qualify
    const bool force = from_step ? st->pending != 0 : true;
    const int N = st->n;
    const double tol = from_step ? st->tol : tol_arg;
    const double mx0 = st->max_eps_sparse;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (from_step) st->sp_left -= 1;
        st->sp_ran = 0;
    }
    const int last = N - 12;
    if (last < 1) {
        if (threadIdx.x == 0 && from_step && force) st->status = DMFE_ERR_CAPACITY;
        return;
    }
    const double thr = tol / 10.0;
    const double* __restrict__ eps = v.eps_sp;
    const int T = blockDim.x, t = threadIdx.x;
    const int P = (N + T - 1) / T;
    const int lo = t * P < N ? t * P : N, hi = lo + P < N ? lo + P : N;
    auto ok = [&](int k) { return k >= 1 && k <= last && eps[k] < thr; };
    // last non-qualifying index before this thread's block
    int zmax = -1;
    for (int k = lo; k < hi; ++k)
        if (!ok(k)) zmax = k;
    int zall;
    const int pf0 = block_exclusive_scan(zmax, -1, [](int x, int y) { return x > y ? x : y; }, s_int, &zall);
    // decisions and the kept count of the block
    int kept = 0, removed_loc = 0;
    double mx = -1.0;
    {
        int pf = pf0;
        for (int k = lo; k < hi; ++k) {
            const bool q = ok(k);
            const bool rm = q && ((k - pf - 1) % 2 == 0);
            if (!q) pf = k;
            kept += rm ? 0 : 1;
            removed_loc += rm ? 1 : 0;
            if (rm) mx = fmax(mx, eps[k]);
        }
    }
    int kept_all;
    const int base = block_exclusive_scan(kept, 0, [](int x, int y) { return x + y; }, s_int, &kept_all);
    double mx_all;
    block_exclusive_scan(mx, -1.0, [](double x, double y) { return fmax(x, y); }, s_dbl, &mx_all);
    {
        int pf = pf0, c = base;
        for (int k = lo; k < hi; ++k) {
            const bool q = ok(k);
            const bool rm = q && ((k - pf - 1) % 2 == 0);
            if (!q) pf = k;
            v.keep[k] = rm ? 0 : 1;
            v.newidx[k] = c;
            c += rm ? 0 : 1;
        }
    }
    int removed = N - kept_all;
    if (removed == 0 && !force) {
        // nothing qualifies and nothing is forced: the pass counts, the history stays
        if (t == 0) {
            st->sparsify_passes += 1;
            st->removed_count = 0;
        }
        return;
    }
    double mx_new = fmax(mx0, mx_all);
    if (removed == 0) {
        // every slice was kept, so newidx[k] = k; remove the smallest residual m (the first
        // of equal ones): a block minimum of the value, then of the index among equal values
        double em = INFINITY;
        for (int k = lo; k < hi; ++k)
            if (k >= 1 && k <= last && eps[k] < em) em = eps[k];
        double em_all;
        block_exclusive_scan(em, (double)INFINITY, [](double x, double y) { return fmin(x, y); }, s_dbl, &em_all);
        int m_loc = 0x7fffffff;
        for (int k = lo; k < hi; ++k)
            if (k >= 1 && k <= last && eps[k] == em_all) { m_loc = k; break; }
        int m;
        block_exclusive_scan(m_loc, 0x7fffffff, [](int x, int y) { return x < y ? x : y; }, s_int, &m);
        if (m == 0x7fffffff) m = 1;  // no finite minimum (NaN residuals): the first candidate, as the scan
        for (int k = lo; k < hi; ++k) {
            if (k == m) v.keep[k] = 0;
            if (k > m) v.newidx[k] = k - 1;
        }
        kept_all = N - 1;
        removed = 1;
        mx_new = fmax(mx_new, em_all);
        if (t == 0) st->forced_removals += 1;
    }
    if (t == 0) {
        st->max_eps_sparse = mx_new;
        st->sparsify_passes += 1;
        st->slices_removed += removed;
        st->removed_count = removed;
        st->n_new = kept_all;
        st->sp_ran = 1;
    }
}

__device__ __forceinline__ void sp_compact_body(const SolverView& v, int cta, int ncta) {
    const DevState* st = v.st;
    if (!st->sp_ran) return;
    const int L = v.L;
    const int N = st->n;
    const int act = st->active, nxt = 1 - act;
    const long long tot = (long long)N * L;
    for (long long q = cta * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)ncta * blockDim.x) {
        const int k = (int)(q / L), i = (int)(q % L);
        if (!v.keep[k]) continue;
        if (!DMFE_IN_BOUNDS(v.st, v.newidx[k] >= 0 && v.newidx[k] < v.cap && N <= v.cap, 32)) continue;
        const size_t dst = (size_t)v.newidx[k] * L + i;
        v.hist[nxt][dst] = v.hist[act][q];
        if (v.hist32[act]) v.hist32[nxt][dst] = v.hist32[act][q];
        if (v.histdf[act]) v.histdf[nxt][dst] = v.histdf[act][q];
        if (v.hcoef[act] && k > 0) {
            // interval from the previous kept slice (slice 0 is never removed)
            int p = k - 1;
            while (p > 0 && !v.keep[p]) --p;
            v.hcoef[nxt][dst - L] = interval_coef(v.hist[act][(size_t)p * L + i], v.hist[act][q],
                                                  v.ht[act][k] - v.ht[act][p]);
            if (v.lcoef[act])
                v.lcoef[nxt][dst - L] = interval_logcoef(v.hist[act][(size_t)p * L + i], v.hist[act][q],
                                                         v.ht[act][k] - v.ht[act][p]);
        }
        if (i == 0) v.ht[nxt][v.newidx[k]] = v.ht[act][k];
    }
}

__device__ __forceinline__ void sp_finish_body(const SolverView& v) {
    DevState* st = v.st;
    if (!st->sp_ran) return;
    __syncthreads();
    const int nxt = 1 - st->active;
    const int nn = st->n_new;
    const bool pend = st->pending != 0;
    __syncthreads();
    // the accepted solution of the step that left the slice pending: Y_n in buffer n & 1,
    // its derivative in k[n] (n = the step's stage count)
    const int nst = st->nst;
    if (pend) append_slice(v, nxt, nn, st->t_pending, v.Y + (size_t)(nst & 1) * 2 * v.L, v.k + (size_t)nst * 2 * v.L);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->active = nxt;
        st->n = pend ? nn + 1 : nn;
        st->sp_ran = 0;
        if (pend) {
            st->pending = 0;
            st->t = st->t_pending;
            if (st->t >= st->t_target) st->done = 1;
        }
    }
}

__global__ void __launch_bounds__(SP_RES_THREADS) k_sp_residual(SolverView v, int from_step) {
    sp_residual_body(v, from_step, blockIdx.x);
}
__global__ void __launch_bounds__(CTL_THREADS) k_sp_select(SolverView v, int from_step, double tol_arg) {
    sp_select_body(v, from_step, tol_arg);
}
__global__ void k_sp_compact(SolverView v) { sp_compact_body(v, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(CTL_THREADS) k_sp_finish(SolverView v) { sp_finish_body(v); }

__global__ void __launch_bounds__(SP_RES_THREADS) k_batch_sp_residual(const BatchTable* __restrict__ bt) {
    const int k = blockIdx.y;
    if (k >= bt->count || !bt->active[k]) return;
    sp_residual_body(bt->views[k], 1, blockIdx.x);
}
__global__ void __launch_bounds__(CTL_THREADS) k_batch_sp_select(const BatchTable* __restrict__ bt) {
    const int k = blockIdx.x;
    if (k >= bt->count || !bt->active[k]) return;
    sp_select_body(bt->views[k], 1, 0.0);
}
__global__ void k_batch_sp_compact(const BatchTable* __restrict__ bt) {
    const int k = blockIdx.y;
    if (k >= bt->count || !bt->active[k]) return;
    sp_compact_body(bt->views[k], blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(CTL_THREADS) k_batch_sp_finish(const BatchTable* __restrict__ bt) {
    const int k = blockIdx.x;
    if (k >= bt->count || !bt->active[k]) return;
    sp_finish_body(bt->views[k]);
}

// ---------------------------------------------------------------- lookups
__global__ void k_lookup(SolverView v, int nq, const double* tq, const double* tpq, int which, double* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const DevState* st = v.st;
    const int L = v.L, n = st->n, act = st->active, s = v.s;
    const double t = tq[q], tp = tpq[q];
    if (which == 1 && tp > t) { out[q] = 0.0; return; }
    const double big = fmax(t, tp), small = fmin(t, tp);
    const double th = big > 0 ? small / big : 1.0;
    const double om = big > 0 ? (big - small) / big : 0.0;
    const double x = frac_index_dev(v, th, om);
    int b = (int)floor(x) - s / 2 + 1;
    b = b < 0 ? 0 : (b > L - s ? L - s : b);
    double w[16];
    stencil_weights(v, b, x, om, w);
    const dbl4* H = v.hist[act];
    const double* ht = v.ht[act];
    auto val = [&](int sl, bool deriv) {
        double acc = 0.0;
        for (int k = 0; k < s; ++k) {
            const dbl4 e = H[(size_t)sl * L + b + k];
            acc += w[k] * (which == 0 ? (deriv ? e.y : e.x) : (deriv ? e.w : e.z));
        }
        return acc;
    };
    // log-R mode for R: the same interpolation of log R and R'/R where the stencil's R is
    // positive on the slices involved (App. A)
    const bool logr = which == 1 && v.log_r;
    auto positive = [&](int sl) {
        for (int k = 0; k < s; ++k)
            if (!(H[(size_t)sl * L + b + k].z > 0.0)) return false;
        return true;
    };
    auto lval = [&](int sl, bool deriv) {
        double acc = 0.0;
        for (int k = 0; k < s; ++k) {
            const dbl4 e = H[(size_t)sl * L + b + k];
            acc += w[k] * (deriv ? e.w / e.z : log(e.z));
        }
        return acc;
    };
    if (n == 1) {
        out[q] = (logr && positive(0)) ? exp(lval(0, false)) : val(0, false);
        return;
    }
    int lo = 0, hi = n - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ht[mid] <= big) lo = mid; else hi = mid - 1;
    }
    const double hh = ht[lo + 1] - ht[lo];
    const double sg = (big - ht[lo]) / hh, o = 1.0 - sg;
    const double h00 = (1.0 + 2.0 * sg) * o * o, h10 = sg * o * o * hh, h01 = sg * sg * (3.0 - 2.0 * sg),
                 h11 = sg * sg * (sg - 1.0) * hh;
    if (logr && positive(lo) && positive(lo + 1)) {
        out[q] = exp(h00 * lval(lo, false) + h10 * lval(lo, true) + h01 * lval(lo + 1, false) +
                     h11 * lval(lo + 1, true));
        return;
    }
    out[q] = h00 * val(lo, false) + h10 * val(lo, true) + h01 * val(lo + 1, false) + h11 * val(lo + 1, true);
}

__global__ void k_refresh_replica(SolverView v) {
    const DevState* st = v.st;
    const int act = st->active;
    const long long tot = (long long)st->n * v.L;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        const dbl4 e = v.hist[act][q];
        if (v.hist32[act]) v.hist32[act][q] = make_float4((float)e.x, (float)e.y, (float)e.z, (float)e.w);
        if (v.histdf[act]) v.histdf[act][q] = df8{df_from_d(e.x), df_from_d(e.y), df_from_d(e.z), df_from_d(e.w)};
        const int k = (int)(q / v.L);
        if (v.hcoef[act] && k + 1 < st->n)
            v.hcoef[act][q] = interval_coef(e, v.hist[act][q + v.L], v.ht[act][k + 1] - v.ht[act][k]);
        if (v.lcoef[act] && k + 1 < st->n)
            v.lcoef[act][q] = interval_logcoef(e, v.hist[act][q + v.L], v.ht[act][k + 1] - v.ht[act][k]);
    }
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_tables(const SolverView& v, cudaStream_t s) {
    k_tables<<<grid_for((long long)v.L * v.L, 256), 256, 0, s>>>(
        v, (double*)v.x1, (double*)v.x2, (double*)v.x3, (uint32_t*)v.p1, (uint32_t*)v.p2, (uint32_t*)v.p3,
        (df*)v.q1, (df*)v.q2, (df*)v.q3);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_assemble(const SolverView& v, const double* row_dev, const double* S_dev, double t,
                    double* dC, double* dR, double* muE, cudaStream_t s) {
    k_assemble<<<1, CTL_THREADS, 0, s>>>(v, row_dev, S_dev, t, dC, dR, muE);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_initial_slice(const SolverView& v, cudaStream_t s) {
    k_initial<<<1, CTL_THREADS, 0, s>>>(v);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_begin_integrate(const SolverView& v, double t_target, double tol, cudaStream_t s) {
    k_begin_integrate<<<1, 32, 0, s>>>(v, t_target, tol);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_sparsify(const SolverView& v, bool from_step, double tol, cudaStream_t s) {
    const int fs = from_step ? 1 : 0;
    k_sp_residual<<<v.cap > 13 ? v.cap - 12 : 1, SP_RES_THREADS, 0, s>>>(v, fs);
    k_sp_select<<<1, CTL_THREADS, 0, s>>>(v, fs, tol);
    k_sp_compact<<<grid_for((long long)v.cap * v.L, 256), 256, 0, s>>>(v);
    k_sp_finish<<<1, CTL_THREADS, 0, s>>>(v);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

// One trial step, in three parts so that a graph can put the stages beyond the
// Dormand-Prince ones into a conditional node: the head (begin and stages 1..6), the
// tail (stages 7..10, which do nothing in a Dormand-Prince step) and the sparsification
// kernels, which do nothing unless the step left a slice pending.
static int ctl_grid_host(int L) {
    int g = (L + kCtlThreads - 1) / kCtlThreads;
    return g < 1 ? 1 : (g > kCtlGrid ? kCtlGrid : g);
}

static int launch_stages(const SolverView& v, int grid_ctas, int s0, int s1, cudaStream_t s) {
    const int g = ctl_grid_host(v.L);
    const int tot = v.L > v.cap ? v.L : v.cap;
    const int prep_blocks = (tot + kPrepThreads - 1) / kPrepThreads;
    for (int stg = s0; stg <= s1; ++stg) {
        const double* row = v.Y + (size_t)(stg & 1) * 2 * v.L;
        int rc = launch_history_integrals(v, row, 0.0, stg, v.S, grid_ctas, s);
        if (rc) return rc;
        k_stage_end<<<g, kCtlThreads, 0, s>>>(v, stg, prep_blocks);
    }
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_step_head(const SolverView& v, int grid_ctas, cudaGraphConditionalHandle cond, int use_cond,
                     cudaStream_t s) {
    if (use_cond) k_step_begin<true><<<ctl_grid_host(v.L), kCtlThreads, 0, s>>>(v, cond);
    else k_step_begin<false><<<ctl_grid_host(v.L), kCtlThreads, 0, s>>>(v, cond);
    return launch_stages(v, grid_ctas, 1, kDP5Stages, s);
}

int launch_step_tail(const SolverView& v, int grid_ctas, cudaStream_t s) {
    return launch_stages(v, grid_ctas, kDP5Stages + 1, kMaxStages, s);
}

// The passes of a sparsification round: sp_passes copies of the pass kernels, each doing
// nothing unless the round still has passes left.
int launch_step_sparsify(const SolverView& v, cudaStream_t s) {
    for (int p = 0; p < (v.sp_passes > 0 ? v.sp_passes : 1); ++p) {
        const int rc = launch_sparsify(v, true, 0.0, s);
        if (rc) return rc;
    }
    return DMFE_OK;
}

int launch_step(const SolverView& v, int grid_ctas, cudaStream_t s) {
    int rc = launch_step_head(v, grid_ctas, 0, 0, s);
    if (!rc) rc = launch_step_tail(v, grid_ctas, s);
    if (!rc) rc = launch_step_sparsify(v, s);
    return rc;
}

int launch_lookup(const SolverView& v, int n, const double* t, const double* tp, int which, double* out,
                  cudaStream_t s) {
    k_lookup<<<(n + 127) / 128, 128, 0, s>>>(v, n, t, tp, which, out);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_refresh_replica(const SolverView& v, cudaStream_t s) {
    if (!v.hist32[0] && !v.histdf[0] && !v.hcoef[0] && !v.lcoef[0]) return DMFE_OK;
    k_refresh_replica<<<grid_for((long long)v.cap * v.L, 256), 256, 0, s>>>(v);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

// One batched trial step over every active slot of the batch table, in the same three
// parts as launch_step, with blockIdx.y (or blockIdx.x for per-slot kernels) the slot.
static int launch_batch_stages(const BatchTable* bt, int precision, int sw, int max_L, int max_cap, int slots,
                               int hi_grid, size_t hi_smem, int s0, int s1, cudaStream_t s) {
    const int g = ctl_grid_host(max_L);
    const int max_tot = max_L > max_cap ? max_L : max_cap;
    for (int stg = s0; stg <= s1; ++stg) {
        int rc = launch_batch_prep(bt, stg, max_tot, slots, s);
        if (rc) return rc;
        rc = launch_batch_hi(bt, precision, sw, stg, hi_grid, hi_smem, s);
        if (rc) return rc;
        k_batch_stage_end<<<dim3(g, slots), kCtlThreads, 0, s>>>(bt, stg);
    }
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

int launch_batch_step_head(const BatchTable* bt, int precision, int sw, int max_L, int max_cap, int slots,
                           int hi_grid, size_t hi_smem, cudaGraphConditionalHandle cond, int use_cond,
                           cudaStream_t s) {
    const dim3 grid(ctl_grid_host(max_L), slots);
    if (use_cond) k_batch_step_begin<true><<<grid, kCtlThreads, 0, s>>>(bt, cond);
    else k_batch_step_begin<false><<<grid, kCtlThreads, 0, s>>>(bt, cond);
    return launch_batch_stages(bt, precision, sw, max_L, max_cap, slots, hi_grid, hi_smem, 1, kDP5Stages, s);
}

int launch_batch_step_tail(const BatchTable* bt, int precision, int sw, int max_L, int max_cap, int slots,
                           int hi_grid, size_t hi_smem, cudaStream_t s) {
    return launch_batch_stages(bt, precision, sw, max_L, max_cap, slots, hi_grid, hi_smem, kDP5Stages + 1,
                               kMaxStages, s);
}

int launch_batch_step_sparsify(const BatchTable* bt, int max_cap, int slots, cudaStream_t s) {
    k_batch_sp_residual<<<dim3(max_cap > 13 ? max_cap - 12 : 1, slots), SP_RES_THREADS, 0, s>>>(bt);
    k_batch_sp_select<<<slots, CTL_THREADS, 0, s>>>(bt);
    k_batch_sp_compact<<<dim3(64, slots), 256, 0, s>>>(bt);
    k_batch_sp_finish<<<slots, CTL_THREADS, 0, s>>>(bt);
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}
