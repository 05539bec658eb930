// Internal declarations shared by the translation units of libdmfe.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/dmfe.h"
#include "df64.h"

#define DMFE_CUDA_TRY(call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return DMFE_ERR_CUDA;          \
    } while (0)

// 32-byte history element {C, dC/dt, R, dR/dt} (own type: CUDA 13 deprecates double4).
struct __align__(32) dbl4 {
    double x, y, z, w;
};

// Polynomial f(q), f'(q), f''(q) as dense Horner coefficients (kernel argument, so that
// solvers with different f can run concurrently in one process).
struct Poly {
    int deg0, deg1, deg2;                // degrees of f, f' and f''
    double a0[DMFE_MAX_POWER + 1];       // f(q)   = sum_m a0[m] q^m
    double a1[DMFE_MAX_POWER];           // f'(q)  = sum_m a1[m] q^m
    double a2[DMFE_MAX_POWER];           // f''(q) = sum_m a2[m] q^m
    float f1[DMFE_MAX_POWER];            // FP32 f' (also the hi part of the double-float f')
    float f2[DMFE_MAX_POWER];
    float g1[DMFE_MAX_POWER];            // lo parts: f' = f1 + g1 as a double-float
    float g2[DMFE_MAX_POWER];
};

// Double-float history element and stage-row element (32 bytes each).
struct __align__(32) df8 {
    df C, dC, R, dR;
};
struct __align__(32) dfrow {
    df K, D, C, R;
};
// B1 time interpolation of output index j for one stage: value at time theta_j t =
// w0 Y[a0] + w1 dY[a0] + w2 Y[a1] + w3 dY[a1] (a1 < 0: the stage row, w3 = 0).
struct __align__(16) B1Desc {
    int a0, a1;
    double w[4];
    df wd[4];
    double s;  // interior interval (a1 = a0 + 1): (theta_j t - t_a0) / (t_a1 - t_a0)
};

// Cubic Hermite interpolant of the history between slices k and k+1 (Sec. 3.3) in monomial
// form in s = (tau - t_k) / (t_{k+1} - t_k): C = c0 + s (c1 + s (c2 + s c3)), R alike.
// The FP64 kernel evaluates it by Horner's rule instead of forming four basis weights.
struct __align__(64) dbl8 {
    double c0, c1, c2, c3, r0, r1, r2, r3;
};

// Per-slice constants of one stage for the double-float kernel: complement
// v_k = (t - t_k)/t, inv_k = t/(t_{k+1} - t_k), h_k = t_{k+1} - t_k.
struct __align__(8) dfslice {
    df v, inv;
    float h;
    float pad;
};

template <typename R>
__device__ __forceinline__ R poly_eval(const R* a, int deg, R q) {
    R v = a[deg];
    for (int m = deg - 1; m >= 0; --m) v = fma(v, q, a[m]);
    return v;
}
__device__ __forceinline__ double fp0(const Poly& P, double q) { return poly_eval(P.a0, P.deg0, q); }
__device__ __forceinline__ double fp1(const Poly& P, double q) { return poly_eval(P.a1, P.deg1, q); }
__device__ __forceinline__ double fp2(const Poly& P, double q) { return poly_eval(P.a2, P.deg2, q); }
__device__ __forceinline__ float fp1(const Poly& P, float q) { return poly_eval(P.f1, P.deg1, q); }
__device__ __forceinline__ float fp2(const Poly& P, float q) { return poly_eval(P.f2, P.deg2, q); }

// f'(q) and f''(q) (FP32) at two points in one loop: the same Horner steps, in the same
// order, as four separate fp1 / fp2 calls (f'' has degree deg1 - 1, so f' takes one step
// more, peeled in front), with a quarter of the loop overhead and coefficient loads.
__device__ __forceinline__ void fp12_pair(const Poly& P, float qa, float qb, float& f1a, float& f2a, float& f1b,
                                          float& f2b) {
    const int d1 = P.deg1;
    f1a = f1b = P.f1[d1];
    if (d1 == 0) {
        f2a = f2b = P.f2[0];
        return;
    }
    f2a = f2b = P.f2[d1 - 1];
    f1a = fmaf(f1a, qa, P.f1[d1 - 1]);
    f1b = fmaf(f1b, qb, P.f1[d1 - 1]);
    for (int m = d1 - 2; m >= 0; --m) {
        const float c1 = P.f1[m], c2 = P.f2[m];
        f1a = fmaf(f1a, qa, c1);
        f2a = fmaf(f2a, qa, c2);
        f1b = fmaf(f1b, qb, c1);
        f2b = fmaf(f2b, qb, c2);
    }
}

// Step-control and history bookkeeping, resident in device memory. Kernels of the
// integrate loop read and update it; the host reads it only to poll and report.
struct DevState {
    double t;            // time of the last accepted slice
    double dt;           // controller step
    double h;            // size of the trial step in progress
    double t_stage;      // time of the stage being evaluated
    double t_target;     // integrate target
    double tol;
    double dt_min;
    double eps;          // eps_RK of the last trial step
    double mu, E;        // of the last stage row evaluated by the assemble kernel
    double max_eps_sparse;
    double t_pending;    // time of an accepted slice waiting for a sparsification pass
    long long steps_accepted, steps_rejected, stages;
    long long sparsify_passes, slices_removed, forced_removals;
    int n;               // stored slices in the active buffer
    int active;          // 0/1: which history buffer is live
    int status;          // 0 or a DMFE_ERR_* code
    int done;            // 1 once t reached t_target
    int pending;         // 1: an accepted slice waits for a sparsification pass
    int removed_count;   // slices removed by the last pass
    int sp_ran;          // 1 between the select and finish kernels of a pass
    int n_new;           // slice count after the pass
    int method;          // integrator of the next step: 0 Dormand-Prince 5(4), 1 SSPRK(10,4)
    int rk;              // integrator of the step in progress (set by its first kernel)
    int nst;             // its number of stage evaluations (6 or 10)
    int sp_left;         // sparsification passes left in the current round (set on accept)
    int bounds_site;     // checked builds: site code of the first failed bounds check (0: none)
    int pad_;
    double t_switch;     // time of the switch to SSPRK(10,4), -1 if none
};

constexpr int kMaxStages = 10;  // stage evaluations per step of the longest method
constexpr int kMaxSparsifyPasses = 8;  // passes per sparsification round (dmfe_params.sparsify_passes)
constexpr int kDP5Stages = 6;   // stage evaluations per Dormand-Prince step

#if defined(__CUDACC__)
// Bounds checks of the checked build (-DDMFE_CHECKED): every stencil base and history row
// index of the history-integral and sparsification kernels is tested before its access. A
// failed test records its site code in DevState::bounds_site (the first failure wins) and
// the access is skipped or made at an in-bounds index instead; nothing traps. Without
// DMFE_CHECKED the tests are `true`. Site codes: 1-5 FP64 kernel (B1 rows, A1, A2 and B2
// stencil bases, B2 interval), 11-15 FP32 kernel, 21-24 double-float kernel, 31-32
// sparsification (residual rows, compaction target).
#ifdef DMFE_CHECKED
__device__ __forceinline__ bool dmfe_in_bounds(DevState* st, bool ok, int site) {
    if (!ok) atomicCAS(&st->bounds_site, 0, site);
    return ok;
}
#define DMFE_IN_BOUNDS(st, cond, site) dmfe_in_bounds((st), (cond), (site))
#else
#define DMFE_IN_BOUNDS(st, cond, site) true
#endif

// Sparsification residual of one grid point (Sec. 3.6): the Hermite integrals over
// [t_{n-1}, t_n] and [t_n, t_{n+1}] minus the one over [t_{n-1}, t_{n+1}] without slice n,
// written as one linear form in the values y and derivatives d of slices n-1, n, n+1.
struct SpWeights {
    double ya, yb, yc, da, db, dc;
};
__host__ __device__ __forceinline__ SpWeights sp_weights(double h1, double h2) {
    const double h = h1 + h2;
    return SpWeights{-0.5 * h2, 0.5 * h, -0.5 * h1, (h1 * h1 - h * h) / 12.0, (h2 * h2 - h1 * h1) / 12.0,
                     (h * h - h2 * h2) / 12.0};
}
__device__ __forceinline__ double sp_delta(const SpWeights& w, double ya, double da, double yb, double db, double yc,
                                           double dc) {
    return fma(w.ya, ya, fma(w.yb, yb, fma(w.yc, yc, fma(w.da, da, fma(w.db, db, w.dc * dc)))));
}

// Gate of the kernels of stage `stage` (>= 1) of a step: they do nothing once the solve
// has stopped (error or target reached) or when the step's method has fewer stages.
// stage == 0 marks an explicit call outside the step loop (never gated).
__device__ __forceinline__ bool stage_off(const DevState* st, int stage) {
    return stage > 0 && (st->status != 0 || st->done || stage > st->nst);
}
#endif

// Everything a kernel needs about one solver (passed by value).
struct SolverView {
    int L, s, cap, precision;
    int sparsify;         // 1: round when the store is full
    int sp_every;         // > 0: a round after every sp_every-th accepted step
    int sp_passes;        // passes per round (>= 1)
    double rk_switch_dt;  // controller step of the switch to SSPRK(10,4) (+inf: never)
    int interp, fh_d;     // theta-stencil scheme (DMFE_INTERP_*) and Floater-Hormann degree
    int hi_threads;       // block size of a single solve's history-integral launch
    int log_r;            // 1: logarithmic interpolation of the response history
    double T, beta0;
    double gamma, ga, gD, alpha, delta;  // grid: gamma, atan(e^-gamma), atan(e^gamma) - atan(e^-gamma)
    Poly poly;
    const double* theta;  // [L]
    const double* omega;  // [L] 1 - theta
    const double* nu;     // [L]
    const float* omega32; // [L]
    const float* nu32;    // [L]
    const double* x1;     // [L*L] FP64 fractional index (only while dmfe_tables runs)
    const double* x2;
    const double* x3;
    const unsigned char* wt1;  // [L*L] FP64 path: stencil entries {int base, pad, s FP64
    const unsigned char* wt2;  //   weights} of 8 + 8 s bytes for phi1, phi2, psi
    const unsigned char* wt3;
    const uint32_t* p1;   // [L*L] fixed-point index, 19 fraction bits (FP32 path)
    const uint32_t* p2;
    const uint32_t* p3;
    double* ht[2];        // slice times [cap], two buffers (compaction ping-pong)
    dbl4* hist[2];        // [cap][L] {C, dC, R, dR} FP64 master
    float4* hist32[2];    // [cap][L] FP32 replica (FP32 path)
    df8* histdf[2];       // [cap][L] double-float replica (double-float path)
    dbl8* hcoef[2];       // [cap][L] FP64 path: row k = monomial coefficients of interval k
    dbl4* lcoef[2];       // [cap][L] log-R mode: the same for log R (x = NaN: R not positive)
    const df* q1;         // [L*L] double-float fractional index (double-float path)
    const df* q2;
    const df* q3;
    const df* omega_df;   // [L]
    const df* nu_df;      // [L]
    dfrow* rowdf;         // [L] stage row prepared for the double-float kernel
    dfslice* slicedf;     // [cap + 1] (entry n: the stage time, for a stage beyond the last slice)
    df8* vrowdf;          // [L] double-float path: virtual slice at the stage time (see prep)
    float4* vrow32;       // [L] FP32 path: the same in FP32
    dbl4* row64;          // [L] FP64 path: the stage row {K, D, C, R} (written by the prep kernel)
    double* slice64;      // [cap + 1] FP64 path: 1/(t_{k+1} - t_k) of each interval (prep kernel)
    float4* row32f;       // [L] FP32 path: the stage row {K, D, C, R} in FP32 (prep kernel)
    float4* slice32;      // [cap + 1] FP32 path: {(t - t_k)/t, t/(t_{k+1} - t_k), t_{k+1} - t_k, 0}
    int* cell;            // [L] slice of time theta_m t
    B1Desc* b1;           // [L] per-stage B1 time weights
    int hi_chunk;         // summation indices per work unit (-1: the flat split)
    const int2* flat_seg; // flat split: [G + 1] {first pair, its row} of each warp's segment
    const int2* flat_row; // flat split: [L] {first segment, segments} of each row
    DevState* st;
    double* Y;            // [2][2L] stage rows (C then R), double-buffered: stage stg reads
                          // Y + (stg & 1) * 2L and writes the other buffer
    double* mupart;       // [2][kMaxPrepBlocks] per-block partial sums of mu's and E's integrands
    double* epart;        // [kCtlGrid] per-CTA partial sums of the step error
    int* ctl_count;       // CTAs finished in the last stage of a step (zero between steps)
    double* k;            // [kMaxStages + 1][2L] stage derivatives
    double* ynew;         // [2L] 5th-order solution of the trial step
    double* S;            // [NS][L]
    double* Spart;        // [parts][9][L] partial sums of the chunks of the i-range
    int* jcount;          // [L] parts finished per output index (zero between launches)
    double* eps_sp;       // [cap] sparsification residuals
    int* keep;            // [cap]
    int* newidx;          // [cap]
};

// Batch table (device memory): the slots of a batch, read by the batched kernels of one
// captured step graph; the host rewrites it between graph launches when slots change.
constexpr int kMaxSlots = 256;
struct BatchTable {
    int count;                      // slots 0 .. count-1 are examined
    int pad;
    long long uoff[kMaxSlots + 1];  // history-integral unit offsets (0 units: idle slot)
    long long woff[kMaxSlots + 1];  // work (pair) offsets: CTAs split the batch by work
    long long woff_late[kMaxSlots + 1];  // the same over the slots whose step runs more than
                                         // kDP5Stages stages (written on the device by the
                                         // first kernel of every batched step)
    int active[kMaxSlots];          // 1: slot holds a solver
    SolverView views[kMaxSlots];
};

static const int FIX_FRAC_BITS = 19;  // x = packed / 2^19
constexpr int kPrepThreads = 128;     // block size of the per-stage prep kernel
constexpr int kMaxPrepBlocks = (8192 + kPrepThreads - 1) / kPrepThreads;
constexpr int kCtlThreads = 256;      // block size of the multi-CTA stage kernels
constexpr int kCtlGrid = 64;          // their maximal grid

// ---- launchers (defined in the .cu files) ----
int launch_tables(const SolverView& v, cudaStream_t s);
// history integrals: row_dev = [2L] (C, R); t_dev != NULL reads the stage time from
// device memory (integrate loop) and gates on the status word; otherwise uses t.
int launch_history_integrals(const SolverView& v, const double* row_dev, double t, int stage,
                             double* S_dev, int grid_ctas, cudaStream_t s);
// grid and block size (stored in v.hi_threads) of a single solve's history-integral launch
int hi_config(SolverView& v, int* grid_ctas, size_t* smem);
int hi_launch_shape(long long units, int nsm, int max_warps, int* warps);
int launch_assemble(const SolverView& v, const double* row_dev, const double* S_dev, double t,
                    double* dC, double* dR, double* muE, cudaStream_t s);
// one trial step: head = begin + stages 1..kDP5Stages, tail = the later stages (SSPRK),
// then the sparsification kernels; launch_step issues all three
int launch_step(const SolverView& v, int grid_ctas, cudaStream_t s);
int launch_step_head(const SolverView& v, int grid_ctas, cudaGraphConditionalHandle cond, int use_cond,
                     cudaStream_t s);
int launch_step_tail(const SolverView& v, int grid_ctas, cudaStream_t s);
int launch_step_sparsify(const SolverView& v, cudaStream_t s);
int launch_begin_integrate(const SolverView& v, double t_target, double tol, cudaStream_t s);
int launch_initial_slice(const SolverView& v, cudaStream_t s);
int launch_sparsify(const SolverView& v, bool from_step, double tol, cudaStream_t s);
int launch_lookup(const SolverView& v, int n, const double* t, const double* tp, int which,
                  double* out, cudaStream_t s);
int launch_refresh_replica(const SolverView& v, cudaStream_t s);
// per-stage preparation for every precision (kernels_df.cu)
int launch_stage_prep(const SolverView& v, const double* row_dev, double t, int stage, cudaStream_t s);
// double-float path (kernels_df.cu)
int launch_history_integrals_df(const SolverView& v, const double* row_dev, double t, int stage,
                                double* S_dev, int grid_ctas, cudaStream_t s);
int hi_config_df(SolverView& v, int* grid_ctas, size_t* smem);

// ---- batched execution (batch.cu and the kernel files) ----
int batch_hi_config(int precision, int sw, int max_L, int max_cap, int* grid_ctas, size_t* smem);
int batch_hi_config_df(int sw, int max_L, int max_cap, int* grid_ctas, size_t* smem);
int launch_batch_hi(const BatchTable* bt, int precision, int sw, int stg, int grid, size_t smem, cudaStream_t s);
int launch_batch_hi_df(const BatchTable* bt, int sw, int stg, int grid, size_t smem, cudaStream_t s);
int launch_batch_prep(const BatchTable* bt, int stg, int max_tot, int slots, cudaStream_t s);
int launch_batch_step_head(const BatchTable* bt, int precision, int sw, int max_L, int max_cap, int slots,
                           int hi_grid, size_t hi_smem, cudaGraphConditionalHandle cond, int use_cond,
                           cudaStream_t s);
int launch_batch_step_tail(const BatchTable* bt, int precision, int sw, int max_L, int max_cap, int slots,
                           int hi_grid, size_t hi_smem, cudaStream_t s);
int launch_batch_step_sparsify(const BatchTable* bt, int max_cap, int slots, cudaStream_t s);

// Capture one step into an executable graph on stream `cap`: head(cond, use_cond, stream),
// then tail(stream) inside a conditional IF node that the head's first kernel enables
// (if `conditional`; otherwise inline), then sp(stream). (graph.cu)
struct StepParts {
    virtual int head(cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) = 0;
    virtual int tail(cudaStream_t s) = 0;
    virtual int sp(cudaStream_t s) = 0;
    virtual ~StepParts() = default;
};
int capture_step_graph(cudaStream_t cap, bool conditional, StepParts& parts, cudaGraphExec_t* out);
bool step_graph_plain();  // DMFE_STEP_GRAPH=plain: no conditional nodes (graph.cu)
// accessors of a solver's internals (api.cu)
struct dmfe_solver;
const SolverView& solver_view(const dmfe_solver* h);
void solver_set_chunk(dmfe_solver* h, int chunk);  // a batch slot's work-unit size
int solver_read_state(dmfe_solver* h, DevState* out);

// ---- host grid (host_grid.cpp) ----
double host_gamma_from_tmax(double t_max);
void host_theta_grid(int L, double gamma, double alpha, double delta, std::vector<double>& theta,
                     std::vector<double>& omega);
int host_spline_weights(const std::vector<double>& theta, std::vector<double>& nu);
