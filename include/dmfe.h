/*
 * dmfe.h -- C ABI of libdmfe.so, a GB300 (sm_103a) solver for the causal history
 * integrals of the spherical mixed p-spin dynamical mean-field equations on the
 * non-uniform two-time grid (DYNAMITE, arXiv 2604.06309).
 *
 * Fields are stored on the grid (t_n, theta_i t_n): Cf(t, theta) = C(t, theta t),
 * Rf(t, theta) = R(t, theta t) (Sec. 3.1). theta_i, i = 0..L-1, is the fixed grid of
 * Eq. (theta) (Sec. 3.2); t_n are the slices accepted by the adaptive Runge-Kutta
 * integrator (Dormand-Prince 5(4), then SSPRK(10,4); Sec. 3.5), thinned by
 * sparsification (Sec. 3.6).
 *
 * Conventions for every entry point:
 *  - Return value: DMFE_OK (0) or a negative DMFE_ERR_* code; dmfe_strerror maps it
 *    to text. A failed call leaves the solver at its last accepted slice, readable.
 *  - Pointers named *_dev are device pointers; every other pointer is host memory,
 *    owned by the caller, read or written only during the call.
 *  - Rows are double arrays of length L in grid order (theta ascending). Histories
 *    are row-major [n][L].
 *  - One solver must not be used from two host threads at once; distinct solvers
 *    are independent. The library's only global state besides the CUDA context is a
 *    mutex-guarded cache of stencil tables: solvers on one device with the same grid,
 *    stencil and precision share one read-only copy (reference-counted; freed with the
 *    last of them), and a solver's stream waits for the kernel that built the copy.
 *  - The solver owns all its device memory; dmfe_destroy frees it.
 */
#ifndef DMFE_H
#define DMFE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define DMFE_OK                  0
#define DMFE_ERR_ARG            -1  /* invalid argument or size                        */
#define DMFE_ERR_OOM            -2  /* device or host allocation failed                 */
#define DMFE_ERR_NONFINITE      -3  /* NaN/Inf in the step error estimate               */
#define DMFE_ERR_STEP_UNDERFLOW -4  /* step below dt_min: the run ends (App. B)         */
#define DMFE_ERR_CAPACITY       -5  /* history full and sparsification disabled         */
#define DMFE_ERR_CUDA           -6  /* a CUDA runtime call failed                       */
#define DMFE_ERR_TIMEOUT        -7  /* a bounded device wait gave up                    */
#define DMFE_ERR_UNSUPPORTED    -8  /* valid but not implemented (e.g. stencil width)   */
#define DMFE_ERR_IO             -9  /* checkpoint file could not be written or read     */

/* ---- precision of the history-integral bulk -------------------------------- */
#define DMFE_FP64              0  /* everything in FP64                                 */
#define DMFE_FP32_COMPENSATED  1  /* interpolation and sums in FP32 with compensated
                                     (Kahan) accumulation over an FP32 history replica;
                                     times, theta, mu, the RK error, step control and
                                     the sparsification test stay FP64                 */

#define DMFE_DOUBLE_FLOAT      2  /* interpolation and sums in double-float arithmetic (pairs of
                                     FP32 numbers, 48-bit significand, ~1e-13 relative) on the
                                     FP32 pipes over a double-float history replica; FP64 for
                                     everything else. FP64-class results at FP32-pipe speed */

/* ---- theta interpolation (Sec. 3.3) ------------------------------------------- */
#define DMFE_INTERP_LAGRANGE_INDEX 0  /* Lagrange in the grid index (default)                  */
#define DMFE_INTERP_FH_INDEX       1  /* Floater-Hormann rational, blending degree fh_d, index  */
#define DMFE_INTERP_LAGRANGE_THETA 2  /* Lagrange on the theta values of the stencil nodes      */
#define DMFE_INTERP_FH_THETA       3  /* Floater-Hormann on the theta values                    */

/* ---- integrator (Sec. 3.5) ---------------------------------------------------- */
#define DMFE_RK_AUTO      0  /* Dormand-Prince 5(4) until the controller step reaches the
                                switch step, then SSPRK(10,4) with the step halved (default) */
#define DMFE_RK_DP5       1  /* Dormand-Prince 5(4) throughout                               */
#define DMFE_RK_SSPRK104  2  /* SSPRK(10,4) throughout                                       */

#define DMFE_NS 10   /* rows of the history-integral output S, see dmfe_history_integrals */
#define DMFE_MAX_TERMS 16
#define DMFE_MAX_POWER 24

typedef struct dmfe_solver dmfe_solver;

/* Problem and numerical parameters (Secs. 2.1, 3.2, 3.5, 3.6). */
typedef struct {
    int           n_terms;      /* f(q) = sum_k coefs[k] q^powers[k], 1 <= n_terms <= 16   */
    const int*    powers;       /* 1 <= powers[k] <= 24; copied at create                  */
    const double* coefs;        /* copied at create                                        */
    double        T;            /* bath temperature                                        */
    double        beta0;        /* inverse temperature of the initial state (0: random)   */
    int           L;            /* theta-grid length, 16 <= L <= 8192                      */
    int           s;            /* theta stencil width: 4, 6, 8 or 10                      */
    double        grid_t_max;   /* t_max of Eq. (theta): gamma = -W_{-1}(-1/grid_t_max) > 1 */
    double        alpha, delta; /* trade-off parameters of Eq. (theta) (default 0, 0)      */
    int           history_cap;  /* stored slices, >= 16 (default L)                        */
    double        dt0, dt_min;  /* initial and minimal step (defaults 1e-4, 1e-12)         */
    int           precision;    /* DMFE_FP64, DMFE_FP32_COMPENSATED or DMFE_DOUBLE_FLOAT   */
    int           sparsify;     /* 1: sparsification round whenever the store is full (default);
                                   0: off (a full store ends the run with DMFE_ERR_CAPACITY;
                                   sparsify_every rounds still run)                       */
    void*         stream;       /* cudaStream_t for all work; NULL: the solver's own stream */
    int           integrator;   /* DMFE_RK_AUTO (default), DMFE_RK_DP5 or DMFE_RK_SSPRK104  */
    double        rk_switch_dt; /* DMFE_RK_AUTO: controller step at which SSPRK(10,4) takes
                                   over; 0 (default): beta_DP / (4 sqrt(f''(1))), the step at
                                   which Dormand-Prince 5 (real stability interval beta_DP =
                                   3.3066) reaches the spectral bound ||J|| <= 4 sqrt(f''(1))
                                   of Sec. 3.5; no switch when f''(1) <= 0              */
    int           hi_chunk;     /* summation indices per work unit of the history-integral
                                   kernel, >= 32; -1: the flat split (the L^2 pairs cut into one
                                   equal segment per warp of the launch, so every SM gets the
                                   same work; single solves with L >= 512 and at least 256
                                   pairs per warp, else as 0); 0 (default): the flat split
                                   where it applies, else chosen from L and the precision, for
                                   a single solve; L for a batch slot (a batch slot given -1
                                   or 0 takes L). Changes only the summation order (see
                                   dmfe_autotune)                                         */
    int           interp;       /* DMFE_INTERP_*: the theta-stencil scheme (default Lagrange in
                                   the index). The other schemes need DMFE_FP64 (their
                                   weights live in the FP64 stencil tables); otherwise
                                   dmfe_create returns DMFE_ERR_UNSUPPORTED              */
    int           fh_d;         /* Floater-Hormann blending degree, 0 <= fh_d <= s-1
                                   (default 3; fh_d = s-1 is the polynomial interpolant)  */
    int           log_r;        /* 1: interpolate the response history in log R (with the
                                   scaled derivative R'/R) wherever the stencil's values
                                   are positive, linearly elsewhere (App. A); DMFE_FP64
                                   single solves only (else DMFE_ERR_UNSUPPORTED from
                                   dmfe_create, dmfe_batch_add, dmfe_server_submit).
                                   Default 0                                              */
    int           sparsify_every; /* P > 0: a sparsification round also after every P-th
                                   accepted step (after its slice is appended), besides the
                                   rounds on a full store; 0 (default): full store only.
                                   Such a round never forces a removal (Sec. 3.6)          */
    int           sparsify_passes; /* passes per round, 1..8 (0 counts as 1; default 1): the
                                   user's control of the degree of sparsification (Sec. 3.6,
                                   last paragraph). Each pass repeats the scan on the history
                                   the previous pass left. On a full store the first pass may
                                   force a removal and the accepted slice is appended after
                                   it, before the further passes. Batch slots and served
                                   requests take 1 (else DMFE_ERR_UNSUPPORTED)              */
} dmfe_params;

/* Per-solve counters. */
typedef struct {
    double    t;                 /* time of the last accepted slice           */
    double    dt;                /* current controller step                   */
    double    mu, E;             /* mu(t) and E(t) of the last slice (Sec. 2.1) */
    double    last_eps;          /* eps_RK of the last trial step (Sec. 3.5)  */
    double    max_eps_sparse;    /* largest eps_sparse of a removed slice     */
    long long steps_accepted, steps_rejected, stages;
    long long sparsify_passes, slices_removed, forced_removals;
    int       n_slices;          /* stored slices                             */
    int       status;            /* device status word (0 or DMFE_ERR_*)      */
    int       L, history_cap;    /* sizes fixed at create                     */
    int       s, precision;
    int       method;            /* integrator of the next step: DMFE_RK_DP5 or DMFE_RK_SSPRK104 */
    double    t_switch;          /* time of the switch to SSPRK(10,4), -1 if none   */
    double    rk_switch_dt;      /* switch step in force (+inf: none)                */
    int       step_graph;        /* 0: no step graph yet; 1: all stages inline (the SSPRK
                                    ones gate themselves off in Dormand-Prince steps);
                                    2: SSPRK stages in a conditional graph node        */
    int       bounds_site;       /* library built with -DDMFE_CHECKED (libdmfe_checked.so):
                                    site code of the first stencil-base or history-row
                                    index that failed its bounds check (the access was
                                    skipped or made in bounds instead); 0 otherwise     */
} dmfe_stats_t;

/* Fill p with defaults for the given f (pointers are kept, not copied). */
void dmfe_default_params(dmfe_params* p);

const char* dmfe_strerror(int code);

/* Create a solver: builds the theta grid and nu (host, FP64), the stencil tables on
 * the device (kernel a), allocates the history at history_cap slices and stores the
 * initial slice t = 0, Cf = Rf = 1 with its derivative. Returns DMFE_ERR_ARG for
 * parameters outside the ranges above, DMFE_ERR_UNSUPPORTED for other stencil widths. */
int  dmfe_create(const dmfe_params* p, dmfe_solver** out);
void dmfe_destroy(dmfe_solver* h);

/* Grid of Eq. (theta) and the quadrature weights nu of Sec. 3.4 (host arrays of L). */
int dmfe_grid(dmfe_solver* h, double* theta, double* omega, double* nu);

/* The same grid without a solver or a device (host code only): theta_i of Eq. (theta)
 * for gamma = -W_{-1}(-1/grid_t_max) and the trade-offs alpha, delta; omega_i = 1 -
 * theta_i computed without cancellation; nu_i of Sec. 3.4. Caller-owned host arrays of L
 * (any may be NULL). DMFE_ERR_ARG for L outside [16, 8192], grid_t_max <= e, alpha outside
 * [0, 1] or delta < 0 (the ranges of dmfe_params). */
int dmfe_theta_grid(int L, double grid_t_max, double alpha, double delta, double* theta, double* omega,
                    double* nu);

/* Fractional stencil positions of kernel (a), FP64, [L][L] each, row j = output index:
 * x1 for phi1 = theta_i theta_j, x2 for phi2 = theta_j + (1 - theta_j) theta_i,
 * x3 for psi = theta_j / phi2 (Sec. 3.3). Any pointer may be NULL. */
int dmfe_tables(dmfe_solver* h, double* x1, double* x2, double* x3);

/* Advance with the adaptive integrator of dmfe_params.integrator to t_max <= grid_t_max
 * with tolerance tol (Secs. 3.1, 3.5, 3.6). Step control, including the switch from
 * Dormand-Prince to SSPRK(10,4), runs on the device; the host polls a status word.
 * Returns DMFE_ERR_STEP_UNDERFLOW, DMFE_ERR_NONFINITE or DMFE_ERR_CAPACITY when the device
 * stops the run; the solver then holds the last accepted slice. */
int dmfe_integrate(dmfe_solver* h, double t_max, double tol);

/* Launch exactly nsteps trial steps toward t_max with tolerance tol on the solver's
 * stream (or `stream` if not NULL) without synchronising: each step is one CUDA-graph
 * launch of the stages (the last four stages of SSPRK(10,4) sit in a conditional graph
 * node that the step's first kernel enables), the device-side step rule and, when the
 * store is full, a sparsification pass. The environment variable DMFE_STEP_GRAPH=plain
 * (read when a solver or batch first captures its graph) keeps every stage inline
 * instead, for profilers that cannot attribute kernels inside conditional graphs. Steps after t_max is reached or after a device error
 * do nothing. dmfe_sync / dmfe_stats read the outcome. Used by benchmarks and by
 * callers that interleave their own work between steps. */
int dmfe_step(dmfe_solver* h, int nsteps, double t_max, double tol, void* stream);

/* Two-time functions at n points (t[k], tp[k]), both <= the current time:
 * C is symmetric; R(t, t') = 0 for t' > t (causality, Sec. 2.2). Cubic Hermite in t
 * between stored slices and the theta stencil at t_small/t_big (Sec. 3.3). */
int dmfe_get_C(dmfe_solver* h, int n, const double* t, const double* tp, double* out);
int dmfe_get_R(dmfe_solver* h, int n, const double* t, const double* tp, double* out);

/* Last accepted slice: time, rows Cf, Rf (length L, may be NULL), mu(t), E(t). */
int dmfe_get_row(dmfe_solver* h, double* t, double* C, double* R, double* mu, double* E);

/* Replace the stored history by n slices (1 <= n <= history_cap): times t[n] with
 * t[0] = 0 strictly increasing, rows C, dC, R, dR [n][L] (dC, dR: d/dt at fixed theta).
 * Used for frozen-history benchmarks and parity tests. */
int dmfe_set_history(dmfe_solver* h, int n, const double* t, const double* C,
                     const double* dC, const double* R, const double* dR);
/* Copy the stored history out; *n receives the slice count, arrays must hold
 * history_cap slices (any array may be NULL). */
int dmfe_get_history(dmfe_solver* h, int* n, double* t, double* C, double* dC,
                     double* R, double* dR);

/* The history integrals of one Runge-Kutta stage (Secs. 3.3, 3.4, Eq. int) at time
 * t >= t_last for the stage row (C_row, R_row) over the stored history, and mu(t)
 * (Sec. 2.1). Output S is [DMFE_NS][L]; with t' = theta_j t and the interpolated
 * values A (current row at phi1 or phi2), B1 = (C, R)(theta_j t, theta_i),
 * B2 = (C, R)(phi2 t, theta_j/phi2):
 *   S[0] = sum_i nu_i K_A1 C_B1   S[1] = sum nu K_A2 C_B2   S[2] = sum nu D_A1 R_B1
 *   S[3] = sum nu K_A2 R_B2       S[4] = sum nu f''(C_B1) R_B1 C_A1
 *   S[5] = sum nu f'(C_B1) R_A1   S[6] = sum nu f'(C_B2) R_A2
 *   S[7] = sum nu f''(C_B2) R_B2 R_A2
 *   S[8] = sum nu [f''(C_B1) C_B1 + f'(C_B1)] R_B1   S[9] = C(theta_j t, 0)
 * (K = f''(C) R, D = f'(C)). Times in (t_last, t] use the quadratic through the last
 * slice and the stage row. mu may be NULL. Host pointers; synchronous. */
int dmfe_history_integrals(dmfe_solver* h, double t, const double* C_row, const double* R_row,
                           double* S, double* mu);
/* Same on device memory, stream-ordered on `stream` (NULL: the solver's stream):
 * row_dev is [2][L] (C then R), S_dev is [DMFE_NS][L]. Does not synchronise. */
int dmfe_history_integrals_dev(dmfe_solver* h, double t, const double* row_dev,
                               double* S_dev, void* stream);

/* Right-hand side of the theta-grid ODE for a stage (t, C_row, R_row): the total
 * derivatives dCf/dt, dRf/dt at fixed theta (d1 + theta d2, with d2 from the DMFE's
 * second-argument equations), theta = 1 pinned to 0; mu(t), E(t). Host pointers. */
int dmfe_rhs(dmfe_solver* h, double t, const double* C_row, const double* R_row,
             double* dC, double* dR, double* mu, double* E);

/* One sparsification pass (Sec. 3.6) on the stored history with tolerance tol, as
 * dmfe_integrate runs it when the store is full. removed (may be NULL, size
 * history_cap) receives 1 for each slice index that was removed. The candidates are
 * slices 1 .. n-12, so with n <= 12 stored slices nothing is removed (DMFE_OK). */
int dmfe_sparsify(dmfe_solver* h, double tol, int* removed);

int dmfe_stats(dmfe_solver* h, dmfe_stats_t* out);

/* Binary checkpoint (parameters, grid key, history, step-control state, counters);
 * a restored solver continues bit-identically. stream as in dmfe_params. */
int dmfe_checkpoint(dmfe_solver* h, const char* path);
int dmfe_restore(const char* path, void* stream, dmfe_solver** out);

/* Autotune the work-unit size of the history-integral kernel (summation indices per
 * unit: the candidates 32, 64, ..., 4096, L and L/P for P = 2..16, at least 32, and the flat
 * split -1 where it applies) by timing the kernel on the solver's current history and
 * stage row, and keep the fastest. Results are cached per
 * (L, history_cap, s, precision) for the process. Changes the summation order of the
 * sums S (rounding-level differences only). *chunk (may be NULL) receives the choice. */
int dmfe_autotune(dmfe_solver* h, int* chunk);

/* Synchronise the solver's stream and return the device status word. */
int dmfe_sync(dmfe_solver* h);

/* ---- batched and served solves ------------------------------------------------------
 * A batch runs many independent solves (one per slot) with one CUDA graph per
 * Runge-Kutta step (slots may be in Dormand-Prince or SSPRK(10,4) steps; the stages beyond
 * the sixth run only for the latter): each stage is one persistent history-integral launch
 * over the units of every active slot (the slots may have different L, history caps, f, T,
 * t_max and integrators), plus batched control kernels. Slots read a batch table in device memory, so
 * slots can be added and removed between steps without re-capturing the graph
 * (continuous batching). A slot's results are bitwise identical to the same solve run
 * alone with the same work-unit size. All slots share the batch's precision and stencil
 * width. Every solve owns its device memory; a slot is a dmfe_solver. */
typedef struct dmfe_batch dmfe_batch;
/* max_slots <= 256; max_L, max_cap bound the slots' L and history_cap (they size the
 * shared-memory tables of the batched kernels). stream as in dmfe_params. */
int dmfe_batch_create(int max_slots, int max_L, int max_cap, int precision, int s, void* stream,
                      dmfe_batch** out);
void dmfe_batch_destroy(dmfe_batch* b);
/* Admit a solve into a free slot: creates its solver (allocates; synchronous), targets
 * t_max with tolerance tol. *slot receives the slot. DMFE_ERR_CAPACITY: no free slot;
 * DMFE_ERR_ARG: parameters outside the batch's bounds or precision/stencil mismatch;
 * DMFE_ERR_UNSUPPORTED: log_r set (log-R interpolation is for single solves). */
int dmfe_batch_add(dmfe_batch* b, const dmfe_params* p, double t_max, double tol, int* slot);
/* Release a slot (synchronises, frees its solver). */
int dmfe_batch_remove(dmfe_batch* b, int slot);
/* The solver of a slot (NULL if free), for dmfe_get_C/R, dmfe_get_row, dmfe_stats. */
dmfe_solver* dmfe_batch_solver(dmfe_batch* b, int slot);
/* Launch nsteps batched steps on the batch stream without synchronising. */
int dmfe_batch_step(dmfe_batch* b, int nsteps);
/* Synchronise and read every slot: status[k] (0, DMFE_ERR_*, or 1 = reached t_max; -100
 * for a free slot) and t[k] (arrays of max_slots, may be NULL). Finished and failed slots
 * stop receiving work. *running receives the number of slots still integrating. */
int dmfe_batch_poll(dmfe_batch* b, int* status, double* t, int* running);

/* Autotuner of the batched history-integral kernel's work units (the batch form of
 * dmfe_autotune; the paper has no counterpart). Tries the unit sizes 0 (one unit per output
 * index, the default), 256, 512, 1024 and 2048 summation indices (a size >= a slot's L means
 * one unit per index there) on every slot of the batch, each for `steps` real batched steps,
 * in two interleaved rounds, and keeps the one with the smallest device time per step for
 * all slots. The timed steps advance the solves, and changing a slot's unit size changes
 * the summation order of its sums (rounding-level differences), so tune on a batch whose
 * results are not kept, or before results matter; a fresh batch whose slots are added with
 * dmfe_params.hi_chunk = *chunk (0: leave 0) then runs bitwise like solo solves with that
 * unit size. *chunk (may be NULL) receives the choice and ms_per_step (may be NULL, 5
 * entries) the best time per step of each candidate. Synchronous. */
#define DMFE_BATCH_TUNE_CANDIDATES 5
int dmfe_batch_autotune(dmfe_batch* b, int steps, int* chunk, double* ms_per_step);

/* Device bytes a solver with these parameters allocates (dmfe_create), rounded up the way
 * large device allocations are; used for admission by footprint. 0 on invalid input. An
 * upper bound: the stencil tables (three [L][L] arrays, the bulk of the footprint in FP64)
 * are shared by every solver on the device with the same grid (L, grid_t_max, alpha, delta),
 * stencil (s, interp, fh_d) and precision, and are allocated only by the first of them. */
unsigned long long dmfe_footprint(const dmfe_params* p);

/* A serving loop over a batch (continuous batching): a host worker thread admits queued
 * requests first-in first-out into free slots while the summed footprint stays within
 * hbm_budget bytes, steps the batch steps_per_round steps at a time, and retires every
 * solve that reaches its t_max or fails, recording its latency. */
typedef struct dmfe_server dmfe_server;
typedef struct {
    long long id;
    int       status;                  /* 0: reached t_max; < 0: DMFE_ERR_* of the solve    */
    int       slot;
    double    t_final, E, mu;          /* last slice: time, energy, Lagrange multiplier     */
    double    submit_s, admit_s, done_s; /* seconds since the server started               */
    long long steps_accepted, steps_rejected;
} dmfe_result;
typedef struct {
    long long submitted, admitted, completed, failed;
    int       queued, running;
    unsigned long long bytes_in_use, hbm_budget;
    long long batched_steps;
} dmfe_server_stats_t;
int dmfe_server_start(int max_slots, int max_L, int max_cap, int precision, int s,
                      unsigned long long hbm_budget, int steps_per_round, dmfe_server** out);
/* Queue a request (parameters copied; thread-safe). *id receives its id. DMFE_ERR_ARG if
 * it can never be admitted (bounds, precision, footprint above the budget);
 * DMFE_ERR_UNSUPPORTED for log_r (as dmfe_batch_add). */
int dmfe_server_submit(dmfe_server* srv, const dmfe_params* p, double t_max, double tol, long long* id);
/* Move up to max_out finished results into out (thread-safe); *n receives the count. */
int dmfe_server_poll(dmfe_server* srv, dmfe_result* out, int max_out, int* n);
int dmfe_server_stats(dmfe_server* srv, dmfe_server_stats_t* out);
/* Stop the worker (running solves are abandoned) and free everything. */
int dmfe_server_stop(dmfe_server* srv);

/* ---- measurement ------------------------------------------------------------------
 * The paper has no counterpart: a measurement utility for the arithmetic rooflines of
 * the history-integral kernels (FP64 kernel: FP64 pipe; double-float and FP32 kernels:
 * FP32 pipes). Measures the fused multiply-add rate of the current device in FP64
 * (bits = 64) or FP32 (bits = 32): independent FMA chains on four 256-thread CTAs per SM,
 * one launch sized to about 80 ms, timed with CUDA events on a private stream, best of
 * three; *gflops receives the rate in GFLOP/s (an FMA counts 2). Synchronous; allocates
 * and frees a small output buffer; changes no clock or other setting of the GPU.
 * DMFE_ERR_ARG for other bit widths or a NULL pointer, DMFE_ERR_OOM, DMFE_ERR_CUDA. */
int dmfe_fma_rate(int bits, double* gflops);

/* ---- allocation-free entry point -------------------------------------------------
 * The paper has no counterpart: this serves callers of the library that cannot call
 * cudaMalloc -- processes whose device memory another framework has reserved up front,
 * and latency-critical loops that cannot afford the synchronisation an allocation may
 * imply. Such callers have no dmfe_solver (creating one allocates).
 *
 * Computes the same decision as dmfe_sparsify (greedy remove-n-skip-n+1 with tolerance
 * tol, forced removal of the smallest residual when none qualifies) for a history held
 * by the caller in device memory: t_dev [n] slice times (t[0] = 0, increasing) and
 * C_dev, dC_dev, R_dev, dR_dev row-major [n][L]. removed_dev [n] (device) receives 1 for
 * each slice to remove, else 0. The candidates are slices 1 .. n-12 (the first slice, the
 * last one and the ten-slice rollback window are kept), so for n <= 12 nothing is removed
 * and DMFE_OK is returned -- as dmfe_sparsify does for such a history. Stream-ordered on
 * `stream` (NULL: the legacy default stream); it does not synchronise. Nothing is
 * allocated: the residuals go to one fixed device array of DMFE_NOALLOC_MAX_SLICES doubles
 * that every GPU loading the library holds until exit. A call looks up that array's
 * device address (with the device current) unless `stream` is capturing, in which case it
 * uses the address found by an earlier call on the same device: make one call on each
 * device before capturing one (and again after a device reset). All calls share the array
 * and it keeps the last call's contents (every value a call reads is written earlier in
 * the same call), so calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised.
 * Returns DMFE_ERR_ARG for NULL pointers, n < 1, L < 1, tol <= 0 or
 * n > DMFE_NOALLOC_MAX_SLICES; DMFE_ERR_UNSUPPORTED for a device ordinal >= 64;
 * DMFE_ERR_CUDA if the address lookup or a launch fails, or if the first call on a device
 * is made while capturing. */
#define DMFE_NOALLOC_MAX_SLICES 16384
int dmfe_sparsify_select_noalloc(const double* t_dev, const double* C_dev, const double* dC_dev,
                                 const double* R_dev, const double* dR_dev, int n, int L,
                                 double tol, int* removed_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DMFE_H */
