// Host side of the C ABI declared in include/dmfe.h: solver lifecycle, the integrate
// loop (one CUDA graph per Runge-Kutta step, step control and the choice of method on
// the device, the host polls a status word), lookups and checkpoint/restore.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "dmfe_internal.h"
#include "hi_units.h"

struct dmfe_solver {
    dmfe_params p{};
    std::vector<int> powers;
    std::vector<double> coefs;
    std::vector<double> theta, omega, nu;
    SolverView v{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture the step graph
    cudaGraphExec_t step_exec = nullptr;
    bool conditional_graph = false;  // the step graph holds the SSPRK stages in an IF node
    int hi_grid = 0;
    size_t hi_smem = 0;
    DevState* hstate = nullptr;  // pinned mirror of the device state
    double* scratch = nullptr;   // device [4L + 16]
    std::vector<void*> allocs;
    std::vector<int2> flat_seg_h, flat_row_h;  // tables of the flat split (host copies)
    int flat_G = 0;              // warps the device tables were built for (0: none)
    bool table_ref = false;      // holds a reference to a cached stencil-table entry
    std::tuple<int, int, int, int, int, int, double, double, double> table_key;
};

namespace {

int dev_alloc(dmfe_solver* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return DMFE_ERR_OOM;
    }
    h->allocs.push_back(*p);
    return DMFE_OK;
}

// ---- stencil tables shared by solvers with the same key ------------------------------
// The stencil tables (FP64 weight entries, double-float positions or FP32 fixed-point
// positions for phi1, phi2 and psi) depend only on the device, the precision, the grid
// (L, gamma, alpha, delta) and the stencil (s, scheme, Floater-Hormann degree), so solvers
// that agree on all of them -- the members of a sweep over T and f at one grid -- share one
// copy. Entries are reference-counted (freed with their last solver) and carry an event
// recorded after the table kernel: a solver that finds an entry orders its stream after it.
using TableKey = std::tuple<int, int, int, int, int, int, double, double, double>;
struct TableEntry {
    void* t[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ready = nullptr;
    int refs = 0;
};
std::mutex g_table_mutex;
std::map<TableKey, TableEntry> g_tables;

void release_tables(dmfe_solver* h);

// The flat split's segment and row tables for a launch of `grid` CTAs of v.hi_threads
// threads (rebuilt only when the warp count changes); stream-ordered before any launch.
int set_flat_tables(dmfe_solver* h, int grid) {
    SolverView& v = h->v;
    const int G = grid * (v.hi_threads / 32);
    if (G == h->flat_G) return DMFE_OK;
    flat_split_tables(v.L, G, h->flat_seg_h, h->flat_row_h);
    void* p = nullptr;
    int rc = dev_alloc(h, &p, h->flat_seg_h.size() * sizeof(int2));
    if (rc) return rc;
    v.flat_seg = (const int2*)p;
    rc = dev_alloc(h, &p, h->flat_row_h.size() * sizeof(int2));
    if (rc) return rc;
    v.flat_row = (const int2*)p;
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.flat_seg, h->flat_seg_h.data(), h->flat_seg_h.size() * sizeof(int2),
                                  cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.flat_row, h->flat_row_h.data(), h->flat_row_h.size() * sizeof(int2),
                                  cudaMemcpyHostToDevice, h->stream));
    h->flat_G = G;
    return DMFE_OK;
}

// The solver's three stencil tables: an existing entry of its key (its stream then waits
// for the entry's table kernel), or a new entry built by the table kernel on the solver's
// stream. Lookup and build are one critical section, so an entry is visible only once its
// kernel and event are queued. Run after the grid arrays have been queued on the stream.
int acquire_tables(dmfe_solver* h, size_t fp64_table_bytes) {
    SolverView& v = h->v;
    const int L = v.L;
    const size_t LL = (size_t)L * L;
    const dmfe_params& pin = h->p;
    int dev = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    h->table_key = TableKey(dev, v.precision, L, v.s, v.interp,
                            (v.interp == DMFE_INTERP_FH_INDEX || v.interp == DMFE_INTERP_FH_THETA) ? v.fh_d : 0,
                            v.gamma, pin.alpha, pin.delta);
    const size_t tb = v.precision == DMFE_FP64 ? fp64_table_bytes
                      : (v.precision == DMFE_FP32_COMPENSATED ? LL * sizeof(uint32_t) : LL * sizeof(df));
    std::lock_guard<std::mutex> lock(g_table_mutex);
    auto it = g_tables.find(h->table_key);
    if (it != g_tables.end()) {
        DMFE_CUDA_TRY(cudaStreamWaitEvent(h->stream, it->second.ready, 0));
    } else {
        TableEntry e;
        for (int q = 0; q < 3; ++q)
            if (cudaMalloc(&e.t[q], tb) != cudaSuccess) {
                cudaGetLastError();
                for (int r = 0; r < q; ++r) cudaFree(e.t[r]);
                return DMFE_ERR_OOM;
            }
        if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
            for (void* q : e.t) cudaFree(q);
            return DMFE_ERR_CUDA;
        }
        it = g_tables.emplace(h->table_key, e).first;
    }
    TableEntry& e = it->second;
    const bool build = e.refs == 0;
    e.refs += 1;
    h->table_ref = true;
    if (v.precision == DMFE_FP64) {
        v.wt1 = (unsigned char*)e.t[0]; v.wt2 = (unsigned char*)e.t[1]; v.wt3 = (unsigned char*)e.t[2];
    } else if (v.precision == DMFE_FP32_COMPENSATED) {
        v.p1 = (uint32_t*)e.t[0]; v.p2 = (uint32_t*)e.t[1]; v.p3 = (uint32_t*)e.t[2];
    } else {
        v.q1 = (df*)e.t[0]; v.q2 = (df*)e.t[1]; v.q3 = (df*)e.t[2];
    }
    if (build) {
        const int rc = launch_tables(v, h->stream);
        if (rc) return rc;
        DMFE_CUDA_TRY(cudaEventRecord(e.ready, h->stream));
    }
    return DMFE_OK;
}

#define TRY(x)                   \
    do {                         \
        int rc_ = (x);           \
        if (rc_) return rc_;     \
    } while (0)

int read_state(dmfe_solver* h) {
    DMFE_CUDA_TRY(cudaMemcpyAsync(h->hstate, h->v.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DMFE_OK;
}

int write_state(dmfe_solver* h) {
    DMFE_CUDA_TRY(cudaMemcpyAsync(h->v.st, h->hstate, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DMFE_OK;
}

void build_poly(const std::vector<int>& pw, const std::vector<double>& cf, Poly& P) {
    std::memset(&P, 0, sizeof(P));
    int pmax = 1;
    for (size_t k = 0; k < pw.size(); ++k) {
        const int p = pw[k];
        const double c = cf[k];
        pmax = std::max(pmax, p);
        P.a0[p] += c;
        P.a1[p - 1] += c * p;
        if (p >= 2) P.a2[p - 2] += c * p * (p - 1);
    }
    P.deg0 = pmax;
    P.deg1 = pmax - 1;
    P.deg2 = std::max(pmax - 2, 0);
    for (int m = 0; m < DMFE_MAX_POWER; ++m) {
        P.f1[m] = (float)P.a1[m];
        P.f2[m] = (float)P.a2[m];
        P.g1[m] = (float)(P.a1[m] - (double)P.f1[m]);
        P.g2[m] = (float)(P.a2[m] - (double)P.f2[m]);
    }
}

// Work-unit size of the history-integral kernels (summation indices per unit).
constexpr int kMinChunk = 32;
int default_chunk(int precision, int L) {
    // Enough units to give every warp slot of the GPU (152 SMs x 16 warps) some work at
    // small L; at large L measured on GB300 (L = 2049, 4097): the FP32-pipe kernels run
    // best with one unit per output index, the FP64 kernel with 1024-index units up to
    // L ~ 3000.
    const long long per_warp = (long long)L * L / (152 * 16);
    int c = per_warp < kMinChunk ? kMinChunk : (int)((per_warp + 31) / 32 * 32);
    const int cap = (precision == DMFE_FP64 && L < 3072) ? 1024 : L;
    if (c > cap) c = cap;
    return c >= L ? L : c;
}

int validate(const dmfe_params* p) {
    if (!p || p->n_terms < 1 || p->n_terms > DMFE_MAX_TERMS || !p->powers || !p->coefs) return DMFE_ERR_ARG;
    for (int k = 0; k < p->n_terms; ++k) {
        if (p->powers[k] < 1 || p->powers[k] > DMFE_MAX_POWER) return DMFE_ERR_ARG;
        if (!std::isfinite(p->coefs[k])) return DMFE_ERR_ARG;
    }
    if (!(p->T >= 0.0) || !std::isfinite(p->T) || !std::isfinite(p->beta0)) return DMFE_ERR_ARG;
    if (p->L < 16 || p->L > 8192) return DMFE_ERR_ARG;
    if (p->s < 2 || p->s > 16 || p->s > p->L) return DMFE_ERR_ARG;
    if (!(p->grid_t_max > 2.718281828459046) || !std::isfinite(p->grid_t_max)) return DMFE_ERR_ARG;
    if (!(p->alpha >= 0.0 && p->alpha <= 1.0) || !(p->delta >= 0.0)) return DMFE_ERR_ARG;
    if (p->history_cap < 16) return DMFE_ERR_ARG;
    if (!(p->dt0 > 0.0) || !(p->dt_min > 0.0)) return DMFE_ERR_ARG;
    if (p->precision != DMFE_FP64 && p->precision != DMFE_FP32_COMPENSATED && p->precision != DMFE_DOUBLE_FLOAT)
        return DMFE_ERR_ARG;
    if (p->integrator != DMFE_RK_AUTO && p->integrator != DMFE_RK_DP5 && p->integrator != DMFE_RK_SSPRK104)
        return DMFE_ERR_ARG;
    if (!(p->rk_switch_dt >= 0.0)) return DMFE_ERR_ARG;
    if (p->hi_chunk != 0 && p->hi_chunk != kFlatSplit && p->hi_chunk < kMinChunk) return DMFE_ERR_ARG;
    if (p->interp < DMFE_INTERP_LAGRANGE_INDEX || p->interp > DMFE_INTERP_FH_THETA) return DMFE_ERR_ARG;
    if ((p->interp == DMFE_INTERP_FH_INDEX || p->interp == DMFE_INTERP_FH_THETA) &&
        (p->fh_d < 0 || p->fh_d > p->s - 1))
        return DMFE_ERR_ARG;
    if (p->s != 4 && p->s != 6 && p->s != 8 && p->s != 10) return DMFE_ERR_UNSUPPORTED;
    // the other schemes' weights live in the FP64 stencil tables
    if (p->interp != DMFE_INTERP_LAGRANGE_INDEX && p->precision != DMFE_FP64) return DMFE_ERR_UNSUPPORTED;
    // the logarithmic response interpolation is built into the FP64 path's coefficient tables
    if (p->log_r != 0 && p->log_r != 1) return DMFE_ERR_ARG;
    if (p->log_r && p->precision != DMFE_FP64) return DMFE_ERR_UNSUPPORTED;
    if (p->sparsify_every < 0 || p->sparsify_passes < 0 || p->sparsify_passes > kMaxSparsifyPasses)
        return DMFE_ERR_ARG;
    return DMFE_OK;
}

// Length of the real stability interval of Dormand-Prince 5: the largest x with
// |R(-y)| <= 1 on [0, x] for its stability polynomial R(z) = sum_{k<=5} z^k/k! + z^6/600
// (Hairer, Norsett & Wanner, Sec. II.5), by a scan and bisection.
double dp5_real_stability() {
    auto R = [](double y) {
        const double z = -y;
        const double c[7] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 600};
        double r = c[6];
        for (int k = 5; k >= 0; --k) r = r * z + c[k];
        return std::fabs(r);
    };
    double y = 0.0;
    const double dy = 1e-3;
    while (R(y + dy) <= 1.0 + 1e-14) y += dy;
    double lo = y, hi = y + dy;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (R(mid) <= 1.0) lo = mid; else hi = mid;
    }
    return lo;
}

// Controller step at which Dormand-Prince hands over to SSPRK(10,4) (Sec. 3.5): the
// Jacobian's spectrum lies on the negative real axis within 4 sqrt(f''(1)).
double switch_dt_for(const dmfe_params* p) {
    if (p->integrator != DMFE_RK_AUTO) return INFINITY;
    if (p->rk_switch_dt > 0.0) return p->rk_switch_dt;
    double fpp1 = 0.0;
    for (int k = 0; k < p->n_terms; ++k)
        if (p->powers[k] >= 2) fpp1 += p->coefs[k] * p->powers[k] * (p->powers[k] - 1);
    if (!(fpp1 > 0.0)) return INFINITY;
    return dp5_real_stability() / (4.0 * std::sqrt(fpp1));
}

int create_impl(const dmfe_params* pin, dmfe_solver* h) {
    h->p = *pin;
    h->powers.assign(pin->powers, pin->powers + pin->n_terms);
    h->coefs.assign(pin->coefs, pin->coefs + pin->n_terms);
    h->p.powers = h->powers.data();
    h->p.coefs = h->coefs.data();
    const int L = pin->L, cap = pin->history_cap;
    SolverView& v = h->v;
    v.L = L;
    v.s = pin->s;
    v.cap = cap;
    v.precision = pin->precision;
    v.sparsify = pin->sparsify ? 1 : 0;
    v.sp_every = pin->sparsify_every;
    v.sp_passes = pin->sparsify_passes < 1 ? 1 : pin->sparsify_passes;
    v.T = pin->T;
    v.beta0 = pin->beta0;
    v.rk_switch_dt = switch_dt_for(&h->p);
    v.interp = pin->interp;
    v.fh_d = pin->fh_d;
    v.log_r = pin->log_r ? 1 : 0;
    build_poly(h->powers, h->coefs, v.poly);
    v.gamma = host_gamma_from_tmax(pin->grid_t_max);
    v.ga = std::atan(std::exp(-v.gamma));
    v.gD = std::atan(std::exp(v.gamma)) - v.ga;
    v.alpha = pin->alpha;
    v.delta = pin->delta;
    host_theta_grid(L, v.gamma, pin->alpha, pin->delta, h->theta, h->omega);
    TRY(host_spline_weights(h->theta, h->nu));

    if (pin->stream) {
        h->stream = (cudaStream_t)pin->stream;
    } else {
        DMFE_CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    DMFE_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (cudaMallocHost((void**)&h->hstate, sizeof(DevState)) != cudaSuccess) return DMFE_ERR_OOM;

    const size_t LL = (size_t)L * L;
    void* p;
    TRY(dev_alloc(h, &p, L * sizeof(double))); v.theta = (double*)p;
    TRY(dev_alloc(h, &p, L * sizeof(double))); v.omega = (double*)p;
    TRY(dev_alloc(h, &p, L * sizeof(double))); v.nu = (double*)p;
    TRY(dev_alloc(h, &p, L * sizeof(float))); v.omega32 = (float*)p;
    TRY(dev_alloc(h, &p, L * sizeof(float))); v.nu32 = (float*)p;
    const size_t wts = 8 + 8 * (size_t)pin->s;  // bytes per stencil entry
    if (v.precision == DMFE_DOUBLE_FLOAT) {
        TRY(dev_alloc(h, &p, L * sizeof(df))); v.omega_df = (df*)p;
        TRY(dev_alloc(h, &p, L * sizeof(df))); v.nu_df = (df*)p;
        TRY(dev_alloc(h, &p, L * sizeof(dfrow))); v.rowdf = (dfrow*)p;
        TRY(dev_alloc(h, &p, (cap + 1) * sizeof(dfslice))); v.slicedf = (dfslice*)p;
        TRY(dev_alloc(h, &p, L * sizeof(df8))); v.vrowdf = (df8*)p;
        TRY(dev_alloc(h, &p, L * sizeof(int))); v.cell = (int*)p;
    }
    for (int b = 0; b < 2; ++b) {
        TRY(dev_alloc(h, &p, cap * sizeof(double))); v.ht[b] = (double*)p;
        TRY(dev_alloc(h, &p, (size_t)cap * L * sizeof(dbl4))); v.hist[b] = (dbl4*)p;
        if (v.precision == DMFE_FP32_COMPENSATED) {
            TRY(dev_alloc(h, &p, (size_t)cap * L * sizeof(float4))); v.hist32[b] = (float4*)p;
            if (b == 0) {
                TRY(dev_alloc(h, &p, L * sizeof(float4))); v.vrow32 = (float4*)p;
                TRY(dev_alloc(h, &p, L * sizeof(float4))); v.row32f = (float4*)p;
                TRY(dev_alloc(h, &p, (cap + 1) * sizeof(float4))); v.slice32 = (float4*)p;
            }
        }
        if (v.precision == DMFE_FP64 && b == 0) {
            TRY(dev_alloc(h, &p, L * sizeof(dbl4))); v.row64 = (dbl4*)p;
            TRY(dev_alloc(h, &p, (cap + 1) * sizeof(double))); v.slice64 = (double*)p;
        }
        if (v.precision == DMFE_DOUBLE_FLOAT) {
            TRY(dev_alloc(h, &p, (size_t)cap * L * sizeof(df8))); v.histdf[b] = (df8*)p;
        }
        if (v.precision == DMFE_FP64) {
            TRY(dev_alloc(h, &p, (size_t)cap * L * sizeof(dbl8))); v.hcoef[b] = (dbl8*)p;
        }
        if (pin->log_r) {
            TRY(dev_alloc(h, &p, (size_t)cap * L * sizeof(dbl4))); v.lcoef[b] = (dbl4*)p;
        }
    }
    TRY(dev_alloc(h, &p, sizeof(DevState))); v.st = (DevState*)p;
    TRY(dev_alloc(h, &p, 2 * 2 * (size_t)L * sizeof(double))); v.Y = (double*)p;
    TRY(dev_alloc(h, &p, 2 * (size_t)kMaxPrepBlocks * sizeof(double))); v.mupart = (double*)p;
    TRY(dev_alloc(h, &p, (size_t)kCtlGrid * sizeof(double))); v.epart = (double*)p;
    TRY(dev_alloc(h, &p, sizeof(int))); v.ctl_count = (int*)p;
    DMFE_CUDA_TRY(cudaMemsetAsync(v.ctl_count, 0, sizeof(int), h->stream));
    TRY(dev_alloc(h, &p, (kMaxStages + 1) * 2 * (size_t)L * sizeof(double))); v.k = (double*)p;
    TRY(dev_alloc(h, &p, 2 * L * sizeof(double))); v.ynew = (double*)p;
    TRY(dev_alloc(h, &p, (size_t)DMFE_NS * L * sizeof(double))); v.S = (double*)p;
    // Partial sums for units of at least kMinChunk summation indices (the smallest chunk
    // the autotuner or an override may select).
    TRY(dev_alloc(h, &p, (size_t)(L / kMinChunk > 1 ? L / kMinChunk : 1) * 9 * L * sizeof(double)));
    v.Spart = (double*)p;
    TRY(dev_alloc(h, &p, (size_t)L * sizeof(B1Desc))); v.b1 = (B1Desc*)p;
    if (!v.cell) { TRY(dev_alloc(h, &p, L * sizeof(int))); v.cell = (int*)p; }
    TRY(dev_alloc(h, &p, (size_t)L * sizeof(int))); v.jcount = (int*)p;
    DMFE_CUDA_TRY(cudaMemsetAsync(v.jcount, 0, (size_t)L * sizeof(int), h->stream));
    // work units of a single solve: the flat split wherever it gives every warp at least 256
    // pairs (all SMs and warp slots get equal work), else units; dmfe_autotune compares it
    // with the unit sizes
    int nsm = 0, dev_ = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev_));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_));
    const bool flat_ok = flat_split_fits(L, (long long)nsm * 16);
    if (pin->hi_chunk == kFlatSplit) v.hi_chunk = flat_ok ? kFlatSplit : default_chunk(v.precision, L);
    else if (pin->hi_chunk > 0) v.hi_chunk = pin->hi_chunk < L ? pin->hi_chunk : L;
    else v.hi_chunk = flat_ok ? kFlatSplit : default_chunk(v.precision, L);
    if (const char* e = std::getenv("DMFE_HI_CHUNK")) {
        const int c = std::atoi(e);
        if (c >= kMinChunk) v.hi_chunk = c < L ? c : L;
    }
    TRY(dev_alloc(h, &p, cap * sizeof(double))); v.eps_sp = (double*)p;
    TRY(dev_alloc(h, &p, cap * sizeof(int))); v.keep = (int*)p;
    TRY(dev_alloc(h, &p, cap * sizeof(int))); v.newidx = (int*)p;
    TRY(dev_alloc(h, &p, (4 * (size_t)L + 16) * sizeof(double))); h->scratch = (double*)p;

    std::vector<float> om32(L), nu32(L);
    for (int i = 0; i < L; ++i) {
        om32[i] = (float)h->omega[i];
        nu32[i] = (float)h->nu[i];
    }
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.theta, h->theta.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.omega, h->omega.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.nu, h->nu.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.omega32, om32.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.nu32, nu32.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    std::vector<df> omdf(L), nudf(L);
    if (v.precision == DMFE_DOUBLE_FLOAT) {
        for (int i = 0; i < L; ++i) {
            omdf[i] = df_from_d(h->omega[i]);
            nudf[i] = df_from_d(h->nu[i]);
        }
        DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.omega_df, omdf.data(), L * sizeof(df), cudaMemcpyHostToDevice, h->stream));
        DMFE_CUDA_TRY(cudaMemcpyAsync((void*)v.nu_df, nudf.data(), L * sizeof(df), cudaMemcpyHostToDevice, h->stream));
    }
    std::memset(h->hstate, 0, sizeof(DevState));
    h->hstate->dt = pin->dt0;
    h->hstate->dt_min = pin->dt_min;
    h->hstate->tol = 1e-8;
    h->hstate->method = pin->integrator == DMFE_RK_SSPRK104 ? 1 : 0;
    h->hstate->t_switch = -1.0;
    TRY(write_state(h));
    TRY(acquire_tables(h, LL * wts));
    TRY(launch_initial_slice(v, h->stream));
    if (hi_config(v, &h->hi_grid, &h->hi_smem) != DMFE_OK) {
        // (a flat split that the launch shape cannot hold falls back to units)
        if (v.hi_chunk != kFlatSplit) return DMFE_ERR_UNSUPPORTED;
        v.hi_chunk = default_chunk(v.precision, L);
        TRY(hi_config(v, &h->hi_grid, &h->hi_smem));
    }
    if (v.hi_chunk == kFlatSplit) TRY(set_flat_tables(h, h->hi_grid));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    DMFE_CUDA_TRY(cudaGetLastError());
    return DMFE_OK;
}

void release_tables(dmfe_solver* h) {
    if (!h->table_ref) return;
    std::lock_guard<std::mutex> lock(g_table_mutex);
    auto it = g_tables.find(h->table_key);
    h->table_ref = false;
    if (it == g_tables.end()) return;
    if (--it->second.refs == 0) {
        // the last user: other solvers' work on these tables has been synchronised by their
        // own destroy; this solver's stream was synchronised by the caller
        if (it->second.ready) cudaEventSynchronize(it->second.ready);
        for (void* q : it->second.t) cudaFree(q);
        if (it->second.ready) cudaEventDestroy(it->second.ready);
        g_tables.erase(it);
    }
}

void destroy_impl(dmfe_solver* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
    release_tables(h);
    for (void* p : h->allocs) cudaFree(p);
    if (h->hstate) cudaFreeHost(h->hstate);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// The three parts of one step of this solver, for the graph capture.
struct SoloParts : StepParts {
    const dmfe_solver* h;
    explicit SoloParts(const dmfe_solver* hh) : h(hh) {}
    int head(cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) override {
        return launch_step_head(h->v, h->hi_grid, cond, use_cond, s);
    }
    int tail(cudaStream_t s) override { return launch_step_tail(h->v, h->hi_grid, s); }
    int sp(cudaStream_t s) override { return launch_step_sparsify(h->v, s); }
};

// Capture one step into a graph on the private capture stream: with the SSPRK stages in
// a conditional node, or (if the runtime refuses that) inline, where they gate
// themselves off in Dormand-Prince steps.
int build_step_graph(dmfe_solver* h) {
    if (h->step_exec) return DMFE_OK;
    SoloParts parts(h);
    if (!step_graph_plain() && capture_step_graph(h->cap_stream, true, parts, &h->step_exec) == DMFE_OK) {
        h->conditional_graph = true;
        return DMFE_OK;
    }
    h->conditional_graph = false;
    return capture_step_graph(h->cap_stream, false, parts, &h->step_exec);
}

int upload_row(dmfe_solver* h, const double* C, const double* R, double* dst) {
    const int L = h->v.L;
    DMFE_CUDA_TRY(cudaMemcpyAsync(dst, C, L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync(dst + L, R, L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    return DMFE_OK;
}

double last_time(dmfe_solver* h) { return h->hstate->t; }

}  // namespace

const SolverView& solver_view(const dmfe_solver* h) { return h->v; }
void solver_set_chunk(dmfe_solver* h, int chunk) { h->v.hi_chunk = chunk; }

int solver_read_state(dmfe_solver* h, DevState* out) {
    TRY(read_state(h));
    *out = *h->hstate;
    return DMFE_OK;
}

extern "C" {

void dmfe_default_params(dmfe_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->T = 0.5;
    p->L = 513;
    p->s = 4;
    p->grid_t_max = 1e5;
    p->history_cap = 0;  // 0 here means "use L" at create
    p->dt0 = 1e-4;
    p->dt_min = 1e-12;
    p->precision = DMFE_FP64;
    p->sparsify = 1;
    p->integrator = DMFE_RK_AUTO;
    p->rk_switch_dt = 0.0;
    p->hi_chunk = 0;
    p->interp = DMFE_INTERP_LAGRANGE_INDEX;
    p->fh_d = 3;
    p->sparsify_every = 0;
    p->sparsify_passes = 1;
}

const char* dmfe_strerror(int code) {
    switch (code) {
        case DMFE_OK: return "ok";
        case DMFE_ERR_ARG: return "invalid argument";
        case DMFE_ERR_OOM: return "out of memory";
        case DMFE_ERR_NONFINITE: return "non-finite value in the step error estimate";
        case DMFE_ERR_STEP_UNDERFLOW: return "step size fell below dt_min";
        case DMFE_ERR_CAPACITY: return "history store full";
        case DMFE_ERR_CUDA: return "CUDA runtime error";
        case DMFE_ERR_TIMEOUT: return "bounded device wait timed out";
        case DMFE_ERR_UNSUPPORTED: return "unsupported configuration";
        case DMFE_ERR_IO: return "checkpoint i/o error";
    }
    return "unknown error";
}

// Mirrors the allocations of create_impl (keep the two in step).
unsigned long long dmfe_footprint(const dmfe_params* pin) {
    if (!pin) return 0;
    dmfe_params p = *pin;
    if (p.history_cap == 0) p.history_cap = p.L;
    if (validate(&p)) return 0;
    const unsigned long long L = p.L, cap = p.history_cap, LL = L * L;
    unsigned long long tot = 0;
    auto add = [&tot](unsigned long long b) {
        const unsigned long long g = b >= (2ull << 20) ? (2ull << 20) : 512ull;
        tot += (b + g - 1) / g * g;
    };
    for (int k = 0; k < 3; ++k) add(L * 8);
    add(L * 4); add(L * 4);
    const unsigned long long wts = 8 + 8 * (unsigned long long)p.s;
    if (p.precision == DMFE_FP64) {
        for (int k = 0; k < 3; ++k) add(LL * wts);
    } else if (p.precision == DMFE_FP32_COMPENSATED) {
        for (int k = 0; k < 3; ++k) add(LL * 4);
    } else {
        for (int k = 0; k < 3; ++k) add(LL * sizeof(df));
        add(L * sizeof(df)); add(L * sizeof(df)); add(L * sizeof(dfrow)); add((cap + 1) * sizeof(dfslice));
        add(L * sizeof(df8)); add(L * 4);
    }
    for (int b = 0; b < 2; ++b) {
        add(cap * 8);
        add(cap * L * sizeof(dbl4));
        if (p.precision == DMFE_FP32_COMPENSATED) add(cap * L * sizeof(float4));
        if (p.precision == DMFE_FP32_COMPENSATED && b == 0) add(L * sizeof(float4));
        if (p.precision == DMFE_DOUBLE_FLOAT) add(cap * L * sizeof(df8));
        if (p.precision == DMFE_FP64) add(cap * L * sizeof(dbl8));
        if (p.log_r) add(cap * L * sizeof(dbl4));
    }
    add(sizeof(DevState)); add(4 * L * 8);
    add(2ull * kMaxPrepBlocks * 8); add(kCtlGrid * 8); add(4);
    add(2ull * (kMaxStages + 1) * L * 8); add(2 * L * 8); add(DMFE_NS * L * 8);
    add((L / kMinChunk > 1 ? L / kMinChunk : 1) * 9 * L * 8); add(L * sizeof(B1Desc));
    if (p.precision != DMFE_DOUBLE_FLOAT) add(L * 4);
    add(L * 4); add(cap * 8); add(cap * 4); add(cap * 4); add((4 * L + 16) * 8);
    return tot;
}

int dmfe_create(const dmfe_params* pin, dmfe_solver** out) {
    if (!out) return DMFE_ERR_ARG;
    *out = nullptr;
    if (!pin) return DMFE_ERR_ARG;
    dmfe_params p = *pin;
    if (p.history_cap == 0) p.history_cap = p.L;
    int rc = validate(&p);
    if (rc) return rc;
    dmfe_solver* h = new (std::nothrow) dmfe_solver();
    if (!h) return DMFE_ERR_OOM;
    rc = create_impl(&p, h);
    if (rc) {
        destroy_impl(h);
        return rc;
    }
    *out = h;
    return DMFE_OK;
}

void dmfe_destroy(dmfe_solver* h) { destroy_impl(h); }

int dmfe_grid(dmfe_solver* h, double* theta, double* omega, double* nu) {
    if (!h) return DMFE_ERR_ARG;
    const int L = h->v.L;
    if (theta) std::memcpy(theta, h->theta.data(), L * sizeof(double));
    if (omega) std::memcpy(omega, h->omega.data(), L * sizeof(double));
    if (nu) std::memcpy(nu, h->nu.data(), L * sizeof(double));
    return DMFE_OK;
}

int dmfe_theta_grid(int L, double grid_t_max, double alpha, double delta, double* theta, double* omega,
                    double* nu) {
    if (L < 16 || L > 8192) return DMFE_ERR_ARG;
    if (!(grid_t_max > 2.718281828459046) || !std::isfinite(grid_t_max)) return DMFE_ERR_ARG;
    if (!(alpha >= 0.0 && alpha <= 1.0) || !(delta >= 0.0) || !std::isfinite(delta)) return DMFE_ERR_ARG;
    std::vector<double> th, om, w;
    host_theta_grid(L, host_gamma_from_tmax(grid_t_max), alpha, delta, th, om);
    if (nu) TRY(host_spline_weights(th, w));
    if (theta) std::memcpy(theta, th.data(), L * sizeof(double));
    if (omega) std::memcpy(omega, om.data(), L * sizeof(double));
    if (nu) std::memcpy(nu, w.data(), L * sizeof(double));
    return DMFE_OK;
}

int dmfe_tables(dmfe_solver* h, double* x1, double* x2, double* x3) {
    if (!h) return DMFE_ERR_ARG;
    const size_t LL = (size_t)h->v.L * h->v.L;
    // positions are recomputed on demand by the table kernel into temporary buffers
    SolverView v = h->v;
    v.p1 = v.p2 = v.p3 = nullptr;
    v.q1 = v.q2 = v.q3 = nullptr;
    v.wt1 = v.wt2 = v.wt3 = nullptr;
    double* buf = nullptr;
    DMFE_CUDA_TRY(cudaMallocAsync((void**)&buf, 3 * LL * sizeof(double), h->stream));
    v.x1 = buf;
    v.x2 = buf + LL;
    v.x3 = buf + 2 * LL;
    int rc = launch_tables(v, h->stream);
    double* outs[3] = {x1, x2, x3};
    for (int q = 0; q < 3 && !rc; ++q)
        if (outs[q] && cudaMemcpyAsync(outs[q], buf + q * LL, LL * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->stream) != cudaSuccess)
            rc = DMFE_ERR_CUDA;
    cudaFreeAsync(buf, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
    return rc;
}

int dmfe_integrate(dmfe_solver* h, double t_max, double tol) {
    if (!h || !std::isfinite(t_max) || !(tol > 0.0)) return DMFE_ERR_ARG;
    if (t_max > h->p.grid_t_max * (1.0 + 1e-12)) return DMFE_ERR_ARG;
    TRY(read_state(h));
    if (h->hstate->status) return h->hstate->status;
    if (h->hstate->t >= t_max) return DMFE_OK;
    TRY(launch_begin_integrate(h->v, t_max, tol, h->stream));
    const bool graph = build_step_graph(h) == DMFE_OK;
    int batch = 1;
    for (;;) {
        for (int it = 0; it < batch; ++it) {
            if (graph) {
                DMFE_CUDA_TRY(cudaGraphLaunch(h->step_exec, h->stream));
            } else {
                TRY(launch_step(h->v, h->hi_grid, h->stream));
            }
        }
        TRY(read_state(h));
        if (h->hstate->status || h->hstate->done) break;
        batch = std::min(batch * 2, 64);
    }
    return h->hstate->status;
}

int dmfe_step(dmfe_solver* h, int nsteps, double t_max, double tol, void* stream) {
    if (!h || nsteps < 0 || !std::isfinite(t_max) || !(tol > 0.0)) return DMFE_ERR_ARG;
    if (t_max > h->p.grid_t_max * (1.0 + 1e-12)) return DMFE_ERR_ARG;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(launch_begin_integrate(h->v, t_max, tol, s));
    const bool graph = build_step_graph(h) == DMFE_OK;
    for (int it = 0; it < nsteps; ++it) {
        if (graph) {
            DMFE_CUDA_TRY(cudaGraphLaunch(h->step_exec, s));
        } else {
            TRY(launch_step(h->v, h->hi_grid, s));
        }
    }
    return DMFE_OK;
}

static int get_two_time(dmfe_solver* h, int n, const double* t, const double* tp, double* out, int which) {
    if (!h || n < 0 || (n > 0 && (!t || !tp || !out))) return DMFE_ERR_ARG;
    if (n == 0) return DMFE_OK;
    TRY(read_state(h));
    const double tl = h->hstate->t;
    for (int q = 0; q < n; ++q) {
        if (!(t[q] >= 0.0) || !(tp[q] >= 0.0)) return DMFE_ERR_ARG;
        if (std::max(t[q], tp[q]) > tl * (1.0 + 1e-15)) return DMFE_ERR_ARG;
    }
    double* buf = nullptr;
    DMFE_CUDA_TRY(cudaMallocAsync((void**)&buf, 3 * (size_t)n * sizeof(double), h->stream));
    int rc = DMFE_OK;
    if (cudaMemcpyAsync(buf, t, n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(buf + n, tp, n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        rc = DMFE_ERR_CUDA;
    if (!rc) rc = launch_lookup(h->v, n, buf, buf + n, which, buf + 2 * n, h->stream);
    if (!rc && cudaMemcpyAsync(out, buf + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = DMFE_ERR_CUDA;
    cudaFreeAsync(buf, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
    return rc;
}

int dmfe_get_C(dmfe_solver* h, int n, const double* t, const double* tp, double* out) {
    return get_two_time(h, n, t, tp, out, 0);
}

int dmfe_get_R(dmfe_solver* h, int n, const double* t, const double* tp, double* out) {
    return get_two_time(h, n, t, tp, out, 1);
}

int dmfe_get_row(dmfe_solver* h, double* t, double* C, double* R, double* mu, double* E) {
    if (!h) return DMFE_ERR_ARG;
    TRY(read_state(h));
    const int L = h->v.L;
    const DevState& s = *h->hstate;
    std::vector<dbl4> row(L);
    DMFE_CUDA_TRY(cudaMemcpyAsync(row.data(), h->v.hist[s.active] + (size_t)(s.n - 1) * L, L * sizeof(dbl4),
                                  cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    std::vector<double> Cv(L), Rv(L);
    for (int i = 0; i < L; ++i) {
        Cv[i] = row[i].x;
        Rv[i] = row[i].z;
    }
    if (t) *t = s.t;
    if (C) std::memcpy(C, Cv.data(), L * sizeof(double));
    if (R) std::memcpy(R, Rv.data(), L * sizeof(double));
    if (mu || E) {
        double* d = h->scratch;
        TRY(upload_row(h, Cv.data(), Rv.data(), d));
        TRY(launch_assemble(h->v, d, h->v.S, s.t, d + 2 * L, d + 3 * L, d + 4 * L, h->stream));
        double muE[2];
        DMFE_CUDA_TRY(cudaMemcpyAsync(muE, d + 4 * L, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (mu) *mu = muE[0];
        if (E) *E = muE[1];
    }
    return DMFE_OK;
}

int dmfe_set_history(dmfe_solver* h, int n, const double* t, const double* C, const double* dC,
                     const double* R, const double* dR) {
    if (!h || !t || !C || !dC || !R || !dR) return DMFE_ERR_ARG;
    const int L = h->v.L;
    if (n < 1 || n > h->v.cap) return DMFE_ERR_ARG;
    if (t[0] != 0.0) return DMFE_ERR_ARG;
    for (int k = 1; k < n; ++k)
        if (!(t[k] > t[k - 1])) return DMFE_ERR_ARG;
    std::vector<dbl4> hist((size_t)n * L);
    for (size_t q = 0; q < (size_t)n * L; ++q) hist[q] = dbl4{C[q], dC[q], R[q], dR[q]};
    TRY(read_state(h));
    DevState& s = *h->hstate;
    s.active = 0;
    s.n = n;
    s.t = t[n - 1];
    s.done = 0;
    s.pending = 0;
    s.sp_ran = 0;
    s.sp_left = 0;
    s.status = 0;
    DMFE_CUDA_TRY(cudaMemcpyAsync(h->v.hist[0], hist.data(), hist.size() * sizeof(dbl4), cudaMemcpyHostToDevice, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync(h->v.ht[0], t, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    TRY(write_state(h));
    TRY(launch_refresh_replica(h->v, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DMFE_OK;
}

int dmfe_get_history(dmfe_solver* h, int* n, double* t, double* C, double* dC, double* R, double* dR) {
    if (!h || !n) return DMFE_ERR_ARG;
    TRY(read_state(h));
    const int L = h->v.L;
    const DevState& s = *h->hstate;
    *n = s.n;
    std::vector<dbl4> hist((size_t)s.n * L);
    DMFE_CUDA_TRY(cudaMemcpyAsync(hist.data(), h->v.hist[s.active], hist.size() * sizeof(dbl4), cudaMemcpyDeviceToHost, h->stream));
    if (t) DMFE_CUDA_TRY(cudaMemcpyAsync(t, h->v.ht[s.active], s.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q < hist.size(); ++q) {
        if (C) C[q] = hist[q].x;
        if (dC) dC[q] = hist[q].y;
        if (R) R[q] = hist[q].z;
        if (dR) dR[q] = hist[q].w;
    }
    return DMFE_OK;
}

int dmfe_history_integrals_dev(dmfe_solver* h, double t, const double* row_dev, double* S_dev, void* stream) {
    if (!h || !row_dev || !S_dev || !std::isfinite(t)) return DMFE_ERR_ARG;
    if (t < last_time(h)) return DMFE_ERR_ARG;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    return launch_history_integrals(h->v, row_dev, t, false, S_dev, h->hi_grid, s);
}

int dmfe_history_integrals(dmfe_solver* h, double t, const double* C_row, const double* R_row, double* S,
                           double* mu) {
    if (!h || !C_row || !R_row || !S) return DMFE_ERR_ARG;
    TRY(read_state(h));
    if (!(t >= h->hstate->t) || !std::isfinite(t)) return DMFE_ERR_ARG;
    const int L = h->v.L;
    double* d = h->scratch;
    TRY(upload_row(h, C_row, R_row, d));
    TRY(launch_history_integrals(h->v, d, t, false, h->v.S, h->hi_grid, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync(S, h->v.S, (size_t)DMFE_NS * L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (mu) {
        TRY(launch_assemble(h->v, d, h->v.S, t, d + 2 * L, d + 3 * L, d + 4 * L, h->stream));
        DMFE_CUDA_TRY(cudaMemcpyAsync(mu, d + 4 * L, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DMFE_OK;
}

int dmfe_rhs(dmfe_solver* h, double t, const double* C_row, const double* R_row, double* dC, double* dR,
             double* mu, double* E) {
    if (!h || !C_row || !R_row) return DMFE_ERR_ARG;
    TRY(read_state(h));
    if (!(t >= h->hstate->t) || !std::isfinite(t)) return DMFE_ERR_ARG;
    const int L = h->v.L;
    double* d = h->scratch;
    TRY(upload_row(h, C_row, R_row, d));
    if (t == 0.0) {
        std::vector<double> S0((size_t)DMFE_NS * L, 0.0);
        std::fill(S0.begin() + 9 * (size_t)L, S0.end(), 1.0);
        DMFE_CUDA_TRY(cudaMemcpyAsync(h->v.S, S0.data(), S0.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    } else {
        TRY(launch_history_integrals(h->v, d, t, false, h->v.S, h->hi_grid, h->stream));
    }
    TRY(launch_assemble(h->v, d, h->v.S, t, d + 2 * L, d + 3 * L, d + 4 * L, h->stream));
    std::vector<double> out(2 * L + 2);
    DMFE_CUDA_TRY(cudaMemcpyAsync(out.data(), d + 2 * L, (2 * L + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (dC) std::memcpy(dC, out.data(), L * sizeof(double));
    if (dR) std::memcpy(dR, out.data() + L, L * sizeof(double));
    if (mu) *mu = out[2 * L];
    if (E) *E = out[2 * L + 1];
    return DMFE_OK;
}

int dmfe_sparsify(dmfe_solver* h, double tol, int* removed) {
    if (!h || !(tol > 0.0)) return DMFE_ERR_ARG;
    TRY(read_state(h));
    const int n_old = h->hstate->n;
    TRY(launch_sparsify(h->v, false, tol, h->stream));
    TRY(read_state(h));
    if (removed) {
        std::vector<int> keep(n_old);
        DMFE_CUDA_TRY(cudaMemcpyAsync(keep.data(), h->v.keep, n_old * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
        const bool ran = h->hstate->n != n_old;
        for (int k = 0; k < h->v.cap; ++k) removed[k] = 0;
        if (ran)
            for (int k = 0; k < n_old; ++k) removed[k] = keep[k] ? 0 : 1;
    }
    return DMFE_OK;
}

int dmfe_stats(dmfe_solver* h, dmfe_stats_t* o) {
    if (!h || !o) return DMFE_ERR_ARG;
    TRY(read_state(h));
    const DevState& s = *h->hstate;
    std::memset(o, 0, sizeof(*o));
    o->t = s.t;
    o->dt = s.dt;
    o->mu = s.mu;
    o->E = s.E;
    o->last_eps = s.eps;
    o->max_eps_sparse = s.max_eps_sparse;
    o->steps_accepted = s.steps_accepted;
    o->steps_rejected = s.steps_rejected;
    o->stages = s.stages;
    o->sparsify_passes = s.sparsify_passes;
    o->bounds_site = s.bounds_site;
    o->slices_removed = s.slices_removed;
    o->forced_removals = s.forced_removals;
    o->n_slices = s.n;
    o->status = s.status;
    o->L = h->v.L;
    o->history_cap = h->v.cap;
    o->s = h->v.s;
    o->precision = h->v.precision;
    o->method = s.method == 1 ? DMFE_RK_SSPRK104 : DMFE_RK_DP5;
    o->t_switch = s.t_switch;
    o->rk_switch_dt = h->v.rk_switch_dt;
    o->step_graph = h->step_exec ? (h->conditional_graph ? 2 : 1) : 0;
    return DMFE_OK;
}

static std::mutex g_tune_mutex;
static std::map<std::tuple<int, int, int, int>, int> g_tune_cache;

int dmfe_autotune(dmfe_solver* h, int* chunk_out) {
    if (!h) return DMFE_ERR_ARG;
    SolverView& v = h->v;
    const auto key = std::make_tuple(v.L, v.cap, v.s, v.precision);
    int best = -1;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best < 0) {
        TRY(read_state(h));
        const int L = v.L;
        const DevState& s = *h->hstate;
        // stage row = the last stored slice
        std::vector<dbl4> row(L);
        DMFE_CUDA_TRY(cudaMemcpyAsync(row.data(), v.hist[s.active] + (size_t)(s.n - 1) * L, L * sizeof(dbl4),
                                      cudaMemcpyDeviceToHost, h->stream));
        DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
        std::vector<double> CR(2 * L);
        for (int i = 0; i < L; ++i) {
            CR[i] = row[i].x;
            CR[L + i] = row[i].z;
        }
        double* d = h->scratch;
        DMFE_CUDA_TRY(cudaMemcpyAsync(d, CR.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        std::vector<int> cands;
        for (int c : {kMinChunk, 64, 128, 256, 512, 1024, 2048, 4096, L}) {
            const int cc = c >= L ? L : c;
            if (cc >= kMinChunk || cc == L)
                if (std::find(cands.begin(), cands.end(), cc) == cands.end()) cands.push_back(cc);
        }
        // L/P for P parts: part counts whose P*L units fill the last wave of warps best
        for (int P = 2; P <= 16; ++P) {
            const int cc = L / P;
            if (cc >= kMinChunk && std::find(cands.begin(), cands.end(), cc) == cands.end()) cands.push_back(cc);
        }
        cands.push_back(kFlatSplit);  // tried where its launch shape fits (hi_config)
        cudaEvent_t e0, e1;
        DMFE_CUDA_TRY(cudaEventCreate(&e0));
        DMFE_CUDA_TRY(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        const int saved = v.hi_chunk;
        int rc = DMFE_OK;
        for (int c : cands) {
            v.hi_chunk = c;
            int grid = 0;
            size_t sm = 0;
            rc = hi_config(v, &grid, &sm);
            if (rc == DMFE_ERR_UNSUPPORTED && c == kFlatSplit) {
                rc = DMFE_OK;  // this grid is too small for the flat split
                continue;
            }
            if (!rc && c == kFlatSplit) rc = set_flat_tables(h, grid);
            if (rc) break;
            float tot = 0.f;
            for (int it = 0; it < 4 && !rc; ++it) {
                if (cudaEventRecord(e0, h->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
                if (!rc) rc = launch_history_integrals(v, d, s.t, false, v.S, grid, h->stream);
                if (!rc && cudaEventRecord(e1, h->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = DMFE_ERR_CUDA;
                float ms = 0.f;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = DMFE_ERR_CUDA;
                if (it > 0) tot += ms;  // first launch warms caches
            }
            if (rc) break;
            if (tot < best_ms) {
                best_ms = tot;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) {
            v.hi_chunk = saved;
            hi_config(v, &h->hi_grid, &h->hi_smem);
            if (saved == kFlatSplit) set_flat_tables(h, h->hi_grid);
            return rc;
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    v.hi_chunk = best;
    TRY(hi_config(v, &h->hi_grid, &h->hi_smem));
    if (best == kFlatSplit) TRY(set_flat_tables(h, h->hi_grid));
    if (h->step_exec) {  // the captured step holds the old launch configuration
        cudaGraphExecDestroy(h->step_exec);
        h->step_exec = nullptr;
    }
    if (chunk_out) *chunk_out = best;
    return DMFE_OK;
}

int dmfe_sync(dmfe_solver* h) {
    if (!h) return DMFE_ERR_ARG;
    TRY(read_state(h));
    return h->hstate->status;
}

// ---- checkpoint format: magic, version, parameters, f, device state, history (FP64).
static const char kMagic[8] = {'D', 'M', 'F', 'E', 'C', 'K', 'P', '2'};
static const int kCkpVersion = 4;  // 2: integrator fields; 3: log-R flag in the parameters;
                                   // 4: sparsification policy and its round state

int dmfe_checkpoint(dmfe_solver* h, const char* path) {
    if (!h || !path) return DMFE_ERR_ARG;
    TRY(read_state(h));
    const DevState s = *h->hstate;
    const int L = h->v.L;
    std::vector<dbl4> hist((size_t)s.n * L);
    std::vector<double> ht(s.n);
    DMFE_CUDA_TRY(cudaMemcpyAsync(hist.data(), h->v.hist[s.active], hist.size() * sizeof(dbl4), cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaMemcpyAsync(ht.data(), h->v.ht[s.active], s.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DMFE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return DMFE_ERR_IO;
    bool ok = true;
    auto W = [&](const void* p, size_t n) { ok = ok && std::fwrite(p, 1, n, f) == n; };
    const int version = kCkpVersion;
    dmfe_params p = h->p;
    p.powers = nullptr;
    p.coefs = nullptr;
    p.stream = nullptr;
    W(kMagic, 8);
    W(&version, sizeof(int));
    W(&p, sizeof(p));
    W(h->powers.data(), p.n_terms * sizeof(int));
    W(h->coefs.data(), p.n_terms * sizeof(double));
    W(&s, sizeof(s));
    W(ht.data(), ht.size() * sizeof(double));
    W(hist.data(), hist.size() * sizeof(dbl4));
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DMFE_OK : DMFE_ERR_IO;
}

int dmfe_restore(const char* path, void* stream, dmfe_solver** out) {
    if (!path || !out) return DMFE_ERR_ARG;
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return DMFE_ERR_IO;
    bool ok = true;
    auto R = [&](void* p, size_t n) { ok = ok && std::fread(p, 1, n, f) == n; };
    char magic[8];
    int version = 0;
    dmfe_params p;
    R(magic, 8);
    R(&version, sizeof(int));
    R(&p, sizeof(p));
    if (!ok || std::memcmp(magic, kMagic, 8) != 0 || version != kCkpVersion || p.n_terms < 1 || p.n_terms > DMFE_MAX_TERMS) {
        std::fclose(f);
        return DMFE_ERR_IO;
    }
    std::vector<int> pw(p.n_terms);
    std::vector<double> cf(p.n_terms);
    DevState s;
    R(pw.data(), pw.size() * sizeof(int));
    R(cf.data(), cf.size() * sizeof(double));
    R(&s, sizeof(s));
    if (!ok || s.n < 1 || s.n > p.history_cap || p.L < 16 || p.L > 8192) {
        std::fclose(f);
        return DMFE_ERR_IO;
    }
    std::vector<double> ht(s.n);
    std::vector<dbl4> hist((size_t)s.n * p.L);
    R(ht.data(), ht.size() * sizeof(double));
    R(hist.data(), hist.size() * sizeof(dbl4));
    std::fclose(f);
    if (!ok) return DMFE_ERR_IO;
    p.powers = pw.data();
    p.coefs = cf.data();
    p.stream = stream;
    dmfe_solver* h = nullptr;
    int rc = dmfe_create(&p, &h);
    if (rc) return rc;
    s.active = 0;
    s.pending = 0;
    s.sp_ran = 0;
    s.sp_left = 0;
    *h->hstate = s;
    rc = DMFE_OK;
    if (cudaMemcpyAsync(h->v.hist[0], hist.data(), hist.size() * sizeof(dbl4), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->v.ht[0], ht.data(), ht.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        rc = DMFE_ERR_CUDA;
    if (!rc) rc = write_state(h);
    if (!rc) rc = launch_refresh_replica(h->v, h->stream);
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
    if (rc) {
        dmfe_destroy(h);
        return rc;
    }
    *out = h;
    return DMFE_OK;
}

}  // extern "C"
