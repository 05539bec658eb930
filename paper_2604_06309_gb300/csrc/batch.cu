// Batched solves: a table of slots in device memory, one captured graph per batched
// Runge-Kutta step (slots may be in Dormand-Prince or SSPRK(10,4) steps), admission and
// release of slots between steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dmfe_internal.h"
#include "hi_units.h"

struct dmfe_batch {
    int max_slots = 0, max_L = 0, max_cap = 0, precision = 0, s = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<dmfe_solver*> slots;
    std::vector<int> finished;  // 1: done or failed (no more work)
    BatchTable* h_table = nullptr;  // pinned
    BatchTable* d_table = nullptr;
    bool dirty = true;
    cudaGraphExec_t exec = nullptr;
    int hi_grid = 0;
    size_t hi_smem = 0;
    DevState* h_state = nullptr;  // pinned, one per slot
    DevState* d_state = nullptr;  // device copies gathered by one kernel per poll
};

namespace {

#define TRYB(x)                \
    do {                       \
        int rc_ = (x);         \
        if (rc_) return rc_;   \
    } while (0)

void rebuild_table(dmfe_batch* b) {
    BatchTable& t = *b->h_table;
    int count = 0;
    for (int k = 0; k < b->max_slots; ++k)
        if (b->slots[k]) count = k + 1;
    t.count = count;
    long long off = 0, woff = 0;
    for (int k = 0; k < b->max_slots; ++k) {
        t.uoff[k] = off;
        t.woff[k] = woff;
        dmfe_solver* h = b->slots[k];
        t.active[k] = h ? 1 : 0;
        if (h) {
            const SolverView& v = solver_view(h);
            t.views[k] = v;
            if (!b->finished[k]) {
                off += (long long)hi_parts(v.L, v.hi_chunk) * v.L;
                woff += (long long)v.L * v.L;
            }
        }
    }
    t.uoff[b->max_slots] = off;
    t.woff[b->max_slots] = woff;
    for (int k = count; k <= b->max_slots && k > 0; ++k) {
        t.uoff[k] = off;
        t.woff[k] = woff;
    }
    b->dirty = true;
}

// Copy every present slot's device state word block into one array, so that a poll is one
// launch and one transfer instead of a transfer per slot.
__global__ void k_gather_states(const BatchTable* __restrict__ bt, DevState* __restrict__ out) {
    const int k = blockIdx.x;
    if (k >= bt->count || !bt->active[k]) return;
    static_assert(sizeof(DevState) % 8 == 0, "state size");
    const long long* src = reinterpret_cast<const long long*>(bt->views[k].st);
    long long* dst = reinterpret_cast<long long*>(out + k);
    for (int q = threadIdx.x; q < (int)(sizeof(DevState) / 8); q += blockDim.x) dst[q] = src[q];
}

int upload_table(dmfe_batch* b) {
    if (!b->dirty) return DMFE_OK;
    DMFE_CUDA_TRY(cudaMemcpyAsync(b->d_table, b->h_table, sizeof(BatchTable), cudaMemcpyHostToDevice, b->stream));
    b->dirty = false;
    return DMFE_OK;
}

struct BatchParts : StepParts {
    const dmfe_batch* b;
    explicit BatchParts(const dmfe_batch* bb) : b(bb) {}
    int head(cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) override {
        return launch_batch_step_head(b->d_table, b->precision, b->s, b->max_L, b->max_cap, b->max_slots,
                                      b->hi_grid, b->hi_smem, cond, use_cond, s);
    }
    int tail(cudaStream_t s) override {
        return launch_batch_step_tail(b->d_table, b->precision, b->s, b->max_L, b->max_cap, b->max_slots,
                                      b->hi_grid, b->hi_smem, s);
    }
    int sp(cudaStream_t s) override { return launch_batch_step_sparsify(b->d_table, b->max_cap, b->max_slots, s); }
};

int build_graph(dmfe_batch* b) {
    if (b->exec) return DMFE_OK;
    BatchParts parts(b);
    if (!step_graph_plain() && capture_step_graph(b->cap_stream, true, parts, &b->exec) == DMFE_OK) return DMFE_OK;
    return capture_step_graph(b->cap_stream, false, parts, &b->exec);
}

}  // namespace

extern "C" {

int dmfe_batch_create(int max_slots, int max_L, int max_cap, int precision, int s, void* stream,
                      dmfe_batch** out) {
    if (!out) return DMFE_ERR_ARG;
    *out = nullptr;
    if (max_slots < 1 || max_slots > kMaxSlots || max_L < 16 || max_L > 8192 || max_cap < 16) return DMFE_ERR_ARG;
    if (precision != DMFE_FP64 && precision != DMFE_FP32_COMPENSATED && precision != DMFE_DOUBLE_FLOAT)
        return DMFE_ERR_ARG;
    dmfe_batch* b = new (std::nothrow) dmfe_batch();
    if (!b) return DMFE_ERR_OOM;
    b->max_slots = max_slots;
    b->max_L = max_L;
    b->max_cap = max_cap;
    b->precision = precision;
    b->s = s;
    b->slots.assign(max_slots, nullptr);
    b->finished.assign(max_slots, 0);
    int rc = batch_hi_config(precision, s, max_L, max_cap, &b->hi_grid, &b->hi_smem);
    if (!rc) {
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
            b->own_stream = true;
        } else {
            rc = DMFE_ERR_CUDA;
        }
    }
    if (!rc && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) rc = DMFE_ERR_CUDA;
    if (!rc && cudaMallocHost((void**)&b->h_table, sizeof(BatchTable)) != cudaSuccess) rc = DMFE_ERR_OOM;
    if (!rc && cudaMallocHost((void**)&b->h_state, sizeof(DevState) * max_slots) != cudaSuccess) rc = DMFE_ERR_OOM;
    if (!rc && cudaMalloc((void**)&b->d_table, sizeof(BatchTable)) != cudaSuccess) rc = DMFE_ERR_OOM;
    if (!rc && cudaMalloc((void**)&b->d_state, sizeof(DevState) * max_slots) != cudaSuccess) rc = DMFE_ERR_OOM;
    if (rc) {
        cudaGetLastError();
        dmfe_batch_destroy(b);
        return rc;
    }
    std::memset(b->h_table, 0, sizeof(BatchTable));
    rebuild_table(b);
    *out = b;
    return DMFE_OK;
}

void dmfe_batch_destroy(dmfe_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (dmfe_solver* h : b->slots)
        if (h) dmfe_destroy(h);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_table) cudaFree(b->d_table);
    if (b->d_state) cudaFree(b->d_state);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int dmfe_batch_add(dmfe_batch* b, const dmfe_params* p, double t_max, double tol, int* slot) {
    if (!b || !p) return DMFE_ERR_ARG;
    const int cap = p->history_cap ? p->history_cap : p->L;
    if (p->precision != b->precision || p->s != b->s || p->L > b->max_L || cap > b->max_cap) return DMFE_ERR_ARG;
    if (!(tol > 0.0) || !(t_max <= p->grid_t_max * (1.0 + 1e-12))) return DMFE_ERR_ARG;
    // the batched kernel is compiled without the log-R reads (they cost it registers)
    if (p->log_r) return DMFE_ERR_UNSUPPORTED;
    // one copy of the pass kernels per batched step graph: one pass per round
    if (p->sparsify_passes > 1) return DMFE_ERR_UNSUPPORTED;
    int k = 0;
    while (k < b->max_slots && b->slots[k]) ++k;
    if (k == b->max_slots) return DMFE_ERR_CAPACITY;
    dmfe_params q = *p;
    q.stream = b->stream;
    // one unit per output index unless asked otherwise: a batch has parallelism across
    // slots, and larger units carry less per-unit reduction overhead
    if (q.hi_chunk <= 0) q.hi_chunk = q.L;  // (the flat split is for single solves)
    dmfe_solver* h = nullptr;
    TRYB(dmfe_create(&q, &h));
    const int rc = launch_begin_integrate(solver_view(h), t_max, tol, b->stream);
    if (rc) {
        dmfe_destroy(h);
        return rc;
    }
    b->slots[k] = h;
    b->finished[k] = 0;
    rebuild_table(b);
    if (slot) *slot = k;
    return DMFE_OK;
}

int dmfe_batch_remove(dmfe_batch* b, int slot) {
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot]) return DMFE_ERR_ARG;
    DMFE_CUDA_TRY(cudaStreamSynchronize(b->stream));
    dmfe_destroy(b->slots[slot]);
    b->slots[slot] = nullptr;
    b->finished[slot] = 0;
    rebuild_table(b);
    return DMFE_OK;
}

dmfe_solver* dmfe_batch_solver(dmfe_batch* b, int slot) {
    if (!b || slot < 0 || slot >= b->max_slots) return nullptr;
    return b->slots[slot];
}

int dmfe_batch_step(dmfe_batch* b, int nsteps) {
    if (!b || nsteps < 0) return DMFE_ERR_ARG;
    TRYB(upload_table(b));
    TRYB(build_graph(b));
    for (int it = 0; it < nsteps; ++it) DMFE_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    return DMFE_OK;
}

// Work-unit sizes the batch autotuner tries for every slot (0: one unit per output index).
static const int kBatchTuneChunks[DMFE_BATCH_TUNE_CANDIDATES] = {0, 256, 512, 1024, 2048};

int dmfe_batch_autotune(dmfe_batch* b, int steps, int* chunk, double* ms_per_step) {
    if (!b || steps < 1) return DMFE_ERR_ARG;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DMFE_CUDA_TRY(cudaEventCreate(&e0));
    DMFE_CUDA_TRY(cudaEventCreate(&e1));
    double best_ms[DMFE_BATCH_TUNE_CANDIDATES];
    for (double& x : best_ms) x = 1e300;
    auto apply = [&](int c) {
        for (dmfe_solver* h : b->slots)
            if (h) {
                const int L = solver_view(h).L;
                solver_set_chunk(h, (c == 0 || c >= L) ? L : c);
            }
        rebuild_table(b);
    };
    int rc = DMFE_OK;
    // two interleaved rounds, the best of each candidate kept: the histories grow while the
    // candidates are timed, and interleaving keeps that drift from favouring one of them
    for (int round = 0; round < 2 && rc == DMFE_OK; ++round) {
        for (int q = 0; q < DMFE_BATCH_TUNE_CANDIDATES && rc == DMFE_OK; ++q) {
            apply(kBatchTuneChunks[q]);
            rc = upload_table(b);
            if (!rc) rc = build_graph(b);
            if (rc) break;
            cudaEventRecord(e0, b->stream);
            for (int it = 0; it < steps; ++it)
                if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) rc = DMFE_ERR_CUDA;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = DMFE_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms[q] = std::min(best_ms[q], (double)ms / steps);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    int best = 0;
    for (int q = 1; q < DMFE_BATCH_TUNE_CANDIDATES; ++q)
        if (best_ms[q] < best_ms[best]) best = q;
    apply(kBatchTuneChunks[best]);
    if (chunk) *chunk = kBatchTuneChunks[best];
    if (ms_per_step)
        for (int q = 0; q < DMFE_BATCH_TUNE_CANDIDATES; ++q) ms_per_step[q] = best_ms[q];
    return DMFE_OK;
}

int dmfe_batch_poll(dmfe_batch* b, int* status, double* t, int* running) {
    if (!b) return DMFE_ERR_ARG;
    TRYB(upload_table(b));
    const int count = b->h_table->count;
    if (count > 0) {
        k_gather_states<<<count, 32, 0, b->stream>>>(b->d_table, b->d_state);
        DMFE_CUDA_TRY(cudaGetLastError());
        DMFE_CUDA_TRY(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(DevState) * count, cudaMemcpyDeviceToHost,
                                      b->stream));
    }
    DMFE_CUDA_TRY(cudaStreamSynchronize(b->stream));
    int run = 0;
    bool changed = false;
    for (int k = 0; k < b->max_slots; ++k) {
        int st = -100;
        double tk = 0.0;
        if (b->slots[k]) {
            const DevState& d = b->h_state[k];
            tk = d.t;
            st = d.status ? d.status : (d.done ? 1 : 0);
            const int fin = st != 0;
            if (fin != b->finished[k]) {
                b->finished[k] = fin;
                changed = true;
            }
            if (!fin) ++run;
        }
        if (status) status[k] = st;
        if (t) t[k] = tk;
    }
    if (changed) rebuild_table(b);
    if (running) *running = run;
    return DMFE_OK;
}

}  // extern "C"
