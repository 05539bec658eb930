// Serving loop over a batch: a worker thread admits queued requests (first in, first out)
// into free slots while their summed device footprint fits the budget, steps the batch
// and retires finished solves with their timestamps. Requests that arrive while others
// run join at the next round: continuous batching.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "dmfe_internal.h"

namespace {

struct Request {
    long long id = 0;
    dmfe_params p{};
    std::vector<int> pw;
    std::vector<double> cf;
    double t_max = 0.0, tol = 0.0;
    double submit_s = 0.0, admit_s = 0.0;
    unsigned long long bytes = 0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct dmfe_server {
    dmfe_batch* batch = nullptr;
    int max_slots = 0, max_L = 0, max_cap = 0, precision = 0, s = 0, steps_per_round = 1;
    unsigned long long budget = 0, in_use = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<dmfe_result> results;
    std::vector<Request> running;  // per slot
    std::vector<char> occupied;
    std::thread worker;
    std::atomic<bool> stop{false};
    long long next_id = 1;
    dmfe_server_stats_t st{};
    int worker_status = DMFE_OK;
    int device = 0;
};

namespace {

void retire(dmfe_server* srv, int k, int status) {
    dmfe_solver* h = dmfe_batch_solver(srv->batch, k);
    dmfe_result r{};
    r.id = srv->running[k].id;
    r.status = status == 1 ? 0 : status;
    r.slot = k;
    r.submit_s = srv->running[k].submit_s;
    r.admit_s = srv->running[k].admit_s;
    double t = 0.0, mu = 0.0, E = 0.0;
    if (h && dmfe_get_row(h, &t, nullptr, nullptr, &mu, &E) == DMFE_OK) {
        r.t_final = t;
        r.mu = mu;
        r.E = E;
    }
    dmfe_stats_t ss{};
    if (h && dmfe_stats(h, &ss) == DMFE_OK) {
        r.steps_accepted = ss.steps_accepted;
        r.steps_rejected = ss.steps_rejected;
    }
    dmfe_batch_remove(srv->batch, k);
    r.done_s = now_s(srv->t0);
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->occupied[k] = 0;
    srv->in_use -= srv->running[k].bytes;
    srv->results.push_back(r);
    if (r.status == 0) srv->st.completed += 1; else srv->st.failed += 1;
    srv->st.running -= 1;
}

void worker_loop(dmfe_server* srv) {
    cudaSetDevice(srv->device);
    std::vector<int> status(srv->max_slots);
    std::vector<double> tt(srv->max_slots);
    while (!srv->stop.load()) {
        // admission: first in, first out, while a slot and the footprint budget allow
        for (;;) {
            Request rq;
            int k = -1;
            {
                std::lock_guard<std::mutex> lock(srv->mu);
                if (srv->queue.empty()) break;
                for (int j = 0; j < srv->max_slots; ++j)
                    if (!srv->occupied[j]) { k = j; break; }
                if (k < 0 || srv->in_use + srv->queue.front().bytes > srv->budget) break;
                rq = std::move(srv->queue.front());
                srv->queue.pop_front();
                srv->occupied[k] = 1;
                srv->in_use += rq.bytes;
            }
            rq.p.powers = rq.pw.data();
            rq.p.coefs = rq.cf.data();
            int slot = -1;
            const int rc = dmfe_batch_add(srv->batch, &rq.p, rq.t_max, rq.tol, &slot);
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->occupied[k] = 0;
            if (rc) {
                srv->in_use -= rq.bytes;
                dmfe_result r{};
                r.id = rq.id;
                r.status = rc;
                r.slot = -1;
                r.submit_s = rq.submit_s;
                r.admit_s = r.done_s = now_s(srv->t0);
                srv->results.push_back(r);
                srv->st.failed += 1;
                continue;
            }
            rq.admit_s = now_s(srv->t0);
            srv->occupied[slot] = 1;
            srv->running[slot] = std::move(rq);
            srv->st.admitted += 1;
            srv->st.running += 1;
        }
        int nrun = 0;
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            nrun = srv->st.running;
        }
        if (nrun == 0) {
            std::unique_lock<std::mutex> lock(srv->mu);
            srv->cv.wait_for(lock, std::chrono::milliseconds(1));
            continue;
        }
        int rc = dmfe_batch_step(srv->batch, srv->steps_per_round);
        int running = 0;
        if (!rc) rc = dmfe_batch_poll(srv->batch, status.data(), tt.data(), &running);
        if (rc) {
            srv->worker_status = rc;
            break;
        }
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->st.batched_steps += srv->steps_per_round;
        }
        for (int k = 0; k < srv->max_slots; ++k)
            if (status[k] != -100 && status[k] != 0) retire(srv, k, status[k]);
    }
}

}  // namespace

extern "C" {

int dmfe_server_start(int max_slots, int max_L, int max_cap, int precision, int s,
                      unsigned long long hbm_budget, int steps_per_round, dmfe_server** out) {
    if (!out || steps_per_round < 1 || hbm_budget == 0) return DMFE_ERR_ARG;
    *out = nullptr;
    dmfe_server* srv = new (std::nothrow) dmfe_server();
    if (!srv) return DMFE_ERR_OOM;
    const int rc = dmfe_batch_create(max_slots, max_L, max_cap, precision, s, nullptr, &srv->batch);
    if (rc) {
        delete srv;
        return rc;
    }
    srv->max_slots = max_slots;
    srv->max_L = max_L;
    srv->max_cap = max_cap;
    srv->precision = precision;
    srv->s = s;
    srv->budget = hbm_budget;
    srv->steps_per_round = steps_per_round;
    srv->running.resize(max_slots);
    srv->occupied.assign(max_slots, 0);
    srv->st.hbm_budget = hbm_budget;
    srv->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&srv->device);
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return DMFE_OK;
}

int dmfe_server_submit(dmfe_server* srv, const dmfe_params* p, double t_max, double tol, long long* id) {
    if (!srv || !p || p->n_terms < 1 || p->n_terms > DMFE_MAX_TERMS || !p->powers || !p->coefs) return DMFE_ERR_ARG;
    const int cap = p->history_cap ? p->history_cap : p->L;
    if (p->precision != srv->precision || p->s != srv->s || p->L > srv->max_L || cap > srv->max_cap) return DMFE_ERR_ARG;
    if (!(tol > 0.0) || !(t_max <= p->grid_t_max * (1.0 + 1e-12))) return DMFE_ERR_ARG;
    if (p->log_r) return DMFE_ERR_UNSUPPORTED;  // as dmfe_batch_add
    if (p->sparsify_passes > 1) return DMFE_ERR_UNSUPPORTED;
    Request rq;
    rq.p = *p;
    rq.pw.assign(p->powers, p->powers + p->n_terms);
    rq.cf.assign(p->coefs, p->coefs + p->n_terms);
    rq.t_max = t_max;
    rq.tol = tol;
    rq.bytes = dmfe_footprint(p);
    if (rq.bytes == 0 || rq.bytes > srv->budget) return DMFE_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    rq.id = srv->next_id++;
    rq.submit_s = now_s(srv->t0);
    if (id) *id = rq.id;
    srv->queue.push_back(std::move(rq));
    srv->st.submitted += 1;
    srv->cv.notify_one();
    return DMFE_OK;
}

int dmfe_server_poll(dmfe_server* srv, dmfe_result* out, int max_out, int* n) {
    if (!srv || !n || max_out < 0 || (max_out > 0 && !out)) return DMFE_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    const int m = (int)srv->results.size() < max_out ? (int)srv->results.size() : max_out;
    for (int i = 0; i < m; ++i) out[i] = srv->results[i];
    srv->results.erase(srv->results.begin(), srv->results.begin() + m);
    *n = m;
    return srv->worker_status;
}

int dmfe_server_stats(dmfe_server* srv, dmfe_server_stats_t* out) {
    if (!srv || !out) return DMFE_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    *out = srv->st;
    out->queued = (int)srv->queue.size();
    out->bytes_in_use = srv->in_use;
    return srv->worker_status;
}

int dmfe_server_stop(dmfe_server* srv) {
    if (!srv) return DMFE_ERR_ARG;
    srv->stop.store(true);
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    const int rc = srv->worker_status;
    dmfe_batch_destroy(srv->batch);
    delete srv;
    return rc;
}

}  // extern "C"
