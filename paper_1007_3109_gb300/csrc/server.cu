// Serving loop: continuous batching of simulation requests (declared in
// include/lb_rd.h as lb_rd_server_*, lb_rd_submit, lb_rd_poll).
//
// One worker thread per server owns the CUDA work.  Each iteration it
//   1. admits queued requests first-in first-out while slots are free and
//      their device memory fits the budget (stream-ordered allocation from
//      the device's memory pool, H2D copy of rho0, the init kernel),
//   2. advances every resident request by one tick of up to steps_per_tick
//      steps (never past the earliest finishing request): FP32 requests with
//      two state copies by K-step launches of the depth-K kernel over all
//      resident requests (K = 5 for D2Q9, 6 for D2Q5: the two-column form;
//      16-bit deviation storage its own kernel, K = 4) and one shorter
//      depth-K launch for the steps left (a single step if one is left),
//      other requests one batched launch per step; the tick's last launch
//      also writes their densities,
//   3. copies the results of finished requests to host memory, releases
//      their device memory and wakes pollers.
// Submit and poll only touch host state under the server mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lb_rd.h"
#include "lbrd_kernels.h"

namespace lbrd {
int report_error(int code, const std::string &msg);
}

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum ReqState { kQueued = 0, kActive = 1, kDone = 2 };

struct Request {
    uint64_t ticket = 0;
    lb_rd_config cfg{};
    std::vector<double> rho0;
    int64_t nsteps = 0, remaining = 0;
    int state = kQueued;
    int status = LB_RD_OK;
    int64_t arrival_ns = 0, start_ns = 0, end_ns = 0;
    // device side
    char *buf[2] = {nullptr, nullptr};
    char *rho = nullptr;
    int cur = 0;
    int64_t pitch = 0;
    size_t state_bytes = 0, rho_bytes = 0, need = 0;
    // results
    std::vector<double> rho_out;
    double mass[2] = {0.0, 0.0};
};

size_t request_bytes(const lb_rd_config &c, int Q, int64_t pitch, size_t *state_bytes, size_t *rho_bytes) {
    *state_bytes = lbrd::state_plane_bytes(c.precision, Q, c.nspecies, c.ny, pitch);
    *rho_bytes = (size_t)c.nspecies * c.ny * pitch * (c.precision == LB_RD_FP64 ? 8 : 4);
    const size_t copies = c.streaming == LB_RD_STREAM_INPLACE ? 1 : 2;
    return copies * *state_bytes + *rho_bytes;
}

}  // namespace

struct lb_rd_server {
    lb_rd_server_config cfg{};
    int Q = 0, mode = 0, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::map<uint64_t, Request *> all;
    size_t bytes_in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t pending = 0;  // submitted and not finished
    std::thread worker;
    // device work list
    lbrd::BatchItem *d_items = nullptr;
    lbrd::BatchItem *h_items = nullptr;  // pinned
    size_t items_cap = 0;
    lbrd::DeepItem *d_deep = nullptr;  // K-step descriptors, two parities
    lbrd::DeepItem *h_deep = nullptr;  // pinned
    size_t deep_cap = 0;
    double *partials = nullptr;
    unsigned int *counter = nullptr;
    double *d_mass = nullptr;
    size_t partials_cap = 0;
    int64_t launches = 0, ticks = 0, finished = 0;
    std::string worker_error;
};

namespace {

void finish(lb_rd_server *s, Request *r, int status) {
    std::lock_guard<std::mutex> lock(s->mu);
    r->status = status;
    r->state = kDone;
    r->end_ns = now_ns();
    s->pending--;
    s->finished++;
    s->cv_done.notify_all();
}

void release(lb_rd_server *s, Request *r) {
    if (r->buf[0]) cudaFreeAsync(r->buf[0], s->stream);
    if (r->buf[1]) cudaFreeAsync(r->buf[1], s->stream);
    if (r->rho) cudaFreeAsync(r->rho, s->stream);
    r->buf[0] = r->buf[1] = nullptr;
    r->rho = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    s->bytes_in_use -= r->need;
}

// Allocate and initialise an admitted request; false on failure (finished).
bool start_request(lb_rd_server *s, Request *r) {
    const lb_rd_config &c = r->cfg;
    cudaError_t e = cudaSuccess;
    double *stage = nullptr;
    const size_t n = (size_t)c.nspecies * c.ny * c.nx;
    if (!e) e = cudaMallocAsync((void **)&r->buf[0], r->state_bytes, s->stream);
    if (!e && c.streaming != LB_RD_STREAM_INPLACE) e = cudaMallocAsync((void **)&r->buf[1], r->state_bytes, s->stream);
    if (!e) e = cudaMallocAsync((void **)&r->rho, r->rho_bytes, s->stream);
    if (!e) e = cudaMallocAsync((void **)&stage, n * sizeof(double), s->stream);
    if (!e) e = cudaMemcpyAsync(stage, r->rho0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (!e) {
        lbrd::InitArgs a{};
        a.rho0 = stage;
        a.dst = r->buf[0];
        a.nx = c.nx;
        a.ny = c.ny;
        a.pitch = r->pitch;
        a.plane = c.ny * r->pitch;
        for (int k = 0; k < 2; ++k) a.omega[k] = k < c.nspecies ? 1.0 / c.tau[k] : 0.0;
        a.rkind = c.reaction.kind;
        a.kappa = c.reaction.kappa;
        a.F = c.reaction.F;
        a.k = c.reaction.k;
        a.rho_out = r->rho;
        e = lbrd::launch_batch_init(s->mode, s->Q, c.nspecies, a, s->stream);
    }
    if (stage) cudaFreeAsync(stage, s->stream);
    if (e) {
        release(s, r);
        finish(s, r, e == cudaErrorMemoryAllocation ? LB_RD_ENOMEM : LB_RD_ECUDA);
        return false;
    }
    r->cur = 0;
    r->remaining = r->nsteps;
    std::lock_guard<std::mutex> lock(s->mu);
    r->start_ns = now_ns();
    return true;
}

// Results of a finished request to the host, then release its memory.
int collect_request(lb_rd_server *s, Request *r) {
    const lb_rd_config &c = r->cfg;
    const size_t n = (size_t)c.nspecies * c.ny * c.nx;
    double *stage = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&stage, n * sizeof(double), s->stream);
    const int prec = c.precision == LB_RD_FP64 ? LB_RD_FP64 : LB_RD_FP32;  // density cache is float
    const size_t parts = lbrd::mass_partials_needed(c.nx, c.ny) * 2;
    if (!e && parts > s->partials_cap) {
        cudaFreeAsync(s->partials, s->stream);
        s->partials = nullptr;
        e = cudaMallocAsync((void **)&s->partials, parts * sizeof(double), s->stream);
        if (!e) s->partials_cap = parts;
    }
    if (!e) e = lbrd::launch_rho_export(prec, c.nspecies, r->rho, c.nx, c.ny, r->pitch, stage, s->stream);
    r->rho_out.resize(n);
    if (!e) e = cudaMemcpyAsync(r->rho_out.data(), stage, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (!e)
        e = lbrd::launch_mass(prec, c.nspecies, r->rho, c.nx, c.ny, r->pitch, s->partials, s->counter, s->d_mass,
                              s->stream);
    if (!e) e = cudaMemcpyAsync(r->mass, s->d_mass, c.nspecies * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (stage) cudaFreeAsync(stage, s->stream);
    if (!e) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LB_RD_OK : LB_RD_ECUDA;
}

int ensure_items(lb_rd_server *s, size_t n) {
    if (s->items_cap >= 3 * n) return LB_RD_OK;
    cudaStreamSynchronize(s->stream);
    cudaFree(s->d_items);
    cudaFreeHost(s->h_items);
    s->d_items = nullptr;
    s->h_items = nullptr;
    const size_t cap = 3 * std::max<size_t>(n, 64);
    if (cudaMalloc(&s->d_items, cap * sizeof(lbrd::BatchItem)) != cudaSuccess) return LB_RD_ENOMEM;
    if (cudaMallocHost(&s->h_items, cap * sizeof(lbrd::BatchItem)) != cudaSuccess) return LB_RD_ENOMEM;
    s->items_cap = cap;
    return LB_RD_OK;
}

int ensure_deep(lb_rd_server *s, size_t n) {
    if (s->deep_cap >= 3 * n) return LB_RD_OK;
    cudaStreamSynchronize(s->stream);
    cudaFree(s->d_deep);
    cudaFreeHost(s->h_deep);
    s->d_deep = nullptr;
    s->h_deep = nullptr;
    const size_t cap = 3 * std::max<size_t>(n, 64);
    if (cudaMalloc(&s->d_deep, cap * sizeof(lbrd::DeepItem)) != cudaSuccess) return LB_RD_ENOMEM;
    if (cudaMallocHost(&s->h_deep, cap * sizeof(lbrd::DeepItem)) != cudaSuccess) return LB_RD_ENOMEM;
    s->deep_cap = cap;
    return LB_RD_OK;
}

// The resident requests one tick advances: all of them, or with tick_sites
// > 0 those with the least remaining work (sites x steps left) first, as
// many as make up at least tick_sites sites together.
std::vector<Request *> pick_tick_set(const lb_rd_server *s) {
    std::vector<Request *> v = s->active;
    if (s->cfg.tick_sites <= 0 || v.size() < 2) return v;
    std::stable_sort(v.begin(), v.end(), [](const Request *a, const Request *b) {
        return (double)a->cfg.nx * (double)a->cfg.ny * (double)a->remaining <
               (double)b->cfg.nx * (double)b->cfg.ny * (double)b->remaining;
    });
    int64_t sites = 0;
    size_t k = 0;
    while (k < v.size() && sites < s->cfg.tick_sites) {
        sites += v[k]->cfg.nx * v[k]->cfg.ny;
        ++k;
    }
    v.resize(k);
    return v;
}

// Drops the finished requests from the resident list.
void prune_active(lb_rd_server *s) {
    std::vector<Request *> still;
    for (Request *r : s->active)
        if (r->state != kDone) still.push_back(r);
    s->active.swap(still);
}

void run_tick(lb_rd_server *s) {
    std::vector<Request *> act = pick_tick_set(s);
    const size_t n = act.size();
    int64_t tick = s->cfg.steps_per_tick;
    for (Request *r : act) tick = std::min(tick, r->remaining);
    if (ensure_items(s, n) != LB_RD_OK) {
        for (Request *r : act) {
            release(s, r);
            finish(s, r, LB_RD_ENOMEM);
        }
        prune_active(s);
        return;
    }
    // K-step launches: FP32 and 16-bit deviation requests with two state
    // copies run the tick as q = tick / K depth-K launches (FP32:
    // lbrd::batch_deep_default_k; 16-bit storage: lbrd::batch_half_default_k) and, for the r = tick % K
    // steps left, one
    // depth-r launch (r >= 2) or one single step (r = 1); the tick's last
    // launch writes the densities.  Other requests: one launch per step.
    bool any_inplace = false;
    for (Request *r : act) any_inplace = any_inplace || r->cfg.streaming == LB_RD_STREAM_INPLACE;
    bool v16 = true, v8 = true;  // every request has nx and pitch multiples of 4 (of 8)
    for (Request *r : act) v16 = v16 && r->cfg.nx % 4 == 0 && r->pitch % 4 == 0;
    for (Request *r : act) v8 = v8 && r->cfg.nx % 8 == 0 && r->pitch % 8 == 0;
    const bool half = s->mode == 1 || s->mode == 2;  // 16-bit deviation storage: its own depth-K kernels
    const int K = half ? lbrd::batch_half_default_k() : lbrd::batch_deep_default_k(s->Q);
    const bool deep = (s->mode == 0 || half) && !any_inplace && tick >= 2;
    int64_t n_multi = deep ? tick / K : 0;
    int rem = deep ? (int)(tick % K) : 0;  // steps of the depth-r launch (0: none)
    if (rem == 1) rem = 0;                 // one single step instead
    int64_t deep_units = 0, rem_units = 0;
    if ((n_multi > 0 || rem > 0) && ensure_deep(s, n) == LB_RD_OK) {
        for (size_t i = 0; i < n; ++i) {  // parity 0 relative to each request's current copy
            Request *r = act[i];
            const lb_rd_config &c = r->cfg;
            lbrd::DeepItem d{};
            d.a.nx = c.nx;
            d.a.ny = c.ny;
            d.a.pitch = r->pitch;
            d.a.plane = c.ny * r->pitch;
            for (int k = 0; k < 2; ++k) d.a.omega[k] = k < c.nspecies ? 1.0 / c.tau[k] : 0.0;
            d.a.rkind = c.reaction.kind;
            d.a.kappa = c.reaction.kappa;
            d.a.F = c.reaction.F;
            d.a.k = c.reaction.k;
            d.a.src = r->buf[r->cur];
            d.a.dst = r->buf[r->cur ^ 1];
            d.a.rho_out = r->rho;
            s->h_deep[i] = d;
        }
        if (rem > 0) {  // the depth-r launch follows the n_multi K-step launches
            const int par = (int)(n_multi & 1);
            for (size_t i = 0; i < n; ++i) {
                s->h_deep[2 * n + i] = s->h_deep[i];
                s->h_deep[2 * n + i].a.src = act[i]->buf[act[i]->cur ^ par];
                s->h_deep[2 * n + i].a.dst = act[i]->buf[act[i]->cur ^ par ^ 1];
            }
            rem_units = half ? lbrd::batch_half_deep_plan(rem, s->Q, s->cfg.nspecies, s->mode - 1, s->h_deep + 2 * n,
                                                          (int)n)
                             : lbrd::batch_deep_plan(rem, s->Q, s->cfg.nspecies, v16, s->h_deep + 2 * n, (int)n);
        }
        if (n_multi > 0)
            deep_units = half ? lbrd::batch_half_deep_plan(K, s->Q, s->cfg.nspecies, s->mode - 1, s->h_deep, (int)n)
                              : lbrd::batch_deep_plan(K, s->Q, s->cfg.nspecies, v16, s->h_deep, (int)n);
        for (size_t i = 0; i < n; ++i) {  // parity 1: the copies swapped
            s->h_deep[n + i] = s->h_deep[i];
            s->h_deep[n + i].a.src = act[i]->buf[act[i]->cur ^ 1];
            s->h_deep[n + i].a.dst = act[i]->buf[act[i]->cur];
        }
        if ((n_multi == 0 || deep_units > 0) && (rem == 0 || rem_units > 0))
            cudaMemcpyAsync(s->d_deep, s->h_deep, 3 * n * sizeof(lbrd::DeepItem), cudaMemcpyHostToDevice, s->stream);
    }
    if ((n_multi > 0 && deep_units <= 0) || (rem > 0 && rem_units <= 0)) {
        n_multi = 0;  // no plan: one launch per step
        rem = 0;
    }
    const int64_t n_single = tick - K * n_multi - rem;
    // launches of the tick: n_multi K-step launches, the depth-r launch, then
    // single steps; each launch swaps the two copies once
    const int64_t L = n_multi + (rem > 0 ? 1 : 0) + n_single;
    // descriptor sets: [0] even launches, [1] odd launches, [2] the tick's last launch (writes rho)
    int64_t total = 0;
    for (size_t i = 0; i < n; ++i) {
        Request *r = act[i];
        const lb_rd_config &c = r->cfg;
        lbrd::BatchItem it{};
        it.a.nx = c.nx;
        it.a.ny = c.ny;
        it.a.pitch = r->pitch;
        it.a.plane = c.ny * r->pitch;
        for (int k = 0; k < 2; ++k) it.a.omega[k] = k < c.nspecies ? 1.0 / c.tau[k] : 0.0;
        it.a.rkind = c.reaction.kind;
        it.a.kappa = c.reaction.kappa;
        it.a.F = c.reaction.F;
        it.a.k = c.reaction.k;
        it.tiles_x = lbrd::batch_tiles_x(c.nx);
        it.tile_begin = total;
        total += lbrd::batch_tiles(c.nx, c.ny);
        for (int set = 0; set < 3; ++set) {
            const int par = set < 2 ? (r->cur + set) & 1 : (int)((r->cur + L - 1) & 1);
            lbrd::BatchItem v = it;
            if (c.streaming == LB_RD_STREAM_INPLACE) {
                v.a.src = v.a.dst = r->buf[0];
                v.aa = (c.nx % 4 == 0 ? 1 : 3) + par;
            } else {
                v.a.src = r->buf[par];
                v.a.dst = r->buf[par ^ 1];
            }
            v.a.rho_out = set == 2 ? r->rho : nullptr;
            s->h_items[set * n + i] = v;
        }
    }
    cudaMemcpyAsync(s->d_items, s->h_items, 3 * n * sizeof(lbrd::BatchItem), cudaMemcpyHostToDevice, s->stream);
    cudaError_t e = cudaSuccess;
    const int S = s->cfg.nspecies;
    int rk = n > 0 ? act[0]->cfg.reaction.kind : -1;  // the reaction kind every request has, or -1
    for (Request *r : act) rk = r->cfg.reaction.kind == rk ? rk : -1;
    for (int64_t l = 0; l < L && !e; ++l) {
        if (l < n_multi) {
            e = half ? lbrd::launch_batch_half_deep(K, s->Q, S, s->mode - 1, s->d_deep + (l & 1) * n, (int)n,
                                                    deep_units, l == L - 1, rk, v8, s->stream)
                     : lbrd::launch_batch_deep(K, s->Q, S, v16, s->d_deep + (l & 1) * n, (int)n, deep_units,
                                               l == L - 1, rk, s->stream);
        } else if (l == n_multi && rem > 0) {
            e = half ? lbrd::launch_batch_half_deep(rem, s->Q, S, s->mode - 1, s->d_deep + 2 * n, (int)n, rem_units,
                                                    l == L - 1, rk, v8, s->stream)
                     : lbrd::launch_batch_deep(rem, s->Q, S, v16, s->d_deep + 2 * n, (int)n, rem_units, l == L - 1,
                                               rk, s->stream);
        } else {
            const lbrd::BatchItem *items = s->d_items + (l == L - 1 ? 2 : (l & 1)) * n;
            e = lbrd::launch_batch_step(any_inplace ? 4 : s->mode, s->Q, S, items, (int)n, total, s->stream);
        }
        s->launches++;
    }
    if (!e) e = cudaStreamSynchronize(s->stream);  // the pinned descriptors are reused next tick
    s->ticks++;
    for (Request *r : act) {
        if (e) {
            release(s, r);
            finish(s, r, LB_RD_ECUDA);
            continue;
        }
        r->cur = (int)((r->cur + L) & 1);
        r->remaining -= tick;
        if (r->remaining > 0) continue;
        const int st = collect_request(s, r);
        release(s, r);
        finish(s, r, st);
    }
    prune_active(s);
}

void worker_main(lb_rd_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request *> admit;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
            if (s->stop) break;
            // first-in first-out admission while slots and memory allow
            while (!s->queue.empty()) {
                Request *r = s->queue.front();
                if (r->need > s->cfg.hbm_budget_bytes) {  // can never fit
                    s->queue.pop_front();
                    r->status = LB_RD_ENOMEM;
                    r->state = kDone;
                    r->end_ns = now_ns();
                    s->pending--;
                    s->finished++;
                    s->cv_done.notify_all();
                    continue;
                }
                if ((int)(s->active.size() + admit.size()) >= s->cfg.max_slots ||
                    s->bytes_in_use + r->need > s->cfg.hbm_budget_bytes)
                    break;
                s->queue.pop_front();
                s->bytes_in_use += r->need;
                r->state = kActive;
                admit.push_back(r);
            }
        }
        for (Request *r : admit)
            if (start_request(s, r)) s->active.push_back(r);
        if (s->active.empty()) continue;
        run_tick(s);
    }
}

}  // namespace

extern "C" {

int lb_rd_server_create(const lb_rd_server_config *cfg, lb_rd_server **out) {
    if (!cfg || !out) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_create: NULL argument");
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->steps_per_tick < 1 || cfg->hbm_budget_bytes == 0 || cfg->tick_sites < 0)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_create: need max_slots >= 1, steps_per_tick >= 1, "
                                                "budget > 0, tick_sites >= 0");
    if (cfg->lattice != LB_RD_D2Q9 && cfg->lattice != LB_RD_D2Q5)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_create: unknown lattice");
    if (cfg->nspecies < 1 || cfg->nspecies > 2)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_create: nspecies must be 1 or 2");
    if (cfg->precision < LB_RD_FP64 || cfg->precision > LB_RD_FP32_FP16DEV)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_create: unknown precision");
    lb_rd_server *s = new lb_rd_server();
    s->cfg = *cfg;
    s->Q = cfg->lattice == LB_RD_D2Q9 ? 9 : 5;
    s->mode = lbrd::batch_mode(cfg->precision);
    cudaError_t e = cudaGetDevice(&s->device);
    if (!e) {
        if (cfg->stream) {
            s->stream = static_cast<cudaStream_t>(cfg->stream);
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = true;
        }
    }
    // keep freed request memory in the device pool for the next admission
    cudaMemPool_t pool;
    if (!e && cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = cfg->hbm_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->partials_cap = lbrd::mass_partials_needed(4096, 4096) * 2;
    if (!e) e = cudaMalloc(&s->partials, s->partials_cap * sizeof(double));
    if (!e) e = cudaMalloc(&s->counter, sizeof(unsigned int));
    if (!e) e = cudaMemset(s->counter, 0, sizeof(unsigned int));
    if (!e) e = cudaMalloc(&s->d_mass, 2 * sizeof(double));
    if (e) {
        cudaFree(s->partials);
        cudaFree(s->counter);
        cudaFree(s->d_mass);
        if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return lbrd::report_error(LB_RD_ECUDA, std::string("lb_rd_server_create: ") + cudaGetErrorString(e));
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LB_RD_OK;
}

int lb_rd_server_destroy(lb_rd_server *s) {
    if (!s) return LB_RD_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (Request *r : s->active) {
        if (r->buf[0]) cudaFreeAsync(r->buf[0], s->stream);
        if (r->buf[1]) cudaFreeAsync(r->buf[1], s->stream);
        if (r->rho) cudaFreeAsync(r->rho, s->stream);
    }
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->all) delete kv.second;
    cudaFree(s->d_items);
    cudaFreeHost(s->h_items);
    cudaFree(s->d_deep);
    cudaFreeHost(s->h_deep);
    cudaFree(s->partials);
    cudaFree(s->counter);
    cudaFree(s->d_mass);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return LB_RD_OK;
}

int lb_rd_submit(lb_rd_server *s, const lb_rd_config *cfg, const double *rho0, int64_t nsteps, uint64_t *ticket) {
    if (!s || !cfg || !rho0 || !ticket) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: NULL argument");
    int rc = lb_rd_check_config(cfg, nullptr);
    if (rc) return rc;
    if (cfg->lattice != s->cfg.lattice || cfg->nspecies != s->cfg.nspecies || cfg->precision != s->cfg.precision)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: lattice, nspecies and precision must match the server");
    if (cfg->reaction.kind == LB_RD_REACTION_MASS_ACTION)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: serving takes no mass-action network");
    if (cfg->streaming == LB_RD_STREAM_INPLACE && cfg->precision != LB_RD_FP32)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: in-place requests need FP32 storage");
    if ((s->mode == 1 || s->mode == 2) && cfg->nx % 4)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: 16-bit deviation storage needs nx % 4 == 0");
    if (nsteps < 1) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_submit: nsteps must be >= 1");
    Request *r = new Request();
    r->cfg = *cfg;
    const size_t n = (size_t)cfg->nspecies * cfg->ny * cfg->nx;
    r->rho0.assign(rho0, rho0 + n);
    r->nsteps = nsteps;
    r->pitch = (cfg->nx + 31) / 32 * 32;
    r->need = request_bytes(*cfg, s->Q, r->pitch, &r->state_bytes, &r->rho_bytes);
    r->arrival_ns = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
        s->pending++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return LB_RD_OK;
}

int lb_rd_poll(lb_rd_server *s, uint64_t ticket, double *rho_out, double *mass_out, lb_rd_request_stats *stats) {
    if (!s) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_poll: server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return lbrd::report_error(LB_RD_ENOTFOUND, "lb_rd_poll: unknown or collected ticket");
    Request *r = it->second;
    if (stats) {
        stats->arrival_ns = r->arrival_ns;
        stats->start_ns = r->start_ns;
        stats->end_ns = r->end_ns;
        stats->steps = r->nsteps;
        stats->status = r->state == kDone ? r->status : LB_RD_EPENDING;
    }
    if (r->state != kDone) return LB_RD_EPENDING;
    const int status = r->status;
    if (status == LB_RD_OK) {
        if (rho_out) std::memcpy(rho_out, r->rho_out.data(), r->rho_out.size() * sizeof(double));
        if (mass_out) std::memcpy(mass_out, r->mass, r->cfg.nspecies * sizeof(double));
    }
    s->all.erase(it);
    delete r;
    if (status != LB_RD_OK)
        return lbrd::report_error(status, "lb_rd_poll: request failed (" + std::to_string(status) + ")");
    return LB_RD_OK;
}

int lb_rd_server_drain(lb_rd_server *s, int64_t timeout_ms) {
    if (!s) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_drain: server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] { return s->pending == 0; });
    return ok ? LB_RD_OK : lbrd::report_error(LB_RD_ETIMEOUT, "lb_rd_server_drain: requests still pending");
}

int lb_rd_server_stats(const lb_rd_server *s, int64_t *launches, int64_t *ticks, int64_t *finished) {
    if (!s) return lbrd::report_error(LB_RD_EINVAL, "lb_rd_server_stats: server is NULL");
    if (launches) *launches = s->launches;
    if (ticks) *ticks = s->ticks;
    if (finished) *finished = s->finished;
    return LB_RD_OK;
}

}  // extern "C"
