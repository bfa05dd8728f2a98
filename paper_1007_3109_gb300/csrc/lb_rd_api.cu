// C ABI of the single-simulation path (declared in include/lb_rd.h).
//
// A handle owns two copies of the post-collision state f*(t) (ping-pong), the
// density cache rho(t) written by the last kernel that advanced it, the FP64
// mass buffers and a lazily allocated FP64 staging buffer for host transfers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lb_rd.h"
#include "lbrd_kernels.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? LB_RD_ENOMEM : LB_RD_ECUDA, m);
}

#define LBRD_CUDA(call, what)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int64_t kMaxSide = 65535;

int lattice_q(int lattice) { return lattice == LB_RD_D2Q9 ? 9 : (lattice == LB_RD_D2Q5 ? 5 : 0); }

int64_t pitch_for(int64_t nx) { return lbrd::state_pitch(nx); }

size_t rho_elem(int prec) { return prec == LB_RD_FP64 ? 8 : 4; }

// Configurations the specialised kernels do not cover run the general kernel
// (one thread per site, up to four species, mass-action networks).
bool needs_general(const lb_rd_config &c) {
    return c.nspecies > 2 || c.reaction.kind == LB_RD_REACTION_MASS_ACTION;
}

}  // namespace

namespace lbrd {
// Error reporting for entry points defined in other translation units.
int report_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace lbrd

struct lb_rd_handle {
    lb_rd_config cfg{};
    int Q = 0, S = 0, prec = 0;
    int64_t pitch = 0, plane = 0;
    size_t state_bytes = 0, rho_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    void *rho = nullptr;
    double *stage = nullptr;
    size_t stage_elems = 0;
    double *partials = nullptr;
    unsigned int *counter = nullptr;
    double *mass = nullptr;
    int *status = nullptr;  // device error word of the step kernels (bounded waits)
    bool mass_fresh = false;
    bool initialized = false;
    int64_t t = 0;
    int64_t rho_t = -1;  // time the density cache holds (recomputed on demand)
    cudaStream_t stream = nullptr;
    bool timing = false;
    std::vector<cudaEvent_t> events;  // start/stop pairs of timed step kernels
    int64_t launches = 0;
    int inject_timeout = 0;  // one-shot test switch for the bounded-wait error path
    int variant = 0;      // single-step launch variant of the step kernel
    int tb_variant = -1;  // multi-step (temporal blocking, K steps per launch) variant, or -1
    // depth-K variants per steps per launch d = 2 .. 8 (-1: none fits) and, once
    // tuned, their time per step (ms): the launches that cover the last steps of a call
    int depth_variant[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    double depth_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool depth_tuned = false;
    std::vector<int> event_steps;    // steps of each timed launch (events[2i], events[2i + 1])
    std::vector<int> event_variant;  // and its launch variant
    bool general = false; // runs the general kernel
    bool inplace = false; // one state copy, AA pattern (buf[1] unused)
};

namespace {
// Autotuner choices per (device, precision, Q, S, nx, ny): single-step
// variant, multi-step variant (-1 if none is faster) and the fastest depth-K
// variant with its time per step for every d = 2 .. 8.
struct TuneEntry {
    int variant = 0, tb_variant = -1;
    int depth_variant[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    double depth_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int64_t, int64_t>, TuneEntry> g_tune_cache;

std::tuple<int, int, int, int, int64_t, int64_t> tune_key(const lb_rd_handle *h) {
    int dev = 0;
    cudaGetDevice(&dev);
    return std::make_tuple(dev, h->prec + (h->general ? 16 : 0) + (h->inplace ? 32 : 0), h->Q, h->S, h->cfg.nx,
                           h->cfg.ny);
}

int variant_count(int prec) {
    return prec == LB_RD_FP32 ? lbrd::kF32VariantCount : (prec == LB_RD_FP64 ? 1 : lbrd::kHalfVariantCount);
}

int handle_variant_count(const lb_rd_handle *h) {
    if (h->inplace) return h->prec == LB_RD_FP64 ? 1 : lbrd::kAAVariantCount;
    if (h->general) return h->prec == LB_RD_FP64 ? 1 : lbrd::kGeneralVariantCount;
    return variant_count(h->prec);
}

bool is_half(const lb_rd_handle *h) { return h->prec == LB_RD_FP32_BF16DEV || h->prec == LB_RD_FP32_FP16DEV; }

int variant_steps(const lb_rd_handle *h, int v) {
    if (h->general || h->inplace || v < 0) return 1;
    if (h->prec == LB_RD_FP32) return lbrd::kF32Variants[v].steps;
    return is_half(h) ? lbrd::kHalfVariantSteps[v] : 1;
}

bool variant_fits(const lb_rd_handle *h, int v) {
    if (h->inplace) return h->prec == LB_RD_FP64 || h->cfg.nx % lbrd::kAAVariants[v].sites == 0;
    if (h->general) return h->prec == LB_RD_FP64 || h->cfg.nx % lbrd::kGeneralVariants[v].sites == 0;
    if (is_half(h)) return h->cfg.nx % lbrd::kHalfVariantNx[v] == 0;
    return h->prec != LB_RD_FP32 || h->cfg.nx % lbrd::kF32Variants[v].nx_multiple == 0;
}

// A variant of a depth-K kernel (it can write the densities of its last level):
// the FP32 ones and the 16-bit deviation ones of two or more steps.
bool is_deep(const lb_rd_handle *h, int v) {
    if (h->general || h->inplace || v < 0) return false;
    if (h->prec == LB_RD_FP32) return lbrd::kF32Variants[v].cache == 4;
    return is_half(h) && lbrd::kHalfVariantSteps[v] >= 2;
}

// Untuned depth table: per d = 2 .. 8 the first depth-K variant of d steps
// that fits the grid, in table order.
void default_depths(lb_rd_handle *h) {
    for (int d = 0; d < 9; ++d) {
        h->depth_variant[d] = -1;
        h->depth_ms[d] = 0.0;
    }
    h->depth_tuned = false;
    for (int v = 0; v < handle_variant_count(h); ++v) {
        const int d = variant_steps(h, v);
        if (is_deep(h, v) && d >= 2 && d <= 8 && h->depth_variant[d] < 0 && variant_fits(h, v))
            h->depth_variant[d] = v;
    }
}

void apply_tune(lb_rd_handle *h, const TuneEntry &t) {
    h->variant = t.variant;
    h->tb_variant = t.tb_variant;
    bool tuned = false;
    for (int d = 0; d < 9; ++d) {
        if (t.depth_variant[d] >= 0) h->depth_variant[d] = t.depth_variant[d];
        h->depth_ms[d] = t.depth_ms[d];
        tuned = tuned || t.depth_ms[d] > 0.0;
    }
    h->depth_tuned = tuned;
}

// Launches of one lb_rd_step call: `bulk` launches of K steps, then the
// launches of `tail` (steps per launch, largest first).  With a depth-K
// variant the last r + K min(q, 4) steps (nsteps = q K + r) are split by
// dynamic programming over d = 1 .. K steps per launch, each d at the time of
// its fastest variant (the autotuner's figures, else a fixed relative table
// of the depth sweep's shape), so that a call of any length runs close to the
// per-step rate of the deepest launches and ends on a launch that also writes
// rho.  Other multi-step variants (two-step kernels, which cannot write rho)
// keep the last step single, like one-step variants.
struct LaunchPlan {
    int64_t bulk = 0;
    int K = 1;
    std::vector<int> tail;
};

LaunchPlan plan_launches(const lb_rd_handle *h, int64_t nsteps) {
    LaunchPlan p;
    if (nsteps <= 0) return p;
    const int K = h->tb_variant >= 0 ? variant_steps(h, h->tb_variant) : 1;
    if (K == 1 || !is_deep(h, h->tb_variant)) {
        p.K = K;
        p.bulk = K > 1 ? (nsteps - 1) / K : 0;
        for (int64_t n = nsteps - K * p.bulk; n > 0; --n) p.tail.push_back(1);
        return p;
    }
    static const double kRelStep[9] = {0, 3.45, 2.11, 1.49, 1.17, 1.01, 1.00, 1.05, 1.10};
    double cost[9];
    bool ok[9];
    for (int d = 1; d <= 8; ++d) {
        ok[d] = d == 1 || d == K || (d < K && h->depth_variant[d] >= 0);
        const double per = h->depth_tuned && h->depth_ms[d] > 0.0 ? h->depth_ms[d] : kRelStep[d];
        cost[d] = per * d;
    }
    const int64_t q = nsteps / K, r = nsteps % K;
    const int64_t qt = q < 4 ? q : 4;
    p.K = K;
    p.bulk = q - qt;
    const int T = (int)(r + K * qt);
    std::vector<double> best(T + 1, 1e300);
    std::vector<int> choice(T + 1, 0);
    best[0] = 0.0;
    for (int n = 1; n <= T; ++n)
        for (int d = 1; d <= K && d <= n; ++d)
            if (ok[d] && best[n - d] + cost[d] < best[n]) {
                best[n] = best[n - d] + cost[d];
                choice[n] = d;
            }
    for (int n = T; n > 0; n -= choice[n]) p.tail.push_back(choice[n]);
    std::sort(p.tail.begin(), p.tail.end(), [](int x, int y) { return x > y; });
    return p;
}

cudaError_t launch_step(const lb_rd_handle *h, const lbrd::StepArgs &a, int variant) {
    if (h->general) return lbrd::launch_step_general(h->prec == LB_RD_FP64 ? 0 : 1, h->Q, h->S, a, h->stream, variant);
    switch (h->prec) {
        case LB_RD_FP64: return lbrd::launch_step_f64(h->Q, h->S, a, h->stream);
        case LB_RD_FP32: return lbrd::launch_step_f32_variant(variant, h->Q, h->S, a, h->stream);
        default:
            return lbrd::launch_step_half_variant(variant, h->Q, h->S, h->prec == LB_RD_FP32_FP16DEV, a, h->stream);
    }
}
}  // namespace

extern "C" {

const char *lb_rd_last_error(void) { return g_err.c_str(); }

const char *lb_rd_version(void) { return "lb_rd 1.0 sm_103a"; }

double lb_rd_tau_from_diffusion(double D) { return 3.0 * D + 0.5; }

int lb_rd_check_config(const lb_rd_config *cfg, size_t *bytes) {
    if (!cfg) return fail(LB_RD_EINVAL, "config is NULL");
    const int Q = lattice_q(cfg->lattice);
    if (!Q) return fail(LB_RD_EINVAL, "lattice: unknown value " + std::to_string(cfg->lattice));
    if (cfg->nspecies < 1 || cfg->nspecies > LB_RD_MAX_SPECIES)
        return fail(LB_RD_EINVAL, "nspecies must be in [1, 4], got " + std::to_string(cfg->nspecies));
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nx > kMaxSide || cfg->ny > kMaxSide)
        return fail(LB_RD_EINVAL, "nx and ny must be in [1, 65535]");
    for (int s = 0; s < cfg->nspecies; ++s)
        if (!(cfg->tau[s] > 0.5) || !(cfg->tau[s] < 1e6))
            return fail(LB_RD_EINVAL, "tau[" + std::to_string(s) + "] must be in (1/2, 1e6) (D = (tau - 1/2)/3 > 0)");
    const lb_rd_reaction &r = cfg->reaction;
    if (r.kind < LB_RD_REACTION_NONE || r.kind > LB_RD_REACTION_MASS_ACTION)
        return fail(LB_RD_EINVAL, "reaction.kind: unknown value " + std::to_string(r.kind));
    if (r.kind == LB_RD_REACTION_GRAY_SCOTT && cfg->nspecies != 2)
        return fail(LB_RD_EINVAL, "Gray-Scott needs nspecies = 2");
    if (r.kind == LB_RD_REACTION_LINEAR && cfg->nspecies > 2)
        return fail(LB_RD_EINVAL, "the transformation A -> B takes 1 or 2 species (use a mass-action network)");
    if (r.kind == LB_RD_REACTION_MASS_ACTION) {
        if (r.nreactions < 1 || r.nreactions > LB_RD_MAX_REACTIONS)
            return fail(LB_RD_EINVAL, "reaction.nreactions must be in [1, 16]");
        for (int q = 0; q < r.nreactions; ++q) {
            const std::string at = "reaction step " + std::to_string(q) + ": ";
            if (!(r.rate[q] >= 0.0) || !(r.rate[q] < 1e300)) return fail(LB_RD_EINVAL, at + "rate must be finite and >= 0");
            for (int j = 0; j < LB_RD_MAX_SPECIES; ++j) {
                const bool used = j < cfg->nspecies;
                if (r.order[q][j] < 0 || r.order[q][j] > 3 || (!used && r.order[q][j] != 0))
                    return fail(LB_RD_EINVAL, at + "order must be in [0, 3] (0 for species beyond nspecies)");
                if (r.change[q][j] < -4 || r.change[q][j] > 4 || (!used && r.change[q][j] != 0))
                    return fail(LB_RD_EINVAL, at + "change must be in [-4, 4] (0 for species beyond nspecies)");
            }
        }
    }
    if (cfg->precision < LB_RD_FP64 || cfg->precision > LB_RD_FP32_FP16DEV)
        return fail(LB_RD_EINVAL, "precision: unknown value " + std::to_string(cfg->precision));
    if (needs_general(*cfg) && cfg->precision != LB_RD_FP64 && cfg->precision != LB_RD_FP32)
        return fail(LB_RD_EINVAL, "more than two species or a mass-action network: FP64 or FP32 storage only");
    if (cfg->streaming != LB_RD_STREAM_PINGPONG && cfg->streaming != LB_RD_STREAM_INPLACE)
        return fail(LB_RD_EINVAL, "streaming: unknown value " + std::to_string(cfg->streaming));
    if (cfg->streaming == LB_RD_STREAM_INPLACE && cfg->precision != LB_RD_FP64 && cfg->precision != LB_RD_FP32)
        return fail(LB_RD_EINVAL, "in-place streaming: FP64 or FP32 storage only");
    if (cfg->tb_depth < 0 || cfg->tb_depth > 8)
        return fail(LB_RD_EINVAL, "tb_depth must be in [0, 8] (0: the autotuner's choice)");
    if (cfg->tb_depth > 1 && (cfg->precision == LB_RD_FP64 || cfg->streaming != LB_RD_STREAM_PINGPONG ||
                              needs_general(*cfg)))
        return fail(LB_RD_EINVAL, "tb_depth > 1 needs FP32 or 16-bit deviation storage with two state copies and "
                                  "at most two species without a mass-action network");
    if (bytes) {
        const int64_t pitch = pitch_for(cfg->nx);
        const size_t st = lbrd::state_plane_bytes(cfg->precision, Q, cfg->nspecies, cfg->ny, pitch);
        const size_t rb = (size_t)cfg->nspecies * cfg->ny * pitch * rho_elem(cfg->precision);
        const size_t np1 = lbrd::max_persistent_blocks(), np2 = lbrd::mass_partials_needed(cfg->nx, cfg->ny);
        const size_t copies = cfg->streaming == LB_RD_STREAM_INPLACE ? 1 : 2;
        *bytes = copies * st + rb + (np1 > np2 ? np1 : np2) * cfg->nspecies * sizeof(double) +
                 LB_RD_MAX_SPECIES * sizeof(double) + 2 * sizeof(int);
    }
    return LB_RD_OK;
}

int lb_rd_destroy(lb_rd_handle *h) {
    if (!h) return LB_RD_OK;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->rho);
    cudaFree(h->stage);
    cudaFree(h->partials);
    cudaFree(h->counter);
    cudaFree(h->mass);
    cudaFree(h->status);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    delete h;
    return LB_RD_OK;
}

int lb_rd_create(const lb_rd_config *cfg, lb_rd_handle **out) {
    if (!out) return fail(LB_RD_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = lb_rd_check_config(cfg, nullptr);
    if (rc) return rc;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(LB_RD_ECUDA, std::string("no CUDA device: ") + (e ? cudaGetErrorString(e) : "count is 0"));
    if (cfg->precision == LB_RD_FP32_BF16DEV || cfg->precision == LB_RD_FP32_FP16DEV) {
        if (cfg->nx % 4 != 0)
            return fail(LB_RD_EINVAL, "16-bit deviation storage needs nx to be a multiple of 4");
    }
    lb_rd_handle *h = new lb_rd_handle();
    h->cfg = *cfg;
    h->Q = lattice_q(cfg->lattice);
    h->S = cfg->nspecies;
    h->prec = cfg->precision;
    h->general = needs_general(*cfg);
    h->inplace = cfg->streaming == LB_RD_STREAM_INPLACE;
    h->pitch = pitch_for(cfg->nx);
    h->plane = cfg->ny * h->pitch;
    h->stream = static_cast<cudaStream_t>(cfg->stream);
    h->state_bytes = lbrd::state_plane_bytes(h->prec, h->Q, h->S, cfg->ny, h->pitch);
    h->rho_bytes = (size_t)h->S * h->plane * rho_elem(h->prec);
    const size_t nparts = (size_t)lbrd::max_persistent_blocks();
    const size_t nparts2 = lbrd::mass_partials_needed(cfg->nx, cfg->ny);
    const size_t parts = (nparts > nparts2 ? nparts : nparts2) * h->S;
    cudaError_t err = cudaSuccess;
    if (!err) err = cudaMalloc(&h->buf[0], h->state_bytes);
    if (!err && !h->inplace) err = cudaMalloc(&h->buf[1], h->state_bytes);
    if (!err) err = cudaMalloc(&h->rho, h->rho_bytes);
    if (!err) err = cudaMalloc(&h->partials, parts * sizeof(double));
    if (!err) err = cudaMalloc(&h->counter, sizeof(unsigned int));
    if (!err) err = cudaMalloc(&h->mass, LB_RD_MAX_SPECIES * sizeof(double));
    if (!err) err = cudaMalloc(&h->status, sizeof(int));
    if (!err) err = cudaMemset(h->status, 0, sizeof(int));
    if (!err) err = cudaMemset(h->counter, 0, sizeof(unsigned int));
    if (!err) err = cudaMemset(h->buf[0], 0, h->state_bytes);
    if (!err && !h->inplace) err = cudaMemset(h->buf[1], 0, h->state_bytes);
    if (!err) err = cudaMemset(h->rho, 0, h->rho_bytes);
    if (err) {
        rc = cuda_fail(err, "lb_rd_create allocation");
        lb_rd_destroy(h);
        return rc;
    }
    default_depths(h);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(h));
        if (it != g_tune_cache.end()) apply_tune(h, it->second);
    }
    if (cfg->tb_depth == 1) {
        h->tb_variant = -1;
    } else if (cfg->tb_depth > 1) {
        if (h->depth_variant[cfg->tb_depth] < 0) {
            lb_rd_destroy(h);
            return fail(LB_RD_EINVAL, "tb_depth " + std::to_string(cfg->tb_depth) + ": no launch variant of that "
                                      "many steps fits nx = " + std::to_string(cfg->nx));
        }
        h->tb_variant = h->depth_variant[cfg->tb_depth];
    }
    *out = h;
    return LB_RD_OK;
}

static int ensure_stage(lb_rd_handle *h, size_t elems) {
    if (h->stage_elems >= elems) return LB_RD_OK;
    if (h->stage) {
        LBRD_CUDA(cudaStreamSynchronize(h->stream), "stage sync");
        cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_elems = 0;
    }
    LBRD_CUDA(cudaMalloc(&h->stage, elems * sizeof(double)), "staging allocation");
    h->stage_elems = elems;
    return LB_RD_OK;
}


int lb_rd_init(lb_rd_handle *h, const double *rho0, int is_device) {
    if (!h || !rho0) return fail(LB_RD_EINVAL, "handle or rho0 is NULL");
    const size_t n = (size_t)h->S * h->cfg.ny * h->cfg.nx;
    const double *src = rho0;
    if (!is_device) {
        int rc = ensure_stage(h, n);
        if (rc) return rc;
        LBRD_CUDA(cudaMemcpyAsync(h->stage, rho0, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "rho0 upload");
        src = h->stage;
    }
    LBRD_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "status reset");
    lbrd::InitArgs a{};
    a.rho0 = src;
    a.dst = h->buf[h->cur];
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    lbrd::fill_reaction(h->cfg, a.omega, &a.rkind, &a.kappa, &a.F, &a.k, &a.net);
    a.rho_out = h->rho;
    cudaError_t e;
    if (h->general) e = lbrd::launch_init_general(h->prec == LB_RD_FP64 ? 0 : 1, h->Q, h->S, a, h->stream);
    else switch (h->prec) {
        case LB_RD_FP64: e = lbrd::launch_init_f64(h->Q, h->S, a, h->stream); break;
        case LB_RD_FP32: e = lbrd::launch_init_f32(h->Q, h->S, a, h->stream); break;
        default: e = lbrd::launch_init_half(h->Q, h->S, h->prec == LB_RD_FP32_FP16DEV, a, h->stream); break;
    }
    if (e) return cuda_fail(e, "init kernel");
    h->launches++;
    if (!is_device) LBRD_CUDA(cudaStreamSynchronize(h->stream), "init sync");
    h->t = 0;
    h->rho_t = 0;
    h->mass_fresh = false;
    h->initialized = true;
    return LB_RD_OK;
}

// Make the density cache hold rho(t): after a step the previous copy of the
// state, f*(t - 1), is still intact and its pull-sum is rho(t).
static int ensure_rho(lb_rd_handle *h) {
    if (h->rho_t == h->t) return LB_RD_OK;
    if (h->inplace) return fail(LB_RD_EINVAL, "in-place handle: the density cache is out of date");
    cudaError_t e = lbrd::launch_pull_rho(h->prec, h->Q, h->S, h->buf[h->cur ^ 1], h->cfg.nx, h->cfg.ny, h->pitch,
                                          h->rho, h->stream);
    if (e) return cuda_fail(e, "density kernel");
    h->launches++;
    h->rho_t = h->t;
    return LB_RD_OK;
}

int lb_rd_step(lb_rd_handle *h, int64_t nsteps) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(LB_RD_EINVAL, "nsteps must be >= 0");
    if (!h->initialized) return fail(LB_RD_EINVAL, "lb_rd_init has not been called");
    lbrd::StepArgs a{};
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    lbrd::fill_reaction(h->cfg, a.omega, &a.rkind, &a.kappa, &a.F, &a.k, &a.net);
    a.partials = h->partials;
    a.counter = h->counter;
    a.status = h->status;
    if (h->inplace) {
        // one copy: phase by the parity of t; the last launch writes rho(t)
        for (int64_t n = 0; n < nsteps; ++n) {
            a.src = a.dst = h->buf[0];
            a.rho_out = n == nsteps - 1 ? h->rho : nullptr;
            a.mass_out = h->cfg.track_mass ? h->mass : nullptr;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (h->timing) {
                LBRD_CUDA(cudaEventCreate(&e0), "event create");
                LBRD_CUDA(cudaEventCreate(&e1), "event create");
                LBRD_CUDA(cudaEventRecord(e0, h->stream), "event record");
            }
            cudaError_t e = lbrd::launch_step_aa(h->prec == LB_RD_FP64 ? 0 : 1, h->Q, h->S, (int)(h->t & 1), a,
                                                 h->stream, h->variant);
            if (e) return cuda_fail(e, "in-place step kernel");
            h->launches++;
            if (h->timing) {
                LBRD_CUDA(cudaEventRecord(e1, h->stream), "event record");
                h->events.push_back(e0);
                h->events.push_back(e1);
                h->event_steps.push_back(1);
                h->event_variant.push_back(h->variant);
            }
            h->t += 1;
        }
        if (nsteps > 0) {
            h->rho_t = h->t;
            h->mass_fresh = h->cfg.track_mass != 0;
        }
        return LB_RD_OK;
    }
    // K steps per launch for the bulk of the call, then the planned tail; a
    // last launch of d >= 2 steps writes rho(t) (the other copy then no longer
    // holds f*(t - 1)), a last single step leaves it to be recomputed on demand
    // from the other copy (ensure_rho).
    const LaunchPlan plan = plan_launches(h, nsteps);
    const int64_t nl = plan.bulk + (int64_t)plan.tail.size();
    for (int64_t n = 0; n < nl; ++n) {
        const int d = n < plan.bulk ? plan.K : plan.tail[(size_t)(n - plan.bulk)];
        const int v = d == 1 ? h->variant : (d == plan.K ? h->tb_variant : h->depth_variant[d]);
        const bool last = n == nl - 1;
        a.src = h->buf[h->cur];
        a.dst = h->buf[h->cur ^ 1];
        a.rho_out = last && d >= 2 ? h->rho : nullptr;
        a.mass_out = h->cfg.track_mass ? h->mass : nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing) {
            LBRD_CUDA(cudaEventCreate(&e0), "event create");
            LBRD_CUDA(cudaEventCreate(&e1), "event create");
            LBRD_CUDA(cudaEventRecord(e0, h->stream), "event record");
        }
        a.inject_timeout = h->inject_timeout;
        h->inject_timeout = 0;
        cudaError_t e = launch_step(h, a, v);
        if (e) return cuda_fail(e, "step kernel");
        h->launches++;
        if (h->timing) {
            LBRD_CUDA(cudaEventRecord(e1, h->stream), "event record");
            h->events.push_back(e0);
            h->events.push_back(e1);
            h->event_steps.push_back(d);
            h->event_variant.push_back(v);
        }
        h->cur ^= 1;
        h->t += d;
        if (last && d >= 2) h->rho_t = h->t;
    }
    if (nsteps > 0) h->mass_fresh = h->cfg.track_mass != 0;
    return LB_RD_OK;
}

int lb_rd_get_time(const lb_rd_handle *h, int64_t *t) {
    if (!h || !t) return fail(LB_RD_EINVAL, "handle or t is NULL");
    *t = h->t;
    return LB_RD_OK;
}

int lb_rd_moments(lb_rd_handle *h, double *rho_out, double *mass_out, int is_device) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    if (!h->initialized) return fail(LB_RD_EINVAL, "lb_rd_init has not been called");
    const int64_t nx = h->cfg.nx, ny = h->cfg.ny;
    const size_t n = (size_t)h->S * ny * nx;
    if (rho_out || (mass_out && !h->mass_fresh)) {
        int rc = ensure_rho(h);
        if (rc) return rc;
    }
    if (rho_out) {
        double *dst = rho_out;
        if (!is_device) {
            int rc = ensure_stage(h, n);
            if (rc) return rc;
            dst = h->stage;
        }
        cudaError_t e = lbrd::launch_rho_export(h->prec, h->S, h->rho, nx, ny, h->pitch, dst, h->stream);
        if (e) return cuda_fail(e, "rho export kernel");
        h->launches++;
        if (!is_device)
            LBRD_CUDA(cudaMemcpyAsync(rho_out, h->stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                      "rho download");
    }
    if (mass_out) {
        if (!h->mass_fresh) {
            cudaError_t e = lbrd::launch_mass(h->prec, h->S, h->rho, nx, ny, h->pitch, h->partials, h->counter,
                                              h->mass, h->stream);
            if (e) return cuda_fail(e, "mass kernel");
            h->launches++;
            h->mass_fresh = true;
        }
        LBRD_CUDA(cudaMemcpyAsync(mass_out, h->mass, h->S * sizeof(double),
                                  is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
                  "mass download");
    }
    int status = 0;
    LBRD_CUDA(cudaMemcpyAsync(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status read");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "moments sync");
    if (status) return fail(status, "a step kernel gave up a bounded wait; the state is not valid");
    return LB_RD_OK;
}

int lb_rd_get_distributions(lb_rd_handle *h, double *f_out, int is_device) {
    if (!h || !f_out) return fail(LB_RD_EINVAL, "handle or f_out is NULL");
    if (!h->initialized) return fail(LB_RD_EINVAL, "lb_rd_init has not been called");
    const size_t n = (size_t)h->S * h->Q * h->cfg.ny * h->cfg.nx;
    double *dst = f_out;
    if (!is_device) {
        int rc = ensure_stage(h, n);
        if (rc) return rc;
        dst = h->stage;
    }
    cudaError_t e = h->inplace && (h->t & 1)
                         ? lbrd::launch_export_swapped(h->prec == LB_RD_FP64 ? 0 : 1, h->Q, h->S, h->buf[0], h->cfg.nx,
                                                       h->cfg.ny, h->pitch, dst, h->stream)
                         : lbrd::launch_export(h->prec, h->Q, h->S, h->buf[h->cur], h->cfg.nx, h->cfg.ny, h->pitch,
                                               dst, h->stream);
    if (e) return cuda_fail(e, "export kernel");
    h->launches++;
    if (!is_device)
        LBRD_CUDA(cudaMemcpyAsync(f_out, h->stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                  "distribution download");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "export sync");
    return LB_RD_OK;
}

// Checkpoint layout: header, then the current state copy, then the rho cache.
struct CkptHeader {
    char magic[8];
    int32_t prec, Q, S, pad;  // pad: 1 for the in-place state layout
    int64_t nx, ny, pitch, t;
};

int lb_rd_state_size(const lb_rd_handle *h, size_t *bytes) {
    if (!h || !bytes) return fail(LB_RD_EINVAL, "handle or bytes is NULL");
    *bytes = sizeof(CkptHeader) + h->state_bytes + h->rho_bytes;
    return LB_RD_OK;
}

int lb_rd_save(lb_rd_handle *h, void *host_buf, size_t bytes) {
    size_t need = 0;
    int rc = lb_rd_state_size(h, &need);
    if (rc) return rc;
    if (!host_buf || bytes < need) return fail(LB_RD_EINVAL, "checkpoint buffer too small");
    if (!h->initialized) return fail(LB_RD_EINVAL, "lb_rd_init has not been called");
    rc = ensure_rho(h);
    if (rc) return rc;
    CkptHeader hd{};
    std::memcpy(hd.magic, "LBRDCKP1", 8);
    hd.prec = h->prec;
    hd.Q = h->Q;
    hd.S = h->S;
    hd.pad = h->inplace ? 1 : 0;  // state layout
    hd.nx = h->cfg.nx;
    hd.ny = h->cfg.ny;
    hd.pitch = h->pitch;
    hd.t = h->t;
    char *p = static_cast<char *>(host_buf);
    std::memcpy(p, &hd, sizeof(hd));
    LBRD_CUDA(cudaMemcpyAsync(p + sizeof(hd), h->buf[h->cur], h->state_bytes, cudaMemcpyDeviceToHost, h->stream),
              "checkpoint state");
    LBRD_CUDA(cudaMemcpyAsync(p + sizeof(hd) + h->state_bytes, h->rho, h->rho_bytes, cudaMemcpyDeviceToHost, h->stream),
              "checkpoint rho");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "checkpoint sync");
    return LB_RD_OK;
}

int lb_rd_restore(lb_rd_handle *h, const void *host_buf, size_t bytes) {
    size_t need = 0;
    int rc = lb_rd_state_size(h, &need);
    if (rc) return rc;
    if (!host_buf || bytes < need) return fail(LB_RD_EINVAL, "checkpoint buffer too small");
    CkptHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    if (std::memcmp(hd.magic, "LBRDCKP1", 8) != 0 || hd.prec != h->prec || hd.Q != h->Q || hd.S != h->S ||
        hd.nx != h->cfg.nx || hd.ny != h->cfg.ny || hd.pitch != h->pitch || hd.pad != (h->inplace ? 1 : 0))
        return fail(LB_RD_EINVAL, "checkpoint does not match this handle's configuration");
    const char *p = static_cast<const char *>(host_buf);
    LBRD_CUDA(cudaMemcpyAsync(h->buf[h->cur], p + sizeof(hd), h->state_bytes, cudaMemcpyHostToDevice, h->stream),
              "restore state");
    LBRD_CUDA(cudaMemcpyAsync(h->rho, p + sizeof(hd) + h->state_bytes, h->rho_bytes, cudaMemcpyHostToDevice, h->stream),
              "restore rho");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "restore sync");
    h->t = hd.t;
    h->rho_t = hd.t;
    h->mass_fresh = false;
    h->initialized = true;
    return LB_RD_OK;
}

int lb_rd_set_timing(lb_rd_handle *h, int enable) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "timing sync");
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    h->events.clear();
    h->event_steps.clear();
    h->event_variant.clear();
    h->timing = enable != 0;
    return LB_RD_OK;
}

int lb_rd_launch_times(lb_rd_handle *h, double *ms, int32_t *steps, int32_t *variant, int64_t max, int64_t *count) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    if (max < 0) return fail(LB_RD_EINVAL, "max must be >= 0");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "timing sync");
    const int64_t n = (int64_t)h->event_steps.size();
    for (int64_t i = 0; i < n && i < max; ++i) {
        float t = 0.f;
        LBRD_CUDA(cudaEventElapsedTime(&t, h->events[2 * i], h->events[2 * i + 1]), "event elapsed");
        if (ms) ms[i] = t;
        if (steps) steps[i] = h->event_steps[(size_t)i];
        if (variant) variant[i] = h->event_variant[(size_t)i];
    }
    if (count) *count = n;
    return LB_RD_OK;
}

int lb_rd_kernel_time(lb_rd_handle *h, double *total_ms, int64_t *launches) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    LBRD_CUDA(cudaStreamSynchronize(h->stream), "timing sync");
    double sum = 0.0;
    for (size_t i = 0; i + 1 < h->events.size(); i += 2) {
        float ms = 0.f;
        LBRD_CUDA(cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]), "event elapsed");
        sum += ms;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = (int64_t)(h->events.size() / 2);
    return LB_RD_OK;
}

int lb_rd_launch_count(const lb_rd_handle *h, int64_t *launches) {
    if (!h || !launches) return fail(LB_RD_EINVAL, "handle or launches is NULL");
    *launches = h->launches;
    return LB_RD_OK;
}

int lb_rd_debug_inject_wait_timeout(lb_rd_handle *h, int32_t enable) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    h->inject_timeout = enable ? 1 : 0;
    return LB_RD_OK;
}

int lb_rd_variant_count(int32_t precision, int32_t *count) {
    if (!count || precision < LB_RD_FP64 || precision > LB_RD_FP32_FP16DEV)
        return fail(LB_RD_EINVAL, "bad precision or NULL count");
    *count = variant_count(precision);
    return LB_RD_OK;
}

const char *lb_rd_variant_name(int32_t precision, int32_t variant) {
    if (precision == LB_RD_FP32 && variant >= 0 && variant < lbrd::kF32VariantCount)
        return lbrd::kF32Variants[variant].name;
    if (precision == LB_RD_FP64) return variant == 0 ? "f64_32x4" : "";
    if ((precision == LB_RD_FP32_BF16DEV || precision == LB_RD_FP32_FP16DEV) && variant >= 0 &&
        variant < lbrd::kHalfVariantCount)
        return lbrd::kHalfVariantNames[variant];
    return "";
}

int lb_rd_handle_variant_count(const lb_rd_handle *h, int32_t *count) {
    if (!h || !count) return fail(LB_RD_EINVAL, "handle or count is NULL");
    *count = handle_variant_count(h);
    return LB_RD_OK;
}

const char *lb_rd_handle_variant_name(const lb_rd_handle *h, int32_t variant) {
    if (!h || variant < 0 || variant >= handle_variant_count(h)) return "";
    if (h->inplace) return h->prec == LB_RD_FP64 ? "aa_f64" : lbrd::kAAVariants[variant].name;
    if (!h->general) return lb_rd_variant_name(h->prec, variant);
    return h->prec == LB_RD_FP64 ? "general_f64" : lbrd::kGeneralVariants[variant].name;
}

int lb_rd_set_variant(lb_rd_handle *h, int32_t variant) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    if (variant == -1) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(h));
        default_depths(h);
        h->variant = 0;
        h->tb_variant = -1;
        if (it != g_tune_cache.end()) apply_tune(h, it->second);
        return LB_RD_OK;
    }
    if (variant < 0 || variant >= handle_variant_count(h))
        return fail(LB_RD_EINVAL, "variant out of range for this configuration");
    if (!variant_fits(h, variant))
        return fail(LB_RD_EINVAL, std::string("variant ") + lb_rd_handle_variant_name(h, variant) +
                                      " needs nx to be a multiple of " +
                                      std::to_string(h->inplace   ? lbrd::kAAVariants[variant].sites
                                                     : h->general ? lbrd::kGeneralVariants[variant].sites
                                                     : is_half(h) ? lbrd::kHalfVariantNx[variant]
                                                                  : lbrd::kF32Variants[variant].nx_multiple));
    if (variant_steps(h, variant) >= 2) {
        h->tb_variant = variant;
    } else {
        h->variant = variant;
        h->tb_variant = -1;
    }
    return LB_RD_OK;
}

int lb_rd_get_variant(const lb_rd_handle *h, int32_t *variant) {
    if (!h || !variant) return fail(LB_RD_EINVAL, "handle or variant is NULL");
    *variant = h->tb_variant >= 0 ? h->tb_variant : h->variant;
    return LB_RD_OK;
}

// In-place handles have no spare copy: the variants are timed on a temporary
// copy of the state (alternating the two phases from the handle's parity),
// which is freed afterwards; the handle's own state is not touched.
static int autotune_inplace(lb_rd_handle *h, int32_t iters, int32_t *best, double *times_ms, int32_t max_times) {
    void *scratch = nullptr;
    LBRD_CUDA(cudaMalloc(&scratch, h->state_bytes), "autotune scratch");
    cudaError_t e = cudaMemcpyAsync(scratch, h->buf[0], h->state_bytes, cudaMemcpyDeviceToDevice, h->stream);
    lbrd::StepArgs a{};
    a.src = a.dst = scratch;
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    lbrd::fill_reaction(h->cfg, a.omega, &a.rkind, &a.kappa, &a.F, &a.k, &a.net);
    a.status = h->status;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    const int prec = h->prec == LB_RD_FP64 ? 0 : 1;
    int64_t t = h->t;
    int bestv = -1;
    double bestms = 0.0;
    for (int v = 0; v < handle_variant_count(h) && !e; ++v) {
        if (!variant_fits(h, v)) {
            if (times_ms && v < max_times) times_ms[v] = -1.0;
            continue;
        }
        for (int k = 0; k < 2 && !e; ++k, ++t) e = lbrd::launch_step_aa(prec, h->Q, h->S, (int)(t & 1), a, h->stream, v);
        if (!e) e = cudaEventRecord(e0, h->stream);
        for (int k = 0; k < iters && !e; ++k, ++t) e = lbrd::launch_step_aa(prec, h->Q, h->S, (int)(t & 1), a, h->stream, v);
        if (!e) e = cudaEventRecord(e1, h->stream);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e) break;
        h->launches += iters + 2;
        const double per = ms / iters;
        if (times_ms && v < max_times) times_ms[v] = per;
        if (bestv < 0 || per < bestms) {
            bestv = v;
            bestms = per;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaFree(scratch);
    if (e) return cuda_fail(e, "in-place autotune");
    h->variant = bestv >= 0 ? bestv : 0;
    h->tb_variant = -1;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        TuneEntry t;
        t.variant = h->variant;
        g_tune_cache[tune_key(h)] = t;
    }
    if (best) *best = h->variant;
    return LB_RD_OK;
}

int lb_rd_autotune(lb_rd_handle *h, int32_t iters, int32_t *best, double *times_ms, int32_t max_times) {
    if (!h) return fail(LB_RD_EINVAL, "handle is NULL");
    if (iters < 1) return fail(LB_RD_EINVAL, "iters must be >= 1");
    if (!h->initialized) return fail(LB_RD_EINVAL, "lb_rd_init has not been called");
    if (h->inplace) return autotune_inplace(h, iters, best, times_ms, max_times);
    int rc = ensure_rho(h);  // the tuner overwrites f*(t - 1), from which rho(t) would be recomputed
    if (rc) return rc;
    lbrd::StepArgs a{};
    a.src = h->buf[h->cur];
    a.dst = h->buf[h->cur ^ 1];  // spare copy: the state is not advanced
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    lbrd::fill_reaction(h->cfg, a.omega, &a.rkind, &a.kappa, &a.F, &a.k, &a.net);
    a.status = h->status;
    cudaEvent_t e0, e1;
    LBRD_CUDA(cudaEventCreate(&e0), "event create");
    LBRD_CUDA(cudaEventCreate(&e1), "event create");
    const int n = handle_variant_count(h);
    int best1 = -1, best2 = -1;
    double ms1 = 0.0, ms2 = 0.0;
    TuneEntry te;
    for (int v = 0; v < n; ++v) {
        if (!variant_fits(h, v)) {  // variant not applicable to this grid
            if (times_ms && v < max_times) times_ms[v] = -1.0;
            continue;
        }
        cudaError_t e = launch_step(h, a, v);  // warm-up
        for (int it = 0; it < iters && !e; ++it) {
            if (it == 0) cudaEventRecord(e0, h->stream);
            e = launch_step(h, a, v);
        }
        if (!e) e = cudaEventRecord(e1, h->stream);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "autotune launch");
        }
        h->launches += iters + 1;
        const int steps = variant_steps(h, v);
        const double per = ms / iters / steps;  // per time step
        if (times_ms && v < max_times) times_ms[v] = per;
        if (steps == 1 && (best1 < 0 || per < ms1)) {
            best1 = v;
            ms1 = per;
        }
        if (steps >= 2 && (best2 < 0 || per < ms2)) {
            best2 = v;
            ms2 = per;
        }
        if (is_deep(h, v) && steps >= 2 && (te.depth_variant[steps] < 0 || per < te.depth_ms[steps])) {
            te.depth_variant[steps] = v;
            te.depth_ms[steps] = per;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    te.variant = best1 >= 0 ? best1 : 0;
    te.tb_variant = (best2 >= 0 && ms2 < ms1) ? best2 : -1;
    te.depth_ms[1] = best1 >= 0 ? ms1 : 0.0;
    default_depths(h);
    apply_tune(h, te);
    const int arg = h->tb_variant >= 0 ? h->tb_variant : h->variant;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[tune_key(h)] = te;
    }
    if (best) *best = arg;
    return LB_RD_OK;
}

}  // extern "C"
