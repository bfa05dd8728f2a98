// Batched simulations: one persistent launch per time step over the combined
// (instance x tile) work list of all instances, replayed as CUDA graphs.
//
// Every instance has its own grid, relaxation times and reaction constants
// in a descriptor; the kernel walks global tile indices with a grid-stride
// loop, finds the instance a tile belongs to by a forward scan (a block's
// tiles only increase) and runs the same tile body as the single-simulation
// kernels (step_f32_kernel.cuh, step_half_kernel.cuh), so each instance
// computes exactly what a single handle computes.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lb_rd.h"
#include "lbrd_kernels.h"
#include "step_aa_kernel.cuh"
#include "step_f32_kernel.cuh"
#include "step_f64_kernel.cuh"
#include "step_half_kernel.cuh"

namespace lbrd {
int report_error(int code, const std::string &msg);

namespace {

constexpr int kBX = 64, kBY = 2, kNT = kBX * kBY;  // the tile shape of both tile bodies
static_assert(half::kBX == kBX && half::kBY == kBY, "tile shapes must agree");

// MODE 0: FP32 storage, 1: bf16 deviations, 2: fp16 deviations, 3: FP64,
// 4: FP32 where some instances keep one copy updated in place (the AA tile
// body of step_aa_kernel.cuh; BatchItem::aa selects the body per instance).
// An FP64 tile covers the same 256 x 2 sites; a thread updates the sites
// x = x_tile + threadIdx.x + 64 j, j < 4 (coalesced), one at a time.
template <int Q, int S, int MODE>
__global__ void __launch_bounds__(kNT, 4) batch_kernel(const BatchItem *__restrict__ items, int nitems,
                                                       int64_t total_tiles) {
    const int lane = threadIdx.x & 31;
    __shared__ aa::AANet no_network;  // batched instances have no mass-action network; never read
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    int it = 0;
    for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        while (it + 1 < nitems && items[it + 1].tile_begin <= t) ++it;
        const BatchItem &b = items[it];
        const int64_t local = t - b.tile_begin;
        const int64_t ty = local / b.tiles_x, tx = local - ty * b.tiles_x;
        const int64_t y = ty * kBY + threadIdx.y;
        if constexpr (MODE == 3) {
            if (y < b.a.ny) {
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    const int64_t x = tx * kBX * 4 + threadIdx.x + j * kBX;
                    if (x < b.a.nx) f64::site_f64<Q, S>(b.a, x, y, acc);
                }
            }
        } else {
            const int64_t x0 = (tx * kBX + threadIdx.x) * 4;
            if constexpr (MODE == 0) {
                f32::tile_f32<Q, S, 0>(b.a, x0, y, lane, acc);
            } else if constexpr (MODE == 4) {
                if (b.aa == 0) {
                    f32::tile_f32<Q, S, 0>(b.a, x0, y, lane, acc);
                } else if (b.aa <= 2) {  // nx % 4 == 0: four sites per thread
                    if (b.aa == 1) aa::tile_aa<Q, S, 4, 0>(b.a, no_network, x0, y, lane, acc);
                    else aa::tile_aa<Q, S, 4, 1>(b.a, no_network, x0, y, lane, acc);
                } else if (y < b.a.ny) {  // any nx: the tile's 256 x 2 sites one at a time, coalesced
#pragma unroll 1
                    for (int j = 0; j < 4; ++j) {
                        const int64_t x = tx * kBX * 4 + threadIdx.x + j * kBX;
                        if (x >= b.a.nx) continue;
                        if (b.aa == 3) aa::site_aa<float, Q, S, 0>(b.a, no_network, x, y, acc);
                        else aa::site_aa<float, Q, S, 1>(b.a, no_network, x, y, acc);
                    }
                }
            } else {
                half::tile_half<Q, S, MODE - 1>(b.a, x0, y, lane, acc);
            }
        }
    }
}

template <int Q, int S, int MODE>
cudaError_t launch_batch(const BatchItem *items, int n, int64_t total, cudaStream_t st) {
    auto kern = batch_kernel<Q, S, MODE>;
    const unsigned grid = persistent_blocks(kern, kNT, total);
    kern<<<grid, dim3(kBX, kBY), 0, st>>>(items, n, total);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_batch(int Q, int S, const BatchItem *items, int n, int64_t total, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_batch<9, 1, MODE>(items, n, total, st);
    if (Q == 9 && S == 2) return launch_batch<9, 2, MODE>(items, n, total, st);
    if (Q == 5 && S == 1) return launch_batch<5, 1, MODE>(items, n, total, st);
    if (Q == 5 && S == 2) return launch_batch<5, 2, MODE>(items, n, total, st);
    return cudaErrorInvalidValue;
}

int64_t pitch_for(int64_t nx) { return state_pitch(nx); }

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

int batch_mode(int precision) {
    switch (precision) {
        case LB_RD_FP32: return 0;
        case LB_RD_FP32_BF16DEV: return 1;
        case LB_RD_FP32_FP16DEV: return 2;
        default: return 3;
    }
}

cudaError_t launch_batch_init(int mode, int Q, int S, const InitArgs &a, cudaStream_t st) {
    if (mode == 0 || mode == 4) return launch_init_f32(Q, S, a, st);
    if (mode == 3) return launch_init_f64(Q, S, a, st);
    return launch_init_half(Q, S, mode == 2, a, st);
}

int64_t batch_tiles_x(int64_t nx) { return ((nx + 3) / 4 + kBX - 1) / kBX; }

int64_t batch_tiles(int64_t nx, int64_t ny) { return batch_tiles_x(nx) * ((ny + kBY - 1) / kBY); }

cudaError_t launch_batch_step(int mode, int Q, int S, const BatchItem *items, int n, int64_t total_tiles,
                             cudaStream_t st) {
    switch (mode) {
        case 0: return dispatch_batch<0>(Q, S, items, n, total_tiles, st);
        case 1: return dispatch_batch<1>(Q, S, items, n, total_tiles, st);
        case 2: return dispatch_batch<2>(Q, S, items, n, total_tiles, st);
        case 3: return dispatch_batch<3>(Q, S, items, n, total_tiles, st);
        case 4: return dispatch_batch<4>(Q, S, items, n, total_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd

struct lb_rd_batch {
    std::vector<lb_rd_config> cfgs;
    int Q = 0, S = 0, prec = 0, mode = 0;
    cudaStream_t stream = nullptr;
    std::vector<size_t> state_off, rho_off;  // byte offsets of each instance (state: copy 0 in buf[0])
    std::vector<size_t> state_off1;          // copy 1 in buf[1]; unused for in-place instances
    std::vector<bool> inplace;
    size_t state_total1 = 0;
    std::vector<int64_t> pitch;
    size_t state_total = 0, rho_total = 0;
    char *buf[2] = {nullptr, nullptr};
    char *rho = nullptr;
    lbrd::BatchItem *d_items[4] = {nullptr, nullptr, nullptr, nullptr};  // [parity + 2 * emit_rho]
    int64_t total_tiles = 0;
    double *stage = nullptr;
    size_t stage_elems = 0;
    double *partials = nullptr;
    unsigned int *counter = nullptr;
    double *mass = nullptr;
    std::vector<bool> inited;
    int cur = 0;
    int64_t t = 0, launches = 0;
    int graph_steps = 64;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by starting parity
    // K steps per launch: K = 2 the two-step kernel (FP32, two state copies,
    // every nx % strip == 0), otherwise the depth-K kernel (FP32, two state
    // copies; also K = 2 when the two-step kernel does not apply); tb_graph
    // holds graphs of K-step launches for the current K
    bool tb_ok = false;
    int steps_per_launch = 1;
    lbrd::TbwItem *d_tb[2] = {nullptr, nullptr};  // by buffer parity
    int64_t tb_units = 0;
    cudaGraphExec_t tb_graph[2] = {nullptr, nullptr};
    bool deep_ok = false, deep_v16 = false;
    std::vector<lbrd::DeepItem> deep_base;  // per instance, without buffers (rho_out: its density cache)
    lbrd::DeepItem *d_deep[9][2] = {};      // per steps per launch and buffer parity, planned on first use
    int64_t deep_units[9] = {};
};

namespace {

using lbrd::report_error;

int cuda_err(cudaError_t e, const char *what) {
    return report_error(e == cudaErrorMemoryAllocation ? LB_RD_ENOMEM : LB_RD_ECUDA,
                        std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

cudaError_t launch_one(lb_rd_batch *b, int parity, bool emit) {
    const lbrd::BatchItem *items = b->d_items[parity + (emit ? 2 : 0)];
    return lbrd::launch_batch_step(b->mode, b->Q, b->S, items, (int)b->cfgs.size(), b->total_tiles, b->stream);
}

void drop_graphs(lb_rd_batch *b) {
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto &g : b->tb_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// The K-step launches of this batch run the two-step kernel (else the depth-K kernel).
bool uses_tb2(const lb_rd_batch *b) { return b->steps_per_launch == 2 && b->tb_ok; }

// 16-bit deviation storage: the depth-K launches run its own kernel (K <= 5).
bool half_batch(const lb_rd_batch *b) { return b->mode == 1 || b->mode == 2; }

// Plans and uploads the depth-K descriptors of both parities (once per K).
cudaError_t plan_deep(lb_rd_batch *b, int K) {
    if (K < 2 || K > (half_batch(b) ? 5 : 8)) return cudaErrorInvalidValue;
    if (b->deep_units[K] > 0) return cudaSuccess;
    const int n = (int)b->cfgs.size();
    std::vector<lbrd::DeepItem> v = b->deep_base;
    const int64_t units = half_batch(b) ? lbrd::batch_half_deep_plan(K, b->Q, b->S, b->mode - 1, v.data(), n)
                                        : lbrd::batch_deep_plan(K, b->Q, b->S, b->deep_v16, v.data(), n);
    if (units <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int parity = 0; parity < 2 && !e; ++parity) {
        for (int i = 0; i < n; ++i) {
            char *c0 = b->buf[0] + b->state_off[i], *c1 = b->buf[1] + b->state_off1[i];
            v[i].a.src = parity ? c1 : c0;
            v[i].a.dst = parity ? c0 : c1;
        }
        if (!b->d_deep[K][parity]) e = cudaMalloc(&b->d_deep[K][parity], n * sizeof(lbrd::DeepItem));
        if (!e) e = cudaMemcpy(b->d_deep[K][parity], v.data(), n * sizeof(lbrd::DeepItem), cudaMemcpyHostToDevice);
    }
    if (!e) b->deep_units[K] = units;
    return e;
}

// One depth-K launch of K steps from buffer parity `parity`; emit: it also
// writes every instance's densities.
cudaError_t launch_deep(lb_rd_batch *b, int K, int parity, bool emit) {
    cudaError_t e = plan_deep(b, K);
    if (e) return e;
    const int rk = lbrd::list_reaction_kind(b->deep_base.data(), (int)b->deep_base.size());
    if (half_batch(b))
        return lbrd::launch_batch_half_deep(K, b->Q, b->S, b->mode - 1, b->d_deep[K][parity], (int)b->cfgs.size(),
                                            b->deep_units[K], emit, rk,
                                            lbrd::list_nx8(b->deep_base.data(), (int)b->deep_base.size()), b->stream);
    return lbrd::launch_batch_deep(K, b->Q, b->S, b->deep_v16, b->d_deep[K][parity], (int)b->cfgs.size(),
                                   b->deep_units[K], emit, rk, b->stream);
}

// One launch of steps_per_launch (>= 2) steps from buffer parity `parity`.
cudaError_t launch_multi(lb_rd_batch *b, int parity) {
    if (uses_tb2(b))
        return lbrd::launch_batch_tb2(b->d_tb[parity], (int)b->cfgs.size(), b->tb_units, b->Q, b->S, b->stream);
    return launch_deep(b, b->steps_per_launch, parity, false);
}

}  // namespace

extern "C" {

int lb_rd_batch_destroy(lb_rd_batch *b) {
    if (!b) return LB_RD_OK;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->rho);
    for (auto p : b->d_items) cudaFree(p);
    for (auto p : b->d_tb) cudaFree(p);
    for (auto &pk : b->d_deep)
        for (auto p : pk) cudaFree(p);
    cudaFree(b->stage);
    cudaFree(b->partials);
    cudaFree(b->counter);
    cudaFree(b->mass);
    delete b;
    return LB_RD_OK;
}

int lb_rd_batch_create(const lb_rd_config *cfgs, int32_t n, lb_rd_batch **out) {
    if (!out || !cfgs || n < 1) return report_error(LB_RD_EINVAL, "lb_rd_batch_create: need cfgs, n >= 1 and out");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        int rc = lb_rd_check_config(&cfgs[i], nullptr);
        if (rc) return rc;
        if (cfgs[i].nspecies > 2 || cfgs[i].reaction.kind == LB_RD_REACTION_MASS_ACTION)
            return report_error(LB_RD_EINVAL, "lb_rd_batch_create: batches take at most two species and no "
                                              "mass-action network (instance " + std::to_string(i) + ")");
        if (cfgs[i].streaming == LB_RD_STREAM_INPLACE && cfgs[i].precision != LB_RD_FP32)
            return report_error(LB_RD_EINVAL, "lb_rd_batch_create: in-place instances need FP32 storage "
                                              "(instance " + std::to_string(i) + ")");
        if (cfgs[i].lattice != cfgs[0].lattice || cfgs[i].nspecies != cfgs[0].nspecies ||
            cfgs[i].precision != cfgs[0].precision)
            return report_error(LB_RD_EINVAL, "lb_rd_batch_create: instance " + std::to_string(i) +
                                                  " differs from instance 0 in lattice, nspecies or precision");
    }
    const int prec = cfgs[0].precision;
    const bool half = prec == LB_RD_FP32_BF16DEV || prec == LB_RD_FP32_FP16DEV;
    for (int i = 0; i < n; ++i)
        if (half && cfgs[i].nx % 4)
            return report_error(LB_RD_EINVAL, "lb_rd_batch_create: 16-bit deviation storage needs nx % 4 == 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return report_error(LB_RD_ECUDA, "no CUDA device");

    lb_rd_batch *b = new lb_rd_batch();
    b->cfgs.assign(cfgs, cfgs + n);
    b->Q = cfgs[0].lattice == LB_RD_D2Q9 ? 9 : 5;
    b->S = cfgs[0].nspecies;
    b->prec = prec;
    b->mode = lbrd::batch_mode(prec);
    for (int i = 0; i < n; ++i)
        if (cfgs[i].streaming == LB_RD_STREAM_INPLACE) b->mode = 4;  // FP32 with in-place instances
    b->stream = static_cast<cudaStream_t>(cfgs[0].stream);
    b->inited.assign(n, false);
    size_t max_parts = 0;
    std::vector<lbrd::BatchItem> items(n);
    for (int i = 0; i < n; ++i) {
        const lb_rd_config &c = cfgs[i];
        const int64_t pitch = lbrd::pitch_for(c.nx);
        b->pitch.push_back(pitch);
        const size_t sb = lbrd::align256(lbrd::state_plane_bytes(prec, b->Q, b->S, c.ny, pitch));
        const bool ip = c.streaming == LB_RD_STREAM_INPLACE;
        b->inplace.push_back(ip);
        b->state_off.push_back(b->state_total);
        b->state_off1.push_back(ip ? 0 : b->state_total1);
        b->rho_off.push_back(b->rho_total);
        b->state_total += sb;
        if (!ip) b->state_total1 += sb;
        b->rho_total += lbrd::align256((size_t)b->S * c.ny * pitch * (prec == LB_RD_FP64 ? 8 : 4));
        const size_t parts = lbrd::mass_partials_needed(c.nx, c.ny);
        if (parts > max_parts) max_parts = parts;
        lbrd::BatchItem &it = items[i];
        it.a = lbrd::StepArgs{};
        it.a.nx = c.nx;
        it.a.ny = c.ny;
        it.a.pitch = pitch;
        it.a.plane = c.ny * pitch;
        for (int s = 0; s < 2; ++s) it.a.omega[s] = s < b->S ? 1.0 / c.tau[s] : 0.0;
        it.a.rkind = c.reaction.kind;
        it.a.kappa = c.reaction.kappa;
        it.a.F = c.reaction.F;
        it.a.k = c.reaction.k;
        it.tiles_x = lbrd::batch_tiles_x(c.nx);
        it.tile_begin = b->total_tiles;
        b->total_tiles += lbrd::batch_tiles(c.nx, c.ny);
    }
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaMalloc(&b->buf[0], b->state_total);
    if (!e && b->state_total1) e = cudaMalloc(&b->buf[1], b->state_total1);
    if (!e) e = cudaMalloc(&b->rho, b->rho_total);
    if (!e) e = cudaMalloc(&b->partials, max_parts * b->S * sizeof(double));
    if (!e) e = cudaMalloc(&b->counter, sizeof(unsigned int));
    if (!e) e = cudaMalloc(&b->mass, 2 * sizeof(double));
    if (!e) e = cudaMemset(b->counter, 0, sizeof(unsigned int));
    for (int k = 0; k < 4 && !e; ++k) {
        const int parity = k & 1;
        const bool emit = k >= 2;
        std::vector<lbrd::BatchItem> v = items;
        for (int i = 0; i < n; ++i) {
            char *c0 = b->buf[0] + b->state_off[i];
            if (b->inplace[i]) {
                v[i].a.src = v[i].a.dst = c0;
                v[i].aa = (cfgs[i].nx % 4 == 0 ? 1 : 3) + parity;
            } else {
                char *c1 = b->buf[1] + b->state_off1[i];
                v[i].a.src = parity ? c1 : c0;
                v[i].a.dst = parity ? c0 : c1;
                v[i].aa = 0;
            }
            v[i].a.rho_out = emit ? b->rho + b->rho_off[i] : nullptr;
        }
        e = cudaMalloc(&b->d_items[k], n * sizeof(lbrd::BatchItem));
        if (!e) e = cudaMemcpy(b->d_items[k], v.data(), n * sizeof(lbrd::BatchItem), cudaMemcpyHostToDevice);
    }
    // two-step descriptors: every instance FP32 with two copies and nx % strip == 0
    b->tb_ok = prec == LB_RD_FP32;
    for (int i = 0; i < n && b->tb_ok; ++i)
        if (b->inplace[i] || cfgs[i].nx % lbrd::batch_tb2_strip()) b->tb_ok = false;
    if (b->tb_ok && !e) {
        std::vector<lbrd::TbwItem> tv(n);
        for (int parity = 0; parity < 2 && !e; ++parity) {
            int64_t units = 0;
            for (int i = 0; i < n; ++i) {
                tv[i].a = items[i].a;
                char *c0 = b->buf[0] + b->state_off[i], *c1 = b->buf[1] + b->state_off1[i];
                tv[i].a.src = parity ? c1 : c0;
                tv[i].a.dst = parity ? c0 : c1;
                tv[i].a.rho_out = nullptr;
                tv[i].unit_begin = units;
                units += (cfgs[i].nx / lbrd::batch_tb2_strip()) * cfgs[i].ny;
            }
            b->tb_units = units;
            e = cudaMalloc(&b->d_tb[parity], n * sizeof(lbrd::TbwItem));
            if (!e) e = cudaMemcpy(b->d_tb[parity], tv.data(), n * sizeof(lbrd::TbwItem), cudaMemcpyHostToDevice);
        }
        b->steps_per_launch = 2;
    }
    // depth-K descriptors: FP32 or 16-bit deviation storage with two state copies
    b->deep_ok = prec == LB_RD_FP32 || half;
    b->deep_v16 = true;
    for (int i = 0; i < n; ++i) {
        if (b->inplace[i]) b->deep_ok = false;
        if (cfgs[i].nx % 4 || b->pitch[i] % 4) b->deep_v16 = false;
    }
    if (b->deep_ok) {
        b->deep_base.resize(n);
        for (int i = 0; i < n; ++i) {
            b->deep_base[i] = lbrd::DeepItem{};
            b->deep_base[i].a = items[i].a;
            b->deep_base[i].a.rho_out = b->rho + b->rho_off[i];
        }
        // default: the depth-K kernel, K = 5 (D2Q9) or 6 (D2Q5) in its
        // two-column form; 16-bit deviation storage: K = 4 (the two-column
        // form where every nx is a multiple of 8); should its descriptors not
        // be planned (no launch shape for this device), the batch keeps the
        // previous default
        const int K = half ? lbrd::batch_half_default_k() : lbrd::batch_deep_default_k(b->Q);
        if (!e && plan_deep(b, K) == cudaSuccess) b->steps_per_launch = K;
        cudaGetLastError();  // clear a non-sticky error of the attempt
    }
    if (!e && cfgs[0].tb_depth > 0) {  // the caller's steps per launch
        b->steps_per_launch = 1;
        const int K = cfgs[0].tb_depth;
        if (K >= 2 && !(K == 2 && b->tb_ok)) e = plan_deep(b, K);
        if (!e) b->steps_per_launch = K;
    }
    if (e) {
        int rc = cuda_err(e, "lb_rd_batch_create allocation");
        lb_rd_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LB_RD_OK;
}

static int batch_stage(lb_rd_batch *b, size_t elems) {
    if (b->stage_elems >= elems) return LB_RD_OK;
    if (b->stage) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->stage);
        b->stage = nullptr;
        b->stage_elems = 0;
    }
    cudaError_t e = cudaMalloc(&b->stage, elems * sizeof(double));
    if (e) return cuda_err(e, "batch staging allocation");
    b->stage_elems = elems;
    return LB_RD_OK;
}

int lb_rd_batch_init(lb_rd_batch *b, int32_t idx, const double *rho0, int is_device) {
    if (!b || !rho0) return report_error(LB_RD_EINVAL, "lb_rd_batch_init: batch or rho0 is NULL");
    if (idx < 0 || idx >= (int)b->cfgs.size()) return report_error(LB_RD_EINVAL, "lb_rd_batch_init: index out of range");
    if (b->t != 0) return report_error(LB_RD_EINVAL, "lb_rd_batch_init: the batch has already been stepped");
    const lb_rd_config &c = b->cfgs[idx];
    const size_t n = (size_t)b->S * c.ny * c.nx;
    const double *src = rho0;
    if (!is_device) {
        int rc = batch_stage(b, n);
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(b->stage, rho0, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e) return cuda_err(e, "rho0 upload");
        src = b->stage;
    }
    lbrd::InitArgs a{};
    a.rho0 = src;
    a.dst = b->buf[0] + b->state_off[idx];  // t == 0: copy 0 (the only copy of an in-place instance)
    a.nx = c.nx;
    a.ny = c.ny;
    a.pitch = b->pitch[idx];
    a.plane = c.ny * a.pitch;
    for (int s = 0; s < 2; ++s) a.omega[s] = s < b->S ? 1.0 / c.tau[s] : 0.0;
    a.rkind = c.reaction.kind;
    a.kappa = c.reaction.kappa;
    a.F = c.reaction.F;
    a.k = c.reaction.k;
    a.rho_out = b->rho + b->rho_off[idx];
    cudaError_t e = lbrd::launch_batch_init(b->mode, b->Q, b->S, a, b->stream);
    if (e) return cuda_err(e, "batch init kernel");
    b->launches++;
    if (!is_device) {
        e = cudaStreamSynchronize(b->stream);
        if (e) return cuda_err(e, "batch init sync");
    }
    b->inited[idx] = true;
    return LB_RD_OK;
}

int lb_rd_batch_set_graph(lb_rd_batch *b, int32_t steps_per_graph) {
    if (!b) return report_error(LB_RD_EINVAL, "batch is NULL");
    if (steps_per_graph != 0 && (steps_per_graph < 2 || steps_per_graph % 2))
        return report_error(LB_RD_EINVAL, "steps_per_graph must be 0 or an even number >= 2");
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    b->graph_steps = steps_per_graph;
    return LB_RD_OK;
}

// two == true: graph_steps / K launches of K = steps_per_launch steps (parity
// alternates per launch).
static int capture_graph(lb_rd_batch *b, int parity, bool two = false) {
    // A private stream: capturing on the legacy default stream is not allowed.
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) return cuda_err(e, "graph stream");
    cudaStream_t saved = b->stream;
    b->stream = cs;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    const int nl = two ? b->graph_steps / b->steps_per_launch : b->graph_steps;
    for (int k = 0; k < nl && !e; ++k)
        e = two ? launch_multi(b, (parity + k) & 1) : launch_one(b, (parity + k) & 1, false);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    b->stream = saved;
    if (!e) e = e2;
    if (!e) e = cudaGraphInstantiate(two ? &b->tb_graph[parity] : &b->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e) return cuda_err(e, "graph capture");
    return LB_RD_OK;
}

// K-step launches (all but the last, in graphs of graph_steps / K launches
// where they fill one) from the current buffer parity.
static int run_multi(lb_rd_batch *b, int64_t n_multi) {
    const int K = b->steps_per_launch;
    const int per_graph = b->graph_steps / K;  // K-step launches per graph
    if (per_graph > 0 && n_multi >= per_graph) {
        const int64_t reps = n_multi / per_graph;
        for (int64_t r = 0; r < reps; ++r) {
            if (!b->tb_graph[b->cur]) {  // captured once per starting parity
                int rc = capture_graph(b, b->cur, true);
                if (rc) return rc;
            }
            cudaError_t e = cudaGraphLaunch(b->tb_graph[b->cur], b->stream);
            if (e) return cuda_err(e, "graph launch");
            if (per_graph & 1) b->cur ^= 1;  // an odd number of launches flips the buffers
        }
        b->launches += reps * per_graph;
        b->t += reps * per_graph * K;
        n_multi -= reps * per_graph;
    }
    for (int64_t k = 0; k < n_multi; ++k) {
        cudaError_t e = launch_multi(b, b->cur);
        if (e) return cuda_err(e, "batch multi-step kernel");
        b->cur ^= 1;
        b->t += K;
        b->launches++;
    }
    return LB_RD_OK;
}

int lb_rd_batch_step(lb_rd_batch *b, int64_t nsteps) {
    if (!b) return report_error(LB_RD_EINVAL, "batch is NULL");
    if (nsteps < 0) return report_error(LB_RD_EINVAL, "nsteps must be >= 0");
    for (size_t i = 0; i < b->inited.size(); ++i)
        if (!b->inited[i])
            return report_error(LB_RD_EINVAL, "lb_rd_batch_step: instance " + std::to_string(i) + " not initialised");
    if (nsteps == 0) return LB_RD_OK;
    const int K = b->steps_per_launch;
    if (K >= 2 && !uses_tb2(b)) {
        // depth-K launches; the last launch of the call (K steps, or the r =
        // nsteps % K left over: one depth-r launch, a single step for r = 1)
        // writes the densities
        const int64_t q = nsteps / K, r = nsteps % K;
        int rc = run_multi(b, r == 0 ? q - 1 : q);
        if (rc) return rc;
        const int d = r == 0 ? K : (int)r;
        cudaError_t e = d == 1 ? launch_one(b, b->cur, true) : launch_deep(b, d, b->cur, true);
        if (e) return cuda_err(e, "batch step kernel");
        b->cur ^= 1;
        b->t += d;
        b->launches++;
        return LB_RD_OK;
    }
    int64_t body = nsteps - 1;  // the last step also writes the densities
    if (K >= 2 && body >= K) {
        const int64_t n_two = body / K;
        body -= K * n_two;
        int rc = run_multi(b, n_two);
        if (rc) return rc;
    }
    if (b->graph_steps > 0 && body >= b->graph_steps) {
        if (!b->graph[b->cur]) {
            int rc = capture_graph(b, b->cur);
            if (rc) return rc;
        }
        const int64_t reps = body / b->graph_steps;
        for (int64_t r = 0; r < reps; ++r) {
            cudaError_t e = cudaGraphLaunch(b->graph[b->cur], b->stream);
            if (e) return cuda_err(e, "graph launch");
        }
        b->launches += reps * b->graph_steps;
        b->t += reps * b->graph_steps;  // even: the parity is unchanged
        body -= reps * b->graph_steps;
    }
    for (int64_t k = 0; k <= body; ++k) {
        cudaError_t e = launch_one(b, b->cur, k == body);
        if (e) return cuda_err(e, "batch step kernel");
        b->cur ^= 1;
        b->t++;
        b->launches++;
    }
    return LB_RD_OK;
}

int lb_rd_batch_set_steps_per_launch(lb_rd_batch *b, int32_t k) {
    if (!b) return report_error(LB_RD_EINVAL, "batch is NULL");
    if (k < 1 || k > 8) return report_error(LB_RD_EINVAL, "steps per launch must be in [1, 8]");
    if (k >= 2 && !b->deep_ok && !(k == 2 && b->tb_ok))
        return report_error(LB_RD_EINVAL, "2 .. 8 steps per launch need FP32 or 16-bit deviation instances with two "
                                          "state copies");
    if (k > 5 && half_batch(b))
        return report_error(LB_RD_EINVAL, "16-bit deviation storage: at most 5 steps per launch");
    cudaStreamSynchronize(b->stream);
    if (k >= 2 && !(k == 2 && b->tb_ok)) {
        cudaError_t e = plan_deep(b, k);
        if (e) return cuda_err(e, "lb_rd_batch_set_steps_per_launch");
    }
    if (k != b->steps_per_launch) drop_graphs(b);  // the multi-step graphs hold launches of the old K
    b->steps_per_launch = k;
    return LB_RD_OK;
}
int lb_rd_batch_moments(lb_rd_batch *b, int32_t idx, double *rho_out, double *mass_out, int is_device) {
    if (!b) return report_error(LB_RD_EINVAL, "batch is NULL");
    if (idx < 0 || idx >= (int)b->cfgs.size()) return report_error(LB_RD_EINVAL, "index out of range");
    const lb_rd_config &c = b->cfgs[idx];
    const void *rho = b->rho + b->rho_off[idx];
    const size_t n = (size_t)b->S * c.ny * c.nx;
    if (rho_out) {
        double *dst = rho_out;
        if (!is_device) {
            int rc = batch_stage(b, n);
            if (rc) return rc;
            dst = b->stage;
        }
        cudaError_t e = lbrd::launch_rho_export(b->prec, b->S, rho, c.nx, c.ny, b->pitch[idx], dst, b->stream);
        if (!e && !is_device) e = cudaMemcpyAsync(rho_out, b->stage, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e) return cuda_err(e, "batch rho export");
        b->launches++;
    }
    if (mass_out) {
        cudaError_t e = lbrd::launch_mass(b->prec, b->S, rho, c.nx, c.ny, b->pitch[idx], b->partials, b->counter,
                                          b->mass, b->stream);
        if (!e)
            e = cudaMemcpyAsync(mass_out, b->mass, b->S * sizeof(double),
                                is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
        if (e) return cuda_err(e, "batch mass");
        b->launches++;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e) return cuda_err(e, "batch moments sync");
    return LB_RD_OK;
}

int lb_rd_batch_get_time(const lb_rd_batch *b, int64_t *t, int64_t *launches) {
    if (!b) return report_error(LB_RD_EINVAL, "batch is NULL");
    if (t) *t = b->t;
    if (launches) *launches = b->launches;
    return LB_RD_OK;
}

}  // extern "C"
