// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lb_rd.h"
#include "lbrd_common.cuh"

namespace lbrd {

static_assert(kMaxSpecies == LB_RD_MAX_SPECIES && kMaxReactions == LB_RD_MAX_REACTIONS, "capacities must agree");

// Row pitch of every state, density and staging plane: nx rounded up to a
// multiple of 32 elements (128-byte rows in FP32, 256 in FP64).
inline int64_t state_pitch(int64_t nx) { return (nx + 31) / 32 * 32; }

// Relaxation rates and reaction constants of a configuration in kernel form:
// omega_s = 1 / tau_s (0 beyond nspecies) and the network of a mass-action
// source (zeroed otherwise).
inline void fill_reaction(const lb_rd_config &c, double *omega, int *rkind, double *kappa, double *F, double *k,
                          Network *net) {
    for (int s = 0; s < kMaxSpecies; ++s) omega[s] = s < c.nspecies ? 1.0 / c.tau[s] : 0.0;
    *rkind = c.reaction.kind;
    *kappa = c.reaction.kappa;
    *F = c.reaction.F;
    *k = c.reaction.k;
    *net = Network{};
    if (c.reaction.kind == LB_RD_REACTION_MASS_ACTION) {
        net->nr = c.reaction.nreactions;
        for (int r = 0; r < c.reaction.nreactions && r < kMaxReactions; ++r) {
            net->rate[r] = c.reaction.rate[r];
            for (int j = 0; j < kMaxSpecies; ++j) {
                net->order[r][j] = c.reaction.order[r][j];
                net->change[r][j] = c.reaction.change[r][j];
            }
        }
    }
}

// Resident blocks per SM of a kernel at a block size (cached per device and
// kernel) times the SM count, capped by the work.  Persistent kernels walk
// their tiles with a grid-stride loop over this many blocks.
unsigned occupancy_blocks(const void *kernel, int nthreads, size_t smem);
template <typename K>
unsigned persistent_blocks(K kernel, int nthreads, int64_t ntiles, size_t smem = 0) {
    const unsigned full = occupancy_blocks(reinterpret_cast<const void *>(kernel), nthreads, smem);
    return (unsigned)(ntiles < (int64_t)full ? (ntiles > 0 ? ntiles : 1) : full);
}
// Upper bound of persistent_blocks over all kernels (sizes mass partials).
unsigned max_persistent_blocks();

// Launch shape of the step kernel of one precision, used to size the
// per-block mass partials.
struct StepShape {
    dim3 grid, block;
};

// General step: 1 .. 4 species, mass-action networks; prec 0 = FP64 (no FMA
// contraction, bit-reproducible), otherwise FP32.  One thread per site.
struct GeneralVariant {
    const char *name;
    int sites;  // consecutive sites per thread; the variant needs nx % sites == 0
};
extern const GeneralVariant kGeneralVariants[];
extern const int kGeneralVariantCount;  // FP32; FP64 has variant 0 only
cudaError_t launch_step_general(int prec, int Q, int S, const StepArgs &a, cudaStream_t st, int variant);
cudaError_t launch_init_general(int prec, int Q, int S, const InitArgs &a, cudaStream_t st);

// In-place (AA) step: phase 0 for t even (natural in, pushed-and-swapped
// out), 1 for t odd; a.src == a.dst.  prec 0 = FP64, otherwise FP32.  And the
// export of a pushed-and-swapped state as packed FP64 [s][i][y][x].
// FP32 launch variants (sites per thread as in GeneralVariant); FP64 has 0.
extern const GeneralVariant kAAVariants[];
extern const int kAAVariantCount;
cudaError_t launch_step_aa(int prec, int Q, int S, int phase, const StepArgs &a, cudaStream_t st, int variant);
cudaError_t launch_export_swapped(int prec, int Q, int S, const void *state, int64_t nx, int64_t ny, int64_t pitch,
                                  double *out, cudaStream_t st);

// FP64: one thread per site, no FMA contraction (bit-reproducible).
StepShape step_shape_f64(int64_t nx, int64_t ny);
cudaError_t launch_step_f64(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_init_f64(int Q, int S, const InitArgs &a, cudaStream_t st);

// FP32: four sites per thread, 128-bit loads and stores, shuffle x-shift.
// Launch variants differ in tile shape, register budget and cache policy.
struct F32Variant {
    const char *name;
    int bx, by, minb, cache;  // cache: 0/1 register path policies, 2 bulk-copy ring, 3 temporal blocking,
                              // 4 temporal blocking to depth by with the levels in registers
    int steps;                // time steps per launch
    int nx_multiple;          // the variant needs nx % nx_multiple == 0
};
extern const F32Variant kF32Variants[];
extern const int kF32VariantCount;
cudaError_t launch_step_f32_variant(int v, int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_f32_variant_b(int v, int Q, int S, const StepArgs &a, cudaStream_t st, bool per_tile);
cudaError_t launch_step_f32_bulk(int v, int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_f32_tb2(int v, int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_f32_deep(int v, int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_f32_pair(int v, int Q, int S, const StepArgs &a, cudaStream_t st);
StepShape step_shape_f32(int64_t nx, int64_t ny);
cudaError_t launch_step_f32(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_init_f32(int Q, int S, const InitArgs &a, cudaStream_t st);

// Reduced storage: float rho* plus (Q - 1) 16-bit deviations per species.
// half_kind: 0 = bf16, 1 = fp16.
StepShape step_shape_half(int64_t nx, int64_t ny);
cudaError_t launch_step_half(int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);
extern const char *const kHalfVariantNames[];
extern const int kHalfVariantSteps[];  // time steps per launch of each variant
extern const int kHalfVariantNx[];     // the variant needs nx % kHalfVariantNx[v] == 0
extern const int kHalfVariantCount;
// Depth-K launches of the 16-bit deviation step (variant v of that family).
cudaError_t launch_step_half_deep(int v, int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_half_pair(int v, int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_half_variant(int v, int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);
cudaError_t launch_init_half(int Q, int S, int half_kind, const InitArgs &a, cudaStream_t st);

// One block per tile (no persistent grid) and the tile counts of those
// launches: used by the allocation-free entry point, whose per-block scratch
// is sized from the launch.
int64_t step_tiles_f64(int64_t nx, int64_t ny);
int64_t step_tiles_f32(int64_t nx, int64_t ny);
int64_t step_tiles_half(int64_t nx, int64_t ny);
cudaError_t launch_step_f64_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_f32_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_step_half_per_tile(int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);

// Post-collision distributions of the stored state as packed FP64
// [s][i][y][x].  prec: lb_rd_precision.
cudaError_t launch_export(int prec, int Q, int S, const void *state, int64_t nx, int64_t ny, int64_t pitch,
                          double *out, cudaStream_t st);

// rho cache ([s][y][pitch] in double (prec 0) or float) to packed FP64
// [s][y][x], and its global FP64 sum per species.
cudaError_t launch_rho_export(int prec, int S, const void *rho, int64_t nx, int64_t ny, int64_t pitch,
                              double *out, cudaStream_t st);
size_t mass_partials_needed(int64_t nx, int64_t ny);
cudaError_t launch_mass(int prec, int S, const void *rho, int64_t nx, int64_t ny, int64_t pitch,
                        double *partials, unsigned int *counter, double *mass, cudaStream_t st);

// Batched step: one persistent launch over the combined (instance x tile)
// work list.  Tiles are 256 x 2 sites (64 x 2 threads, 4 sites each); the
// instance of global tile t is the last item with tile_begin <= t.
struct BatchItem {
    StepArgs a;          // per-instance grid, parameters and buffers
    int64_t tiles_x;     // tiles per row of tiles, ceil(ceil(nx / 4) / 64)
    int64_t tile_begin;  // first global tile of this instance
    int aa;              // FP32: 0 two state copies; in place (a.src == a.dst), phase A (t even) / B:
                         // 1 / 2 four sites per thread (nx % 4 == 0), 3 / 4 one site per thread
};
// Batched two-step launches over (strip, row) units: one item per instance
// (FP32, two state copies, nx % batch_tb2_strip() == 0); the units of item k
// are [unit_begin, unit_begin + (nx / strip) * ny).
struct TbwItem {
    StepArgs a;
    int64_t unit_begin;
};
int batch_tb2_strip();
cudaError_t launch_batch_tb2(const TbwItem *items, int n, int64_t total_units, int Q, int S, cudaStream_t st);
// Batched K-step launches (K = 2 .. 8; FP32, two state copies): the depth-K
// kernel over the (band, strip) units of a list of grids (for K <= 5 (D2Q9)
// or 6 (D2Q5) its two-column form).  Item k's units
// are [unit_begin, unit_begin + nstrips * ceil(ny / band)), strips of the
// kernel's output columns (34 - 2K, or 64 - 2 HL) fastest.  batch_deep_plan
// fills nstrips and band of every item (one band height in rows for the whole
// list, chosen for the launch's warp count) and returns the total unit count,
// or -1 for an unsupported K.  v16: every grid has nx
// and pitch multiples of 4 (16-byte staging).  emit: the launch also writes
// rho(t + K) of every item to its a.rho_out (the last launch of a call).
// rk: the reaction kind that every item has (a.rkind), or -1 when they differ
// (list_reaction_kind); selects a kernel with the kind fixed at compile time.
struct DeepItem {
    StepArgs a;
    int64_t unit_begin, nstrips, band;
};
// The same over 16-bit deviation storage (K = 2 .. 5; half_kind 0 bf16, 1 fp16;
// any nx a multiple of 4): the two-column depth-K kernel of
// step_half_pair_kernel.cuh when every grid has nx a multiple of 8 (v8, which
// the caller passes to the launch as the plan found it), else the one-column
// kernel of step_half_deep_kernel.cuh.
int64_t batch_half_deep_plan(int K, int Q, int S, int half_kind, DeepItem *items, int n);
// Default steps per launch of a 16-bit list: 4, with either kernel (the
// two-column form spills at K = 5).
int batch_half_default_k();
cudaError_t launch_batch_half_deep(int K, int Q, int S, int half_kind, const DeepItem *items, int n,
                                   int64_t total_units, bool emit, int rk, bool v8, cudaStream_t st);
bool batch_deep_depth_ok(int K);
// Default steps per launch of a list of grids: 5 (D2Q9) / 6 (D2Q5), the
// fastest two-column forms over a list (the grid's parameters read from a
// per-warp shared copy where they are used).
int batch_deep_default_k(int Q);
int64_t batch_deep_plan(int K, int Q, int S, bool v16, DeepItem *items, int n);
cudaError_t launch_batch_deep(int K, int Q, int S, bool v16, const DeepItem *items, int n, int64_t total_units,
                              bool emit, int rk, cudaStream_t st);
// Every item of a host-side list has nx and the row pitch multiples of 8.
inline bool list_nx8(const DeepItem *items, int n) {
    for (int i = 0; i < n; ++i)
        if (items[i].a.nx % 8 != 0 || items[i].a.pitch % 8 != 0) return false;
    return true;
}
// The reaction kind every item of a host-side list has, or -1.
inline int list_reaction_kind(const DeepItem *items, int n) {
    if (n <= 0) return -1;
    for (int i = 1; i < n; ++i)
        if (items[i].a.rkind != items[0].a.rkind) return -1;
    return items[0].a.rkind;
}
int64_t batch_tiles_x(int64_t nx);
int64_t batch_tiles(int64_t nx, int64_t ny);
// mode: 0 FP32 storage, 1 bf16 deviations, 2 fp16 deviations, 3 FP64,
// 4 FP32 with in-place instances (BatchItem::aa).
int batch_mode(int precision);
cudaError_t launch_batch_init(int mode, int Q, int S, const InitArgs &a, cudaStream_t st);
cudaError_t launch_batch_step(int mode, int Q, int S, const BatchItem *items, int n, int64_t total_tiles,
                             cudaStream_t st);

// rho(t) from the previous state copy f*(t - 1) into the density cache
// ([s][y][pitch], double for FP64, float otherwise), bitwise equal to the rho
// the step kernel computed for time t.
cudaError_t launch_pull_rho(int prec, int Q, int S, const void *prev_state, int64_t nx, int64_t ny, int64_t pitch,
                            void *rho, cudaStream_t st);

// Bytes of one copy of the state (distributions only) in a given precision.
size_t state_plane_bytes(int prec, int Q, int S, int64_t ny, int64_t pitch);

}  // namespace lbrd
