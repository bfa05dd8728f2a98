// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbrd_common.cuh"

namespace lbrd {

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

// FP64: one thread per site, no FMA contraction (bit-reproducible).
StepShape step_shape_f64(int64_t nx, int64_t ny);
cudaError_t launch_step_f64(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_init_f64(int Q, int S, const InitArgs &a, cudaStream_t st);

// FP32: four sites per thread, 128-bit loads and stores, shuffle x-shift.
StepShape step_shape_f32(int64_t nx, int64_t ny);
cudaError_t launch_step_f32(int Q, int S, const StepArgs &a, cudaStream_t st);
cudaError_t launch_init_f32(int Q, int S, const InitArgs &a, cudaStream_t st);

// Reduced storage: float rho* plus (Q - 1) 16-bit deviations per species.
// half_kind: 0 = bf16, 1 = fp16.
StepShape step_shape_half(int64_t nx, int64_t ny);
cudaError_t launch_step_half(int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st);
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

// Bytes of one copy of the state (distributions only) in a given precision.
size_t state_plane_bytes(int prec, int Q, int S, int64_t ny, int64_t pitch);

}  // namespace lbrd
