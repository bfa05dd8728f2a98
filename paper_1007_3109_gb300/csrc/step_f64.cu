// FP64 step kernels: a persistent grid over 32 x 4 site tiles running the
// per-site update of step_f64_kernel.cuh.  GB300's FP64 rate, not HBM, bounds
// them.
#include "lbrd_kernels.h"
#include "step_f64_kernel.cuh"

namespace lbrd {

namespace {

constexpr int kBX = 32, kBY = 4, kNT = kBX * kBY;

template <int Q, int S>
__global__ void __launch_bounds__(kNT) step_f64_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int64_t x = tx * kBX + threadIdx.x;
        const int64_t y = ty * kBY + threadIdx.y;
        if (x >= a.nx || y >= a.ny) continue;
        f64::site_f64<Q, S>(a, x, y, acc);
    }
    if (a.mass_out) block_mass_reduce<S, kNT>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S>
__global__ void __launch_bounds__(kNT) init_f64_kernel(InitArgs a) {
    const int64_t x = (int64_t)blockIdx.x * kBX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * kBY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    double *__restrict__ dst = static_cast<double *>(a.dst);
    double f[S][Q], rho[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double r0 = a.rho0[((int64_t)s * a.ny + y) * a.nx + x];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = __dmul_rn(weight<Q, double>(i), r0);
        double r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = __dadd_rn(r, f[s][i]);
        rho[s] = r;
    }
    double R[S];
    reaction_f64<S>(a.rkind, a.kappa, a.F, a.k, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double om = a.omega[s];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double w = weight<Q, double>(i);
            const double feq = __dmul_rn(w, rho[s]);
            dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] =
                __dadd_rn(__dadd_rn(f[s][i], __dmul_rn(__dsub_rn(feq, f[s][i]), om)), __dmul_rn(w, R[s]));
        }
        if (a.rho_out) static_cast<double *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
    }
}

dim3 grid_for(int64_t nx, int64_t ny) {
    return dim3((unsigned)((nx + kBX - 1) / kBX), (unsigned)((ny + kBY - 1) / kBY));
}

template <int Q, int S>
cudaError_t launch_tiles(const StepArgs &a, cudaStream_t st) {
    const int64_t tiles_x = (a.nx + kBX - 1) / kBX;
    const int64_t ntiles = tiles_x * ((a.ny + kBY - 1) / kBY);
    const unsigned grid = persistent_blocks(step_f64_kernel<Q, S>, kNT, ntiles);
    step_f64_kernel<Q, S><<<grid, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

}  // namespace

StepShape step_shape_f64(int64_t, int64_t) { return {dim3(max_persistent_blocks()), dim3(kBX, kBY)}; }

cudaError_t launch_step_f64(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tiles<9, 1>(a, st);
    if (Q == 9 && S == 2) return launch_tiles<9, 2>(a, st);
    if (Q == 5 && S == 1) return launch_tiles<5, 1>(a, st);
    if (Q == 5 && S == 2) return launch_tiles<5, 2>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_f64(int Q, int S, const InitArgs &a, cudaStream_t st) {
    const dim3 g = grid_for(a.nx, a.ny), b(kBX, kBY);
    if (Q == 9 && S == 1) init_f64_kernel<9, 1><<<g, b, 0, st>>>(a);
    else if (Q == 9 && S == 2) init_f64_kernel<9, 2><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 1) init_f64_kernel<5, 1><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 2) init_f64_kernel<5, 2><<<g, b, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// One block per tile instead of the persistent grid (allocation-free entry).
int64_t step_tiles_f64(int64_t nx, int64_t ny) { return ((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY); }

namespace {
template <int Q, int S>
cudaError_t launch_per_tile(const StepArgs &a, cudaStream_t st) {
    const int64_t tiles_x = (a.nx + kBX - 1) / kBX;
    const int64_t ntiles = tiles_x * ((a.ny + kBY - 1) / kBY);
    step_f64_kernel<Q, S><<<(unsigned)ntiles, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_step_f64_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_per_tile<9, 1>(a, st);
    if (Q == 9 && S == 2) return launch_per_tile<9, 2>(a, st);
    if (Q == 5 && S == 1) return launch_per_tile<5, 1>(a, st);
    if (Q == 5 && S == 2) return launch_per_tile<5, 2>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbrd
