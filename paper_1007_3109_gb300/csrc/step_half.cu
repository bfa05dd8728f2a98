// Reduced-storage step: initialisation kernel and launchers.  The kernel
// body (and the storage scheme) is in step_half_kernel.cuh.
#include "step_half_kernel.cuh"

namespace lbrd {

namespace {

using half::kBX;
using half::kBY;
using half::kNT;
using half::kVec;
using half::f2h;
using half::step_half_kernel;

template <int Q, int S, int H>
__global__ void __launch_bounds__(256) init_half_kernel(InitArgs a) {
    const int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= a.nx) return;
    const int64_t plane = a.plane;
    const size_t species_bytes = (size_t)plane * (4 + 2 * (Q - 1));
    float f[S][Q], rho[S], R[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float r0 = (float)a.rho0[((int64_t)s * a.ny + y) * a.nx + x];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = rn_mul(weight<Q, float>(i), r0);
        float r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i]);
        rho[s] = r;
    }
    reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        char *base = static_cast<char *>(a.dst) + (size_t)s * species_bytes;
        reinterpret_cast<float *>(base)[y * a.pitch + x] = rn_add(rho[s], R[s]);
        unsigned short *g = reinterpret_cast<unsigned short *>(base + (size_t)plane * 4);
        const float c1 = rn_sub(1.f, (float)a.omega[s]);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            g[(int64_t)(i - 1) * plane + y * a.pitch + x] =
                (unsigned short)f2h<H>(rn_mul(c1, rn_fma(-weight<Q, float>(i), rho[s], f[s][i])));
        if (a.rho_out) static_cast<float *>(a.rho_out)[(int64_t)s * plane + y * a.pitch + x] = rho[s];
    }
}

void tiles_for(int64_t nx, int64_t ny, int64_t *tiles_x, int64_t *ntiles) {
    const int64_t nvec = (nx + kVec - 1) / kVec;
    *tiles_x = (nvec + kBX - 1) / kBX;
    *ntiles = *tiles_x * ((ny + kBY - 1) / kBY);
}

template <int Q, int S, int H>
cudaError_t launch_tiles(const StepArgs &a, cudaStream_t st) {
    int64_t tiles_x, ntiles;
    tiles_for(a.nx, a.ny, &tiles_x, &ntiles);
    const unsigned grid = persistent_blocks(step_half_kernel<Q, S, H>, kNT, ntiles);
    step_half_kernel<Q, S, H><<<grid, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int H>
cudaError_t dispatch_step(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tiles<9, 1, H>(a, st);
    if (Q == 9 && S == 2) return launch_tiles<9, 2, H>(a, st);
    if (Q == 5 && S == 1) return launch_tiles<5, 1, H>(a, st);
    if (Q == 5 && S == 2) return launch_tiles<5, 2, H>(a, st);
    return cudaErrorInvalidValue;
}

template <int H>
cudaError_t dispatch_init(int Q, int S, const InitArgs &a, cudaStream_t st) {
    const dim3 g((unsigned)((a.nx + 255) / 256), (unsigned)a.ny), b(256);
    if (Q == 9 && S == 1) init_half_kernel<9, 1, H><<<g, b, 0, st>>>(a);
    else if (Q == 9 && S == 2) init_half_kernel<9, 2, H><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 1) init_half_kernel<5, 1, H><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 2) init_half_kernel<5, 2, H><<<g, b, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace

StepShape step_shape_half(int64_t, int64_t) { return {dim3(max_persistent_blocks()), dim3(kBX, kBY)}; }

namespace {
template <int Q, int S, int H, int BX, int BY, int MINB>
cudaError_t launch_shape(const StepArgs &a, cudaStream_t st) {
    const int64_t nvec = (a.nx + kVec - 1) / kVec;
    const int64_t tiles_x = (nvec + BX - 1) / BX;
    const int64_t ntiles = tiles_x * ((a.ny + BY - 1) / BY);
    auto kern = half::step_half_shape<Q, S, H, BX, BY, MINB>;
    kern<<<persistent_blocks(kern, BX * BY, ntiles), dim3(BX, BY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}
template <int H, int BX, int BY, int MINB>
cudaError_t dispatch_shape(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_shape<9, 1, H, BX, BY, MINB>(a, st);
    if (Q == 9 && S == 2) return launch_shape<9, 2, H, BX, BY, MINB>(a, st);
    if (Q == 5 && S == 1) return launch_shape<5, 1, H, BX, BY, MINB>(a, st);
    if (Q == 5 && S == 2) return launch_shape<5, 2, H, BX, BY, MINB>(a, st);
    return cudaErrorInvalidValue;
}
template <int H>
cudaError_t dispatch_variant(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    switch (v) {
        case 0: return dispatch_step<H>(Q, S, a, st);
        case 1: return dispatch_shape<H, 64, 2, 5>(Q, S, a, st);
        case 2: return dispatch_shape<H, 32, 4, 4>(Q, S, a, st);
        case 3: return dispatch_shape<H, 128, 2, 2>(Q, S, a, st);
        case 4: return dispatch_shape<H, 64, 2, 6>(Q, S, a, st);
        case 5: case 6: case 7: case 8: case 9: case 10:
            return launch_step_half_deep(v - 5, Q, S, H, a, st);
        case 11: case 12: case 13: case 14: case 15: case 16:
            return launch_step_half_pair(v - 11, Q, S, H, a, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

// One step per launch (tile shape, register budget), then temporal blocking to
// depth K (step_half_deep_kernel.cuh): hdeep<K>_<threads>_minb<blocks>[_s<rows staged>],
// and with two columns per lane (step_half_pair_kernel.cuh, nx a multiple of 8): hpair<K>_.
const char *const kHalfVariantNames[] = {"half_64x2",          "half_64x2_minb5",  "half_32x4_minb4",
                                         "half_128x2_minb2",   "half_64x2_minb6",  "hdeep2_128_minb4",
                                         "hdeep3_128_minb3",   "hdeep4_128_minb2", "hdeep4_128_minb3",
                                         "hdeep3_128_minb3_s5", "hdeep5_128_minb2", "hpair4_128_minb2",
                                         "hpair4_128_minb3",   "hpair5_128_minb2", "hpair3_128_minb3",
                                         "hpair6_128_minb2",   "hpair2_128_minb4"};
const int kHalfVariantSteps[] = {1, 1, 1, 1, 1, 2, 3, 4, 4, 3, 5, 4, 4, 5, 3, 6, 2};
const int kHalfVariantNx[] = {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 8};
const int kHalfVariantCount = 17;

cudaError_t launch_step_half_variant(int v, int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st) {
    if (a.nx % kVec) return cudaErrorInvalidValue;
    return half_kind ? dispatch_variant<1>(v, Q, S, a, st) : dispatch_variant<0>(v, Q, S, a, st);
}

cudaError_t launch_step_half(int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st) {
    if (a.nx % kVec) return cudaErrorInvalidValue;
    return half_kind ? dispatch_step<1>(Q, S, a, st) : dispatch_step<0>(Q, S, a, st);
}

cudaError_t launch_init_half(int Q, int S, int half_kind, const InitArgs &a, cudaStream_t st) {
    return half_kind ? dispatch_init<1>(Q, S, a, st) : dispatch_init<0>(Q, S, a, st);
}

// One block per tile instead of the persistent grid (allocation-free entry).
int64_t step_tiles_half(int64_t nx, int64_t ny) {
    int64_t tiles_x, ntiles;
    tiles_for(nx, ny, &tiles_x, &ntiles);
    return ntiles;
}

namespace {
template <int Q, int S, int H>
cudaError_t launch_per_tile(const StepArgs &a, cudaStream_t st) {
    int64_t tiles_x, ntiles;
    tiles_for(a.nx, a.ny, &tiles_x, &ntiles);
    step_half_kernel<Q, S, H><<<(unsigned)ntiles, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}
template <int H>
cudaError_t dispatch_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_per_tile<9, 1, H>(a, st);
    if (Q == 9 && S == 2) return launch_per_tile<9, 2, H>(a, st);
    if (Q == 5 && S == 1) return launch_per_tile<5, 1, H>(a, st);
    if (Q == 5 && S == 2) return launch_per_tile<5, 2, H>(a, st);
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_step_half_per_tile(int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st) {
    if (a.nx % kVec) return cudaErrorInvalidValue;
    return half_kind ? dispatch_per_tile<1>(Q, S, a, st) : dispatch_per_tile<0>(Q, S, a, st);
}

}  // namespace lbrd
