// FP32 fused collide-and-stream step (the HBM-bound hot path).
//
// One pass over the state per time step: every thread owns four consecutive
// sites of one row and, for every species s and velocity i,
//   1. pulls f_i,s(x, t + 1) = f*_i,s(x - e_i, t) (Eq. relax read as a pull,
//      periodic wrap) with one aligned 128-bit load of its own columns of row
//      y - e_iy; the +-1 column shift is a warp shuffle of the neighbouring
//      lane's vector, and only the lanes at a warp edge or at the periodic
//      edge issue one extra 4-byte load,
//   2. sums rho_s = sum_i f_i,s in index order,
// then evaluates R_s(rho_1..rho_S) in registers (all species are in the same
// thread), relaxes with the source,
//   f*_i,s = f_i,s + (w_i rho_s - f_i,s) / tau_s + w_i R_s
//          = (1 - omega_s) f_i,s + w_i (omega_s rho_s + R_s),
// and writes f*_i,s with one aligned 128-bit store per (s, i).  Optionally it
// also writes rho_s(t + 1) and reduces sum_x rho_s(t + 1) in FP64.
//
// Algorithmic traffic: 2 * 4 * S * Q bytes per site (read once, write once):
// 144 B/site for D2Q9 with two species.
#include "lbrd_kernels.h"

namespace lbrd {

namespace {

constexpr int kBX = 64, kBY = 2, kNT = kBX * kBY, kVec = 4;

template <int Q, int S>
__global__ void __launch_bounds__(kNT) step_f32_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    const int lane = threadIdx.x & 31;
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;

    // Persistent grid: each block walks tiles of kBX * 4 columns x kBY rows in
    // row-major tile order, so the resident blocks sweep a contiguous band.
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int64_t x0 = (tx * kBX + threadIdx.x) * kVec;
    const int64_t y = ty * kBY + threadIdx.y;
    const bool live = (x0 < nx) && (y < ny);
    // Dead lanes load from a valid aligned column so that every lane of the
    // warp can take part in the shuffles.
    const int64_t xc = x0 < nx ? x0 : 0;
    const int64_t yc = y < ny ? y : 0;
    const int64_t xl = xc == 0 ? nx - 1 : xc - 1;                   // column left of the vector
    const int64_t xr = (xc + kVec < nx) ? xc + kVec : xc + kVec - nx;  // column right of the vector
    const bool need_l = (lane == 0) || (xc == 0);
    const bool need_r = (lane == 31) || (xc + kVec >= nx);
    const bool straddle = xc + kVec > nx;  // only when nx % 4 != 0

    float f[S][Q][kVec];
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int64_t ys = wrap(yc - L::ey(i), ny);
            const float *row = src + (int64_t)(s * Q + i) * plane + ys * pitch;
            const float4 v = __ldg(reinterpret_cast<const float4 *>(row + xc));
            if (L::ex(i) == 0) {
                f[s][i][0] = v.x; f[s][i][1] = v.y; f[s][i][2] = v.z; f[s][i][3] = v.w;
            } else if (L::ex(i) == 1) {
                // pull from x - 1
                float left = __shfl_up_sync(kFullMask, v.w, 1);
                if (need_l) left = __ldg(row + xl);
                f[s][i][0] = left; f[s][i][1] = v.x; f[s][i][2] = v.y; f[s][i][3] = v.z;
            } else {
                // pull from x + 1
                float right = __shfl_down_sync(kFullMask, v.x, 1);
                if (need_r) right = __ldg(row + xr);
                f[s][i][0] = v.y; f[s][i][1] = v.z; f[s][i][2] = v.w; f[s][i][3] = right;
                if (straddle) {
                    // the last live column wraps to column 0
                    const float w0 = __ldg(row);
                    const int64_t jl = nx - 1 - xc;
#pragma unroll
                    for (int j = 0; j < kVec - 1; ++j)
                        if (j == jl) f[s][i][j] = w0;
                }
            }
        }
    }

    float rho[S][kVec];
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            float r = f[s][0][j];
#pragma unroll
            for (int i = 1; i < Q; ++i) r += f[s][i][j];
            rho[s][j] = r;
        }
    }

    float R[S][kVec];
    const float kappa = (float)a.kappa, F = (float)a.F, k = (float)a.k;
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
        float rj[S], Rj[S];
#pragma unroll
        for (int s = 0; s < S; ++s) rj[s] = rho[s][j];
        reaction_f32<S>(a.rkind, kappa, F, k, rj, Rj);
#pragma unroll
        for (int s = 0; s < S; ++s) R[s][j] = Rj[s];
    }

    if (live) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float om = (float)a.omega[s];
            const float c1 = 1.f - om;
            float wt[L::kClasses][kVec];
#pragma unroll
            for (int j = 0; j < kVec; ++j) {
                const float t = om * rho[s][j] + R[s][j];
#pragma unroll
                for (int c = 0; c < L::kClasses; ++c) wt[c][j] = L::template wc<float>(c) * t;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int c = L::wclass(i);
                float4 o;
                o.x = fmaf(c1, f[s][i][0], wt[c][0]);
                o.y = fmaf(c1, f[s][i][1], wt[c][1]);
                o.z = fmaf(c1, f[s][i][2], wt[c][2]);
                o.w = fmaf(c1, f[s][i][3], wt[c][3]);
                *reinterpret_cast<float4 *>(dst + (int64_t)(s * Q + i) * plane + y * pitch + x0) = o;
            }
            if (a.rho_out) {
                *reinterpret_cast<float4 *>(static_cast<float *>(a.rho_out) + (int64_t)s * plane + y * pitch + x0) =
                    make_float4(rho[s][0], rho[s][1], rho[s][2], rho[s][3]);
            }
            if (a.mass_out) {
#pragma unroll
                for (int j = 0; j < kVec; ++j)
                    if (x0 + j < nx) acc[s] += (double)rho[s][j];
            }
        }
    }
    }  // tile loop
    if (a.mass_out) block_mass_reduce<S, kNT>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S>
__global__ void __launch_bounds__(256) init_f32_kernel(InitArgs a) {
    using L = Lattice<Q>;
    const int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= a.nx) return;
    float f[S][Q], rho[S], R[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float r0 = (float)a.rho0[((int64_t)s * a.ny + y) * a.nx + x];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = weight<Q, float>(i) * r0;
        float r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r += f[s][i];
        rho[s] = r;
    }
    reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
    float *dst = static_cast<float *>(a.dst);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float om = (float)a.omega[s];
        const float t = om * rho[s] + R[s];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] = fmaf(1.f - om, f[s][i], weight<Q, float>(i) * t);
        if (a.rho_out) static_cast<float *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
    }
}

void tiles_for(int64_t nx, int64_t ny, int64_t *tiles_x, int64_t *ntiles) {
    const int64_t nvec = (nx + kVec - 1) / kVec;
    *tiles_x = (nvec + kBX - 1) / kBX;
    *ntiles = *tiles_x * ((ny + kBY - 1) / kBY);
}

template <int Q, int S>
cudaError_t launch_tiles(const StepArgs &a, cudaStream_t st) {
    int64_t tiles_x, ntiles;
    tiles_for(a.nx, a.ny, &tiles_x, &ntiles);
    const unsigned grid = persistent_blocks(step_f32_kernel<Q, S>, kNT, ntiles);
    step_f32_kernel<Q, S><<<grid, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

}  // namespace

StepShape step_shape_f32(int64_t nx, int64_t ny) {
    int64_t tiles_x, ntiles;
    tiles_for(nx, ny, &tiles_x, &ntiles);
    return {dim3(max_persistent_blocks()), dim3(kBX, kBY)};
}

cudaError_t launch_step_f32(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tiles<9, 1>(a, st);
    if (Q == 9 && S == 2) return launch_tiles<9, 2>(a, st);
    if (Q == 5 && S == 1) return launch_tiles<5, 1>(a, st);
    if (Q == 5 && S == 2) return launch_tiles<5, 2>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_f32(int Q, int S, const InitArgs &a, cudaStream_t st) {
    const dim3 g((unsigned)((a.nx + 255) / 256), (unsigned)a.ny), b(256);
    if (Q == 9 && S == 1) init_f32_kernel<9, 1><<<g, b, 0, st>>>(a);
    else if (Q == 9 && S == 2) init_f32_kernel<9, 2><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 1) init_f32_kernel<5, 1><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 2) init_f32_kernel<5, 2><<<g, b, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// One block per tile instead of the persistent grid: the launch used by the
// allocation-free entry point, whose per-block scratch is sized from the grid.
int64_t step_tiles_f32(int64_t nx, int64_t ny) {
    int64_t tiles_x, ntiles;
    tiles_for(nx, ny, &tiles_x, &ntiles);
    return ntiles;
}

namespace {
template <int Q, int S>
cudaError_t launch_per_tile(const StepArgs &a, cudaStream_t st) {
    int64_t tiles_x, ntiles;
    tiles_for(a.nx, a.ny, &tiles_x, &ntiles);
    step_f32_kernel<Q, S><<<(unsigned)ntiles, dim3(kBX, kBY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_step_f32_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_per_tile<9, 1>(a, st);
    if (Q == 9 && S == 2) return launch_per_tile<9, 2>(a, st);
    if (Q == 5 && S == 1) return launch_per_tile<5, 1>(a, st);
    if (Q == 5 && S == 2) return launch_per_tile<5, 2>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbrd
