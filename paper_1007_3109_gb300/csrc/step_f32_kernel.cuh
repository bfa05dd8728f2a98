// FP32 fused collide-and-stream step (the HBM-bound hot path): kernel
// template shared by the launch variants, the single-simulation path and the
// batched path.
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
//
// Template parameters of a launch variant: BX threads along x (a multiple of
// 32, each thread 4 sites), BY rows per tile, MINB the minimum resident blocks
// per SM requested from the register allocator, CACHE the cache policy
// (0: read-only path loads, default stores; 1: loads that skip L1 allocation
// and evict-first streaming stores).
#pragma once

#include "lbrd_kernels.h"

namespace lbrd {
namespace f32 {

constexpr int kVec = 4;

template <int CACHE>
__device__ __forceinline__ float4 ldv4(const float *p) {
    if (CACHE == 1) {
        float4 v;
        asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p));
        return v;
    }
    return __ldg(reinterpret_cast<const float4 *>(p));
}

template <int CACHE>
__device__ __forceinline__ void stv4(float *p, float4 v) {
    if (CACHE == 1) __stcs(reinterpret_cast<float4 *>(p), v);
    else *reinterpret_cast<float4 *>(p) = v;
}

// One row segment of 4 * 32 * (BX / 32) sites: the fused step for the four
// sites (x0 .. x0 + 3, y) of the calling thread.  Every lane of the warp must
// call it (the column shifts use warp shuffles); lanes with x0 >= nx or
// y >= ny load valid data but store nothing.
template <int Q, int S, int CACHE>
__device__ __forceinline__ void tile_f32(const StepArgs &a, int64_t x0, int64_t y, int lane, double (&acc)[S]) {
    using L = Lattice<Q>;
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    const bool live = (x0 < nx) && (y < ny);
    // Dead lanes load from a valid aligned column so that every lane of the
    // warp can take part in the shuffles.
    const int64_t xc = x0 < nx ? x0 : 0;
    const int64_t yc = y < ny ? y : 0;
    const int64_t xl = xc == 0 ? nx - 1 : xc - 1;                      // column left of the vector
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
            const float4 v = ldv4<CACHE>(row + xc);
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
            for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i][j]);
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

    if (!live) return;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float om = (float)a.omega[s];
        const float c1 = rn_sub(1.f, om);
        float wt[L::kClasses][kVec];
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            const float t = rn_fma(om, rho[s][j], R[s][j]);
#pragma unroll
            for (int c = 0; c < L::kClasses; ++c) wt[c][j] = rn_mul(L::template wc<float>(c), t);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int c = L::wclass(i);
            float4 o;
            o.x = rn_fma(c1, f[s][i][0], wt[c][0]);
            o.y = rn_fma(c1, f[s][i][1], wt[c][1]);
            o.z = rn_fma(c1, f[s][i][2], wt[c][2]);
            o.w = rn_fma(c1, f[s][i][3], wt[c][3]);
            stv4<CACHE>(dst + (int64_t)(s * Q + i) * plane + y * pitch + x0, o);
        }
        if (a.rho_out)
            stv4<CACHE>(static_cast<float *>(a.rho_out) + (int64_t)s * plane + y * pitch + x0,
                        make_float4(rho[s][0], rho[s][1], rho[s][2], rho[s][3]));
        if (a.mass_out) {
            // four sites summed in FP32, one FP64 add per tile (GB300's FP64
            // rate is a small fraction of its FP32 rate)
            float part = 0.f;
#pragma unroll
            for (int j = 0; j < kVec; ++j)
                if (x0 + j < nx) part += rho[s][j];
            acc[s] += (double)part;
        }
    }
}

// Persistent grid (or one block per tile when gridDim.x == ntiles): each
// block walks tiles of BX * 4 columns x BY rows in row-major tile order, so
// the resident blocks sweep a contiguous band of rows.
template <int Q, int S, int BX, int BY, int MINB, int CACHE>
__global__ void __launch_bounds__(BX *BY, MINB) step_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
        tile_f32<Q, S, CACHE>(a, (tx * BX + threadIdx.x) * kVec, ty * BY + threadIdx.y, lane, acc);
    }
    if (a.mass_out) block_mass_reduce<S, BX * BY>(acc, a.partials, a.counter, a.mass_out);
}

template <int BX, int BY>
inline void tiles_for(int64_t nx, int64_t ny, int64_t *tiles_x, int64_t *ntiles) {
    const int64_t nvec = (nx + kVec - 1) / kVec;
    *tiles_x = (nvec + BX - 1) / BX;
    *ntiles = *tiles_x * ((ny + BY - 1) / BY);
}

// per_tile = true: one block per tile; otherwise the persistent grid.
template <int Q, int S, int BX, int BY, int MINB, int CACHE>
cudaError_t launch_shape(const StepArgs &a, cudaStream_t st, bool per_tile) {
    int64_t tiles_x, ntiles;
    tiles_for<BX, BY>(a.nx, a.ny, &tiles_x, &ntiles);
    auto kern = step_kernel<Q, S, BX, BY, MINB, CACHE>;
    const unsigned grid = per_tile ? (unsigned)ntiles : persistent_blocks(kern, BX * BY, ntiles);
    kern<<<grid, dim3(BX, BY), 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int BX, int BY, int MINB, int CACHE>
cudaError_t dispatch_shape(int Q, int S, const StepArgs &a, cudaStream_t st, bool per_tile) {
    if (Q == 9 && S == 1) return launch_shape<9, 1, BX, BY, MINB, CACHE>(a, st, per_tile);
    if (Q == 9 && S == 2) return launch_shape<9, 2, BX, BY, MINB, CACHE>(a, st, per_tile);
    if (Q == 5 && S == 1) return launch_shape<5, 1, BX, BY, MINB, CACHE>(a, st, per_tile);
    if (Q == 5 && S == 2) return launch_shape<5, 2, BX, BY, MINB, CACHE>(a, st, per_tile);
    return cudaErrorInvalidValue;
}

}  // namespace f32
}  // namespace lbrd
