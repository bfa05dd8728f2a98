// Reduced-storage step: FP32 arithmetic, per species and site one FP32 mass
// and Q - 1 sixteen-bit deviations (bf16 or fp16).
//
// The post-collision value of Eq. relax splits exactly into an equilibrium
// part and a deviation:
//   f*_i = f_i + (w_i rho - f_i) / tau + w_i R = w_i rho* + g_i,
//   rho* = rho + R,   g_i = (1 - 1/tau)(f_i - w_i rho),   sum_i g_i = 0.
// Stored per species: plane 0 = rho* (float), planes 1..Q-1 = g_1..g_{Q-1};
// g_0 = -sum_{i>=1} g_i is implied, so sum_i f*_i = rho* holds exactly in the
// stored values and the mass is carried at FP32 accuracy whatever the
// deviation format.  The pull of the next step is
//   f_i(x) = w_i rho*(x - e_i) + g_i(x - e_i),   i >= 1,
//   f_0(x) = w_0 rho*(x) - sum_{i>=1} g_i(x).
// Traffic per species and site: (4 + 2 (Q - 1)) bytes read and written,
// 80 B/site for D2Q9 with two species (144 B in FP32 storage).
//
// Thread layout as in the FP32 kernel: four consecutive sites of one row per
// thread, aligned 128-bit (rho*) and 64-bit (4 deviations) loads, +-1 column
// shifts through warp shuffles.  Needs nx % 4 == 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbrd_kernels.h"

namespace lbrd {
namespace half {

constexpr int kBX = 64, kBY = 2, kNT = kBX * kBY, kVec = 4;

template <int H>  // 0 = bf16, 1 = fp16
__device__ __forceinline__ float h2f(unsigned bits) {
    if (H == 0) return __uint_as_float((bits & 0xffffu) << 16);
    return __half2float(__ushort_as_half((unsigned short)(bits & 0xffffu)));
}

template <int H>
__device__ __forceinline__ unsigned f2h(float v) {
    if (H == 0) return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (unsigned)__half_as_ushort(__float2half_rn(v));
}

// Two values rounded to nearest even and packed (lo in bits 0-15): the bits
// of f2h(lo) | f2h(hi) << 16, in one paired conversion.
template <int H>
__device__ __forceinline__ unsigned f2h2(float lo, float hi) {
    if (H == 0) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&v);
    }
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

struct Cols {
    int64_t xc, xl, xr;
    bool need_l, need_r;
};

// Four consecutive deviations pulled from columns x0 - ex .. x0 + 3 - ex of
// one 16-bit row; ``raw`` returns the aligned word pair (columns x0..x0+3).
template <int H>
__device__ __forceinline__ void pull4h(const unsigned short *row, const Cols &c, int ex, float (&out)[kVec],
                                       uint2 &raw) {
    raw = __ldg(reinterpret_cast<const uint2 *>(row + c.xc));
    const float e0 = h2f<H>(raw.x), e1 = h2f<H>(raw.x >> 16), e2 = h2f<H>(raw.y), e3 = h2f<H>(raw.y >> 16);
    if (ex == 0) {
        out[0] = e0; out[1] = e1; out[2] = e2; out[3] = e3;
    } else if (ex == 1) {
        unsigned left = __shfl_up_sync(kFullMask, raw.y, 1) >> 16;
        if (c.need_l) left = __ldg(row + c.xl);
        out[0] = h2f<H>(left); out[1] = e0; out[2] = e1; out[3] = e2;
    } else {
        unsigned right = __shfl_down_sync(kFullMask, raw.x, 1);
        if (c.need_r) right = __ldg(row + c.xr);
        out[0] = e1; out[1] = e2; out[2] = e3; out[3] = h2f<H>(right);
    }
}

// rho* of one row at columns x0 - 1 .. x0 + 4.
__device__ __forceinline__ void row6(const float *row, const Cols &c, float (&out)[kVec + 2]) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(row + c.xc));
    float left = __shfl_up_sync(kFullMask, v.w, 1);
    float right = __shfl_down_sync(kFullMask, v.x, 1);
    if (c.need_l) left = __ldg(row + c.xl);
    if (c.need_r) right = __ldg(row + c.xr);
    out[0] = left; out[1] = v.x; out[2] = v.y; out[3] = v.z; out[4] = v.w; out[5] = right;
}

// The fused step for the four sites (x0 .. x0 + 3, y) of the calling thread.
// Every lane of the warp must call it (column shifts use warp shuffles).
template <int Q, int S, int H>
__device__ __forceinline__ void tile_half(const StepArgs &a, int64_t x0, int64_t y, int lane, double (&acc)[S]) {
    using L = Lattice<Q>;
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    const size_t species_bytes = (size_t)plane * (4 + 2 * (Q - 1));
    const char *__restrict__ src = static_cast<const char *>(a.src);
    char *__restrict__ dst = static_cast<char *>(a.dst);
    const bool live = (x0 < nx) && (y < ny);
    Cols c;
    c.xc = x0 < nx ? x0 : 0;
    const int64_t yc = y < ny ? y : 0;
    c.xl = c.xc == 0 ? nx - 1 : c.xc - 1;
    c.xr = (c.xc + kVec < nx) ? c.xc + kVec : c.xc + kVec - nx;
    c.need_l = (lane == 0) || (c.xc == 0);
    c.need_r = (lane == 31) || (c.xc + kVec >= nx);
    const int64_t yrow[3] = {wrap(yc - 1, ny), yc, wrap(yc + 1, ny)};  // rows y - 1, y, y + 1

    float f[S][Q][kVec];
    float rho[S][kVec];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const char *base = src + (size_t)s * species_bytes;
        const float *rs = reinterpret_cast<const float *>(base);
        const unsigned short *g = reinterpret_cast<const unsigned short *>(base + (size_t)plane * 4);
        float rw[3][kVec + 2];
#pragma unroll
        for (int d = 0; d < 3; ++d) row6(rs + yrow[d] * pitch, c, rw[d]);
        float gsum[kVec] = {0.f, 0.f, 0.f, 0.f};  // sum_{i>=1} g_i at the site itself
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int ex = L::ex(i), ey = L::ey(i);
            const unsigned short *gi = g + (int64_t)(i - 1) * plane;
            float gp[kVec];
            uint2 raw;
            pull4h<H>(gi + wrap(yc - ey, ny) * pitch, c, ex, gp, raw);
            if (ey != 0) raw = __ldg(reinterpret_cast<const uint2 *>(gi + yc * pitch + c.xc));
            gsum[0] = rn_add(gsum[0], h2f<H>(raw.x));
            gsum[1] = rn_add(gsum[1], h2f<H>(raw.x >> 16));
            gsum[2] = rn_add(gsum[2], h2f<H>(raw.y));
            gsum[3] = rn_add(gsum[3], h2f<H>(raw.y >> 16));
            const float w = weight<Q, float>(i);
#pragma unroll
            for (int j = 0; j < kVec; ++j) f[s][i][j] = rn_fma(w, rw[1 - ey][j + 1 - ex], gp[j]);
        }
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            f[s][0][j] = rn_fma(weight<Q, float>(0), rw[1][j + 1], -gsum[j]);
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

    if (live) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            char *base = dst + (size_t)s * species_bytes;
            float *rs = reinterpret_cast<float *>(base);
            unsigned short *g = reinterpret_cast<unsigned short *>(base + (size_t)plane * 4);
            const float c1 = rn_sub(1.f, (float)a.omega[s]);
            *reinterpret_cast<float4 *>(rs + y * pitch + x0) =
                make_float4(rn_add(rho[s][0], R[s][0]), rn_add(rho[s][1], R[s][1]), rn_add(rho[s][2], R[s][2]),
                            rn_add(rho[s][3], R[s][3]));
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float w = weight<Q, float>(i);
                float hv[kVec];
#pragma unroll
                for (int j = 0; j < kVec; ++j) hv[j] = rn_mul(c1, rn_fma(-w, rho[s][j], f[s][i][j]));
                *reinterpret_cast<uint2 *>(g + (int64_t)(i - 1) * plane + y * pitch + x0) =
                    make_uint2(f2h2<H>(hv[0], hv[1]), f2h2<H>(hv[2], hv[3]));
            }
            if (a.rho_out)
                *reinterpret_cast<float4 *>(static_cast<float *>(a.rho_out) + (int64_t)s * plane + y * pitch + x0) =
                    make_float4(rho[s][0], rho[s][1], rho[s][2], rho[s][3]);
            if (a.mass_out)  // FP32 over the four sites, one FP64 add per tile
                acc[s] += (double)((rho[s][0] + rho[s][1]) + (rho[s][2] + rho[s][3]));
        }
    }
}

template <int Q, int S, int H>
__global__ void __launch_bounds__(kNT) step_half_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
        tile_half<Q, S, H>(a, (tx * kBX + threadIdx.x) * kVec, ty * kBY + threadIdx.y, lane, acc);
    }
    if (a.mass_out) block_mass_reduce<S, kNT>(acc, a.partials, a.counter, a.mass_out);
}

// Launch variants: tile of BX x BY threads (4 sites each), register budget
// from MINB resident blocks per SM.
template <int Q, int S, int H, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX *BY, MINB) step_half_shape(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
        tile_half<Q, S, H>(a, (tx * BX + threadIdx.x) * kVec, ty * BY + threadIdx.y, lane, acc);
    }
    if (a.mass_out) block_mass_reduce<S, BX * BY>(acc, a.partials, a.counter, a.mass_out);
}

}  // namespace half
}  // namespace lbrd
