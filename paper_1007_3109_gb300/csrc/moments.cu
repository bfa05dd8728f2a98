// Densities on demand: rho_s(x, t) = sum_i f*_i,s(x - e_i, t - 1), the
// moment of Eq. relax's pre-collision distributions, computed from the
// previous state copy (still intact after a step: the ping-pong writes the
// other copy).  The pulls and the index-order sum are the ones the step
// kernels perform, operation for operation, so the result is bitwise the
// rho the step computed.  One thread per site; not on the hot path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lb_rd.h"
#include "lbrd_kernels.h"

namespace lbrd {

namespace {

template <int Q, int S>
__global__ void pull_rho_f64(const double *src, int64_t nx, int64_t ny, int64_t pitch, double *rho) {
    using L = Lattice<Q>;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t plane = ny * pitch;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double f = src[(int64_t)(s * Q + i) * plane + wrap(y - L::ey(i), ny) * pitch + wrap(x - L::ex(i), nx)];
            r = i == 0 ? f : __dadd_rn(r, f);
        }
        rho[(int64_t)s * plane + y * pitch + x] = r;
    }
}

template <int Q, int S>
__global__ void pull_rho_f32(const float *src, int64_t nx, int64_t ny, int64_t pitch, float *rho) {
    using L = Lattice<Q>;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t plane = ny * pitch;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float f = src[(int64_t)(s * Q + i) * plane + wrap(y - L::ey(i), ny) * pitch + wrap(x - L::ex(i), nx)];
            r = i == 0 ? f : rn_add(r, f);
        }
        rho[(int64_t)s * plane + y * pitch + x] = r;
    }
}

template <int H>
__device__ __forceinline__ float h2f(unsigned short bits) {
    if (H == 0) return __uint_as_float((unsigned)bits << 16);
    return __half2float(__ushort_as_half(bits));
}

// Reduced storage: f_i(x) = w_i rho*(x - e_i) + g_i(x - e_i) (i >= 1),
// f_0(x) = w_0 rho*(x) - sum_{i>=1} g_i(x), in the step kernel's operations.
template <int Q, int S, int H>
__global__ void pull_rho_half(const char *src, int64_t nx, int64_t ny, int64_t pitch, float *rho) {
    using L = Lattice<Q>;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t plane = ny * pitch;
    const size_t species_bytes = (size_t)plane * (4 + 2 * (Q - 1));
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const char *base = src + (size_t)s * species_bytes;
        const float *rs = reinterpret_cast<const float *>(base);
        const unsigned short *g = reinterpret_cast<const unsigned short *>(base + (size_t)plane * 4);
        float f[Q];
        float gsum = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int64_t ys = wrap(y - L::ey(i), ny), xs = wrap(x - L::ex(i), nx);
            const float gp = h2f<H>(g[(int64_t)(i - 1) * plane + ys * pitch + xs]);
            gsum = rn_add(gsum, h2f<H>(g[(int64_t)(i - 1) * plane + y * pitch + x]));
            f[i] = rn_fma(weight<Q, float>(i), rs[ys * pitch + xs], gp);
        }
        f[0] = rn_fma(weight<Q, float>(0), rs[y * pitch + x], -gsum);
        float r = f[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = rn_add(r, f[i]);
        rho[(int64_t)s * plane + y * pitch + x] = r;
    }
}

template <int Q, int S>
cudaError_t dispatch(int prec, const void *state, int64_t nx, int64_t ny, int64_t pitch, void *rho, cudaStream_t st) {
    const dim3 g((unsigned)((nx + 127) / 128), (unsigned)ny), b(128);
    switch (prec) {
        case LB_RD_FP64:
            pull_rho_f64<Q, S><<<g, b, 0, st>>>(static_cast<const double *>(state), nx, ny, pitch,
                                                static_cast<double *>(rho));
            break;
        case LB_RD_FP32:
            pull_rho_f32<Q, S><<<g, b, 0, st>>>(static_cast<const float *>(state), nx, ny, pitch,
                                                static_cast<float *>(rho));
            break;
        case LB_RD_FP32_BF16DEV:
            pull_rho_half<Q, S, 0><<<g, b, 0, st>>>(static_cast<const char *>(state), nx, ny, pitch,
                                                    static_cast<float *>(rho));
            break;
        default:
            pull_rho_half<Q, S, 1><<<g, b, 0, st>>>(static_cast<const char *>(state), nx, ny, pitch,
                                                    static_cast<float *>(rho));
            break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pull_rho(int prec, int Q, int S, const void *prev_state, int64_t nx, int64_t ny, int64_t pitch,
                            void *rho, cudaStream_t st) {
    if (Q == 9 && S == 1) return dispatch<9, 1>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 9 && S == 2) return dispatch<9, 2>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 5 && S == 1) return dispatch<5, 1>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 5 && S == 2) return dispatch<5, 2>(prec, prev_state, nx, ny, pitch, rho, st);
    if (prec != LB_RD_FP64 && prec != LB_RD_FP32) return cudaErrorInvalidValue;  // 16-bit storage: S <= 2
    if (Q == 9 && S == 3) return dispatch<9, 3>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 9 && S == 4) return dispatch<9, 4>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 5 && S == 3) return dispatch<5, 3>(prec, prev_state, nx, ny, pitch, rho, st);
    if (Q == 5 && S == 4) return dispatch<5, 4>(prec, prev_state, nx, ny, pitch, rho, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbrd
