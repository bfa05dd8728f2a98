// Read-out kernels: distributions and densities to packed FP64, and the FP64
// global sum of the densities (sum_x rho_s, the mass diagnostic; conserved
// when R = 0 because sum_i f_eq = rho and sum_i w_i = 1, Eq. equili).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbrd_kernels.h"
#include "lb_rd.h"

namespace lbrd {

namespace {

template <typename T>
__device__ __forceinline__ double load_as_double(const void *p, int64_t idx) {
    return (double)static_cast<const T *>(p)[idx];
}

// Full-precision state: plane p = s * Q + i, value at [p][y][pitch].
template <typename T>
__global__ void export_plain_kernel(const T *state, int64_t nx, int64_t ny, int64_t pitch, int planes,
                                    double *out) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    const int p = blockIdx.z;
    if (x >= nx) return;
    out[((int64_t)p * ny + y) * nx + x] = (double)state[((int64_t)p * ny + y) * pitch + x];
}

// Reduced state, per species: plane 0 = rho* (float), planes 1..Q-1 the
// 16-bit deviations g_i; f*_i = w_i rho* + g_i, g_0 = -sum_{i>=1} g_i.
template <int Q, typename H>
__global__ void export_half_kernel(const char *state, int64_t nx, int64_t ny, int64_t pitch, int S, double *out) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    const int s = blockIdx.z;
    if (x >= nx) return;
    const int64_t plane = ny * pitch;
    const size_t species_bytes = (size_t)plane * (4 + 2 * (Q - 1));
    const char *base = state + (size_t)s * species_bytes;
    const float rs = reinterpret_cast<const float *>(base)[y * pitch + x];
    const H *g = reinterpret_cast<const H *>(base + (size_t)plane * 4);
    float gs[Q];
    float sum = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        gs[i] = (float)g[(int64_t)(i - 1) * plane + y * pitch + x];
        sum = rn_add(sum, gs[i]);
    }
    gs[0] = -sum;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        out[(((int64_t)s * Q + i) * ny + y) * nx + x] = (double)rn_fma(weight<Q, float>(i), rs, gs[i]);
}

template <typename T>
__global__ void rho_export_kernel(const T *rho, int64_t nx, int64_t ny, int64_t pitch, double *out) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    const int s = blockIdx.z;
    if (x >= nx) return;
    out[((int64_t)s * ny + y) * nx + x] = (double)rho[((int64_t)s * ny + y) * pitch + x];
}

constexpr int kMassNT = 256;
constexpr int kMassRows = 8;

template <typename T, int S>
__global__ void __launch_bounds__(kMassNT) mass_kernel(const T *rho, int64_t nx, int64_t ny, int64_t pitch,
                                                       double *partials, unsigned int *counter, double *mass) {
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    const int64_t x = (int64_t)blockIdx.x * kMassNT + threadIdx.x;
    const int64_t y0 = (int64_t)blockIdx.y * kMassRows;
    if (x < nx) {
        for (int64_t y = y0; y < y0 + kMassRows && y < ny; ++y) {
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] += (double)rho[((int64_t)s * ny + y) * pitch + x];
        }
    }
    block_mass_reduce<S, kMassNT>(acc, partials, counter, mass);
}

dim3 mass_grid(int64_t nx, int64_t ny) {
    return dim3((unsigned)((nx + kMassNT - 1) / kMassNT), (unsigned)((ny + kMassRows - 1) / kMassRows));
}

}  // namespace

size_t state_plane_bytes(int prec, int Q, int S, int64_t ny, int64_t pitch) {
    const size_t plane = (size_t)ny * (size_t)pitch;
    switch (prec) {
        case LB_RD_FP64: return plane * 8 * Q * S;
        case LB_RD_FP32: return plane * 4 * Q * S;
        default: return plane * (4 + 2 * (Q - 1)) * S;
    }
}

cudaError_t launch_export(int prec, int Q, int S, const void *state, int64_t nx, int64_t ny, int64_t pitch,
                          double *out, cudaStream_t st) {
    const dim3 b(256);
    if (prec == LB_RD_FP64 || prec == LB_RD_FP32) {
        const dim3 g((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)(Q * S));
        if (prec == LB_RD_FP64)
            export_plain_kernel<double><<<g, b, 0, st>>>(static_cast<const double *>(state), nx, ny, pitch, Q * S, out);
        else
            export_plain_kernel<float><<<g, b, 0, st>>>(static_cast<const float *>(state), nx, ny, pitch, Q * S, out);
        return cudaGetLastError();
    }
    const dim3 g((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)S);
    const char *p = static_cast<const char *>(state);
    if (prec == LB_RD_FP32_BF16DEV) {
        if (Q == 9) export_half_kernel<9, __nv_bfloat16><<<g, b, 0, st>>>(p, nx, ny, pitch, S, out);
        else export_half_kernel<5, __nv_bfloat16><<<g, b, 0, st>>>(p, nx, ny, pitch, S, out);
    } else {
        if (Q == 9) export_half_kernel<9, __half><<<g, b, 0, st>>>(p, nx, ny, pitch, S, out);
        else export_half_kernel<5, __half><<<g, b, 0, st>>>(p, nx, ny, pitch, S, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_export(int prec, int S, const void *rho, int64_t nx, int64_t ny, int64_t pitch, double *out,
                              cudaStream_t st) {
    const dim3 g((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)S), b(256);
    if (prec == LB_RD_FP64) rho_export_kernel<double><<<g, b, 0, st>>>(static_cast<const double *>(rho), nx, ny, pitch, out);
    else rho_export_kernel<float><<<g, b, 0, st>>>(static_cast<const float *>(rho), nx, ny, pitch, out);
    return cudaGetLastError();
}

size_t mass_partials_needed(int64_t nx, int64_t ny) {
    const dim3 g = mass_grid(nx, ny);
    return (size_t)g.x * g.y;
}

template <typename T>
static cudaError_t mass_dispatch(int S, const T *r, dim3 g, dim3 b, int64_t nx, int64_t ny, int64_t pitch,
                                 double *partials, unsigned int *counter, double *mass, cudaStream_t st) {
    switch (S) {
        case 1: mass_kernel<T, 1><<<g, b, 0, st>>>(r, nx, ny, pitch, partials, counter, mass); break;
        case 2: mass_kernel<T, 2><<<g, b, 0, st>>>(r, nx, ny, pitch, partials, counter, mass); break;
        case 3: mass_kernel<T, 3><<<g, b, 0, st>>>(r, nx, ny, pitch, partials, counter, mass); break;
        case 4: mass_kernel<T, 4><<<g, b, 0, st>>>(r, nx, ny, pitch, partials, counter, mass); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mass(int prec, int S, const void *rho, int64_t nx, int64_t ny, int64_t pitch, double *partials,
                        unsigned int *counter, double *mass, cudaStream_t st) {
    const dim3 g = mass_grid(nx, ny), b(kMassNT);
    if (prec == LB_RD_FP64) return mass_dispatch<double>(S, static_cast<const double *>(rho), g, b, nx, ny, pitch,
                                                         partials, counter, mass, st);
    return mass_dispatch<float>(S, static_cast<const float *>(rho), g, b, nx, ny, pitch, partials, counter, mass, st);
}

}  // namespace lbrd
