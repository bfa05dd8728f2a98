// General step: up to four species (Eq. reac_diff1 is written for N species)
// and mass-action reaction networks, in FP64 or FP32.
//
// One thread per site on a persistent grid over 128 x 1 site tiles: pull
// f_i,s(x, t + 1) = f*_i,s(x - e_i, t) for every species, rho_s = sum_i f_i,s
// (index order), R_s(rho) from the network (or R = 0), then Eq. relax
//   post = f + (w_i rho - f) omega_s + w_i R_s.
// FP64 rounds every operation on its own in that order (bit-reproducible
// against a plain FP64 implementation); the network is evaluated as
//   p = rate_r;  p = p * rho_j  (order[r][j] times, j ascending);
//   R_s = R_s + change[r][s] * p  (steps in order, zero changes skipped).
// FP32 uses post = (1 - omega) f + w (omega rho + R) and plain float
// arithmetic; its launch variants update 1, 2 or 4 consecutive sites per
// thread, or one site in two passes with few registers, all with the same
// per-site arithmetic.  The network is copied to shared
// memory once per block (its entries are indexed by the loop counters).
#include "lbrd_kernels.h"
#include "site_math.cuh"

namespace lbrd {

namespace {

constexpr int kBX = 128;

using namespace sm;

// The general kernel evaluates the network only for mass action (kind 0: R = 0).
template <int S, typename T>
__device__ __forceinline__ void general_source(const NetSmem &n, int kind, const T (&rho)[S], T (&R)[S]) {
    if (kind == kMassAction) {
        network_source<S>(n, rho, R);
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) R[s] = T(0);
    }
}

template <int S, int V>
__device__ __forceinline__ void general_source_vec(const NetSmem &n, int kind, const float (&rho)[S][V],
                                                   float (&R)[S][V]) {
    if (kind == kMassAction) {
        network_source_vec<S, V>(n, rho, R);
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < V; ++v) R[s][v] = 0.f;
    }
}

template <typename T, int Q, int S>
__global__ void __launch_bounds__(kBX, 6) step_general_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ NetSmem net;
    load_net(a.net, net);
    const T *__restrict__ src = static_cast<const T *>(a.src);
    T *__restrict__ dst = static_cast<T *>(a.dst);
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x = (tile - y * tiles_x) * kBX + threadIdx.x;
        if (x >= a.nx) continue;
        T f[S][Q], rho[S], R[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                f[s][i] = src[(int64_t)(s * Q + i) * a.plane + wrap(y - L::ey(i), a.ny) * a.pitch +
                              wrap(x - L::ex(i), a.nx)];
            T r = f[s][0];
#pragma unroll
            for (int i = 1; i < Q; ++i) r = radd(r, f[s][i]);
            rho[s] = r;
        }
        general_source<S>(net, a.rkind, rho, R);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const T om = (T)a.omega[s];
#pragma unroll
            for (int i = 0; i < Q; ++i)
                dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] =
                    relax(f[s][i], weight<Q, T>(i), rho[s], om, R[s]);
            if (a.rho_out) static_cast<T *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
            acc[s] += (double)rho[s];
        }
    }
    if (a.mass_out) block_mass_reduce<S, kBX>(acc, a.partials, a.counter, a.mass_out);
}

// FP32, V = 2 or 4 consecutive sites per thread (nx % V == 0): one aligned
// V-wide load per (species, velocity) from the pulled row; the +-1 column
// shift is a warp shuffle of the neighbouring lane's values, and only the
// lanes at a warp edge or at the periodic edge load one extra float.  The
// per-site arithmetic is the one-site kernel's, so every variant gives the
// same bits.
template <int V>
__device__ __forceinline__ void ldvec(const float *p, float (&v)[V]) {
    if constexpr (V == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = q.x; v[1] = q.y;
    } else {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
}

template <int V>
__device__ __forceinline__ void stvec(float *p, const float (&v)[V]) {
    if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int Q, int S, int V, int MINB>
__global__ void __launch_bounds__(kBX, MINB) step_general_vec_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ NetSmem net;
    load_net(a.net, net);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    const int lane = threadIdx.x & 31;
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x0 = ((tile - y * tiles_x) * kBX + threadIdx.x) * V;
        const bool live = x0 < nx;
        const int64_t xc = live ? x0 : 0;  // dead lanes load valid data for the shuffles
        const int64_t xl = xc == 0 ? nx - 1 : xc - 1;
        const int64_t xr = xc + V < nx ? xc + V : xc + V - nx;
        const bool need_l = lane == 0 || xc == 0;
        const bool need_r = lane == 31 || xc + V >= nx;
        float f[S][Q][V], rho[S][V];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float *row = src + (int64_t)(s * Q + i) * plane + wrap(y - L::ey(i), ny) * pitch;
                float v[V];
                ldvec<V>(row + xc, v);
                if (L::ex(i) == 0) {
#pragma unroll
                    for (int j = 0; j < V; ++j) f[s][i][j] = v[j];
                } else if (L::ex(i) == 1) {  // pull from x - 1
                    float left = __shfl_up_sync(kFullMask, v[V - 1], 1);
                    if (need_l) left = __ldg(row + xl);
                    f[s][i][0] = left;
#pragma unroll
                    for (int j = 1; j < V; ++j) f[s][i][j] = v[j - 1];
                } else {  // pull from x + 1
                    float right = __shfl_down_sync(kFullMask, v[0], 1);
                    if (need_r) right = __ldg(row + xr);
#pragma unroll
                    for (int j = 0; j < V - 1; ++j) f[s][i][j] = v[j + 1];
                    f[s][i][V - 1] = right;
                }
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                float r = f[s][0][j];
#pragma unroll
                for (int i = 1; i < Q; ++i) r = radd(r, f[s][i][j]);
                rho[s][j] = r;
            }
        }
        if (!live) continue;
        float R[S][V];
        general_source_vec<S, V>(net, a.rkind, rho, R);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float om = (float)a.omega[s];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float o[V];
#pragma unroll
                for (int j = 0; j < V; ++j) o[j] = relax(f[s][i][j], weight<Q, float>(i), rho[s][j], om, R[s][j]);
                stvec<V>(dst + (int64_t)(s * Q + i) * plane + y * pitch + x0, o);
            }
            if (a.rho_out) stvec<V>(static_cast<float *>(a.rho_out) + (int64_t)s * plane + y * pitch + x0, rho[s]);
            float part = 0.f;
#pragma unroll
            for (int j = 0; j < V; ++j) part += rho[s][j];
            acc[s] += (double)part;
        }
    }
    if (a.mass_out) block_mass_reduce<S, kBX>(acc, a.partials, a.counter, a.mass_out);
}

// FP32, one site per thread in two passes to keep few registers live: pass 1
// loads the pulled f of every species only to sum rho, then the source is
// evaluated, and pass 2 loads the same values again (L1 hits: the block's
// rows were just read) for the collision.  Many more resident warps hide the
// HBM latency; the arithmetic and its order are the one-site kernel's.
template <int Q, int S, int MINB>
__global__ void __launch_bounds__(kBX, MINB) step_general_2pass_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ NetSmem net;
    load_net(a.net, net);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x = (tile - y * tiles_x) * kBX + threadIdx.x;
        if (x >= nx) continue;
        // pulled rows y + 1, y, y - 1 and columns x + 1, x, x - 1 (periodic)
        const int64_t rows[3] = {wrap(y + 1, ny) * pitch, y * pitch, wrap(y - 1, ny) * pitch};
        const int64_t cols[3] = {wrap(x + 1, nx), x, wrap(x - 1, nx)};
        auto off = [&](int i) { return (int64_t)i * plane + rows[1 + L::ey(i)] + cols[1 + L::ex(i)]; };
        float rho[S], R[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float *sp = src + (int64_t)s * Q * plane;
            float r = __ldg(sp + off(0));
#pragma unroll
            for (int i = 1; i < Q; ++i) r = radd(r, __ldg(sp + off(i)));
            rho[s] = r;
        }
        general_source<S>(net, a.rkind, rho, R);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float *sp = src + (int64_t)s * Q * plane;
            const float om = (float)a.omega[s];
#pragma unroll
            for (int i = 0; i < Q; ++i)
                dst[(int64_t)(s * Q + i) * plane + y * pitch + x] =
                    relax(__ldg(sp + off(i)), weight<Q, float>(i), rho[s], om, R[s]);
            if (a.rho_out) static_cast<float *>(a.rho_out)[(int64_t)s * plane + y * pitch + x] = rho[s];
            acc[s] += (double)rho[s];
        }
    }
    if (a.mass_out) block_mass_reduce<S, kBX>(acc, a.partials, a.counter, a.mass_out);
}

template <typename T, int Q, int S>
__global__ void __launch_bounds__(kBX) init_general_kernel(InitArgs a) {
    __shared__ NetSmem net;
    load_net(a.net, net);
    const int64_t x = (int64_t)blockIdx.x * kBX + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    T *__restrict__ dst = static_cast<T *>(a.dst);
    T f[S][Q], rho[S], R[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const T r0 = (T)a.rho0[((int64_t)s * a.ny + y) * a.nx + x];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = sizeof(T) == 8 ? (T)__dmul_rn(weight<Q, double>(i), (double)r0)
                                                             : (T)rn_mul(weight<Q, float>(i), (float)r0);
        T r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = radd(r, f[s][i]);
        rho[s] = r;
    }
    general_source<S>(net, a.rkind, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const T om = (T)a.omega[s];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] = relax(f[s][i], weight<Q, T>(i), rho[s], om, R[s]);
        if (a.rho_out) static_cast<T *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
    }
}

template <typename T, int Q, int S>
cudaError_t launch_general(const StepArgs &a, cudaStream_t st) {
    const int64_t tiles_x = (a.nx + kBX - 1) / kBX, ntiles = tiles_x * a.ny;
    auto kern = step_general_kernel<T, Q, S>;
    const unsigned grid = persistent_blocks(kern, kBX, ntiles);
    kern<<<grid, kBX, 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int Q, int S, int V, int MINB>
cudaError_t launch_general_vec(const StepArgs &a, cudaStream_t st) {
    if (a.nx % V) return cudaErrorInvalidValue;
    const int64_t tiles_x = (a.nx / V + kBX - 1) / kBX, ntiles = tiles_x * a.ny;
    auto kern = step_general_vec_kernel<Q, S, V, MINB>;
    const unsigned grid = persistent_blocks(kern, kBX, ntiles);
    kern<<<grid, kBX, 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int Q, int S, int MINB>
cudaError_t launch_general_2pass(const StepArgs &a, cudaStream_t st) {
    const int64_t tiles_x = (a.nx + kBX - 1) / kBX, ntiles = tiles_x * a.ny;
    auto kern = step_general_2pass_kernel<Q, S, MINB>;
    const unsigned grid = persistent_blocks(kern, kBX, ntiles);
    kern<<<grid, kBX, 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int MINB>
cudaError_t dispatch_2pass(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_general_2pass<9, 1, MINB>(a, st);
            case 2: return launch_general_2pass<9, 2, MINB>(a, st);
            case 3: return launch_general_2pass<9, 3, MINB>(a, st);
            case 4: return launch_general_2pass<9, 4, MINB>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_general_2pass<5, 1, MINB>(a, st);
            case 2: return launch_general_2pass<5, 2, MINB>(a, st);
            case 3: return launch_general_2pass<5, 3, MINB>(a, st);
            case 4: return launch_general_2pass<5, 4, MINB>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <int V, int MINB>
cudaError_t dispatch_vec(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_general_vec<9, 1, V, MINB>(a, st);
            case 2: return launch_general_vec<9, 2, V, MINB>(a, st);
            case 3: return launch_general_vec<9, 3, V, MINB>(a, st);
            case 4: return launch_general_vec<9, 4, V, MINB>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_general_vec<5, 1, V, MINB>(a, st);
            case 2: return launch_general_vec<5, 2, V, MINB>(a, st);
            case 3: return launch_general_vec<5, 3, V, MINB>(a, st);
            case 4: return launch_general_vec<5, 4, V, MINB>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T, int Q, int S>
cudaError_t launch_general_init(const InitArgs &a, cudaStream_t st) {
    const dim3 g((unsigned)((a.nx + kBX - 1) / kBX), (unsigned)a.ny);
    init_general_kernel<T, Q, S><<<g, kBX, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_step(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_general<T, 9, 1>(a, st);
            case 2: return launch_general<T, 9, 2>(a, st);
            case 3: return launch_general<T, 9, 3>(a, st);
            case 4: return launch_general<T, 9, 4>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_general<T, 5, 1>(a, st);
            case 2: return launch_general<T, 5, 2>(a, st);
            case 3: return launch_general<T, 5, 3>(a, st);
            case 4: return launch_general<T, 5, 4>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_init(int Q, int S, const InitArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_general_init<T, 9, 1>(a, st);
            case 2: return launch_general_init<T, 9, 2>(a, st);
            case 3: return launch_general_init<T, 9, 3>(a, st);
            case 4: return launch_general_init<T, 9, 4>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_general_init<T, 5, 1>(a, st);
            case 2: return launch_general_init<T, 5, 2>(a, st);
            case 3: return launch_general_init<T, 5, 3>(a, st);
            case 4: return launch_general_init<T, 5, 4>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

const GeneralVariant kGeneralVariants[] = {
    {"general_1site", 1}, {"general_2site", 2}, {"general_4site", 4}, {"general_2site_minb3", 2},
    {"general_2pass_minb8", 1}, {"general_2pass_minb10", 1},
};
const int kGeneralVariantCount = sizeof(kGeneralVariants) / sizeof(kGeneralVariants[0]);

cudaError_t launch_step_general(int prec, int Q, int S, const StepArgs &a, cudaStream_t st, int variant) {
    if (prec == 0) return variant == 0 ? dispatch_step<double>(Q, S, a, st) : cudaErrorInvalidValue;
    switch (variant) {
        case 0: return dispatch_step<float>(Q, S, a, st);
        case 1: return dispatch_vec<2, 4>(Q, S, a, st);
        case 2: return dispatch_vec<4, 2>(Q, S, a, st);
        case 3: return dispatch_vec<2, 3>(Q, S, a, st);
        case 4: return dispatch_2pass<8>(Q, S, a, st);
        case 5: return dispatch_2pass<10>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_general(int prec, int Q, int S, const InitArgs &a, cudaStream_t st) {
    return prec == 0 ? dispatch_init<double>(Q, S, a, st) : dispatch_init<float>(Q, S, a, st);
}

}  // namespace lbrd
