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
// arithmetic.  The network is copied to shared memory once per block (its
// entries are indexed by the loop counters).
#include "lbrd_kernels.h"

namespace lbrd {

namespace {

constexpr int kBX = 128;

struct SharedNet {
    int nr;
    double rate[kMaxReactions];
    float ratef[kMaxReactions];
    signed char order[kMaxReactions][kMaxSpecies];
    signed char change[kMaxReactions][kMaxSpecies];
};

__device__ __forceinline__ void load_net(const Network &n, SharedNet &sn) {
    if (threadIdx.x == 0) {
        sn.nr = n.nr;
        for (int r = 0; r < kMaxReactions; ++r) {
            sn.rate[r] = n.rate[r];
            sn.ratef[r] = (float)n.rate[r];
            for (int j = 0; j < kMaxSpecies; ++j) {
                sn.order[r][j] = n.order[r][j];
                sn.change[r][j] = n.change[r][j];
            }
        }
    }
    __syncthreads();
}

template <int S>
__device__ __forceinline__ void network_source(const SharedNet &n, int kind, const double (&rho)[S], double (&R)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.0;
    if (kind != kMassAction) return;
    for (int r = 0; r < n.nr; ++r) {
        double p = n.rate[r];
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int e = 0; e < n.order[r][j]; ++e) p = __dmul_rn(p, rho[j]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int c = n.change[r][s];
            if (c != 0) R[s] = __dadd_rn(R[s], __dmul_rn((double)c, p));
        }
    }
}

template <int S>
__device__ __forceinline__ void network_source(const SharedNet &n, int kind, const float (&rho)[S], float (&R)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.f;
    if (kind != kMassAction) return;
    for (int r = 0; r < n.nr; ++r) {
        float p = n.ratef[r];
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int e = 0; e < n.order[r][j]; ++e) p *= rho[j];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int c = n.change[r][s];
            if (c != 0) R[s] += (float)c * p;
        }
    }
}

// Post-collision value of one population.
__device__ __forceinline__ double relax(double f, double w, double rho, double om, double R) {
    return __dadd_rn(__dadd_rn(f, __dmul_rn(__dsub_rn(__dmul_rn(w, rho), f), om)), __dmul_rn(w, R));
}
__device__ __forceinline__ float relax(float f, float w, float rho, float om, float R) {
    return fmaf(1.f - om, f, w * (om * rho + R));
}

__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return a + b; }

template <typename T, int Q, int S>
__global__ void __launch_bounds__(kBX, 6) step_general_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ SharedNet net;
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
        network_source<S>(net, a.rkind, rho, R);
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

template <typename T, int Q, int S>
__global__ void __launch_bounds__(kBX) init_general_kernel(InitArgs a) {
    __shared__ SharedNet net;
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
                                                             : weight<Q, T>(i) * r0;
        T r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = radd(r, f[s][i]);
        rho[s] = r;
    }
    network_source<S>(net, a.rkind, rho, R);
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

cudaError_t launch_step_general(int prec, int Q, int S, const StepArgs &a, cudaStream_t st) {
    return prec == 0 ? dispatch_step<double>(Q, S, a, st) : dispatch_step<float>(Q, S, a, st);
}

cudaError_t launch_init_general(int prec, int Q, int S, const InitArgs &a, cudaStream_t st) {
    return prec == 0 ? dispatch_init<double>(Q, S, a, st) : dispatch_init<float>(Q, S, a, st);
}

}  // namespace lbrd
