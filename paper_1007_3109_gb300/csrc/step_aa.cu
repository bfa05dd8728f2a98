// In-place streaming (the AA pattern): one copy of the state instead of two.
//
// The ping-pong path stores f*(t) "natural" (slot i of site x holds
// f*_i(x, t)) and pulls it into a second copy.  Here two kinds of step
// alternate on one copy:
//   phase A (t even, natural in): site x reads slot i of x - e_i, which is
//     the pre-collision f_i(x, t + 1), collides, and writes f*_i(x, t + 1)
//     to slot opp(i) of x + e_i ("pushed and swapped");
//   phase B (t odd, pushed-and-swapped in): the pre-collision f_i(z, t + 1)
//     = f*_i(z - e_i, t) sits in slot opp(i) of z itself; site z collides
//     and writes f*_i(z, t + 1) to slot i of z (natural again).
// In phase A the slots site x writes, (x + e_i, opp(i)), are exactly the
// slots it read, (x - e_j, j) with j = opp(i), and no other site reads them;
// phase B touches only the site's own slots.  So every thread reads all its
// values before writing and no two threads share a slot: the update is
// race-free in place (the pointers are not restrict-qualified: source and
// destination are the same buffer).
//
// The per-site arithmetic is the ping-pong kernels' (FP64: every operation
// rounded on its own in the order of Eq. relax; FP32: the register path's
// post = (1 - omega) f + w (omega rho + R) with the same reaction code), so
// both layouts give the same bits.  One thread per site, persistent grid.
#include "lbrd_kernels.h"

namespace lbrd {

namespace {

constexpr int kBX = 128;

template <int Q>
__host__ __device__ constexpr int opp(int i) {
    for (int j = 0; j < Q; ++j)
        if (Lattice<Q>::ex(j) == -Lattice<Q>::ex(i) && Lattice<Q>::ey(j) == -Lattice<Q>::ey(i)) return j;
    return i;
}

struct AANet {
    int nr;
    double rate[kMaxReactions];
    signed char order[kMaxReactions][kMaxSpecies];
    signed char change[kMaxReactions][kMaxSpecies];
};

__device__ __forceinline__ void load_aanet(const Network &n, AANet &sn) {
    if (threadIdx.x == 0) {
        sn.nr = n.nr;
        for (int r = 0; r < kMaxReactions; ++r) {
            sn.rate[r] = n.rate[r];
            for (int j = 0; j < kMaxSpecies; ++j) {
                sn.order[r][j] = n.order[r][j];
                sn.change[r][j] = n.change[r][j];
            }
        }
    }
    __syncthreads();
}

// Reaction source with the arithmetic of the ping-pong kernels: the
// Gray-Scott and transformation sources of lbrd_common.cuh, or the network
// evaluated as in the general kernel.
template <int S>
__device__ __forceinline__ void source(const StepArgs &a, const AANet &n, const double (&rho)[S], double (&R)[S]) {
    if (a.rkind != kMassAction) {
        if constexpr (S <= 2) reaction_f64<S>(a.rkind, a.kappa, a.F, a.k, rho, R);
        else {
#pragma unroll
            for (int s = 0; s < S; ++s) R[s] = 0.0;
        }
        return;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.0;
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
__device__ __forceinline__ void source(const StepArgs &a, const AANet &n, const float (&rho)[S], float (&R)[S]) {
    if (a.rkind != kMassAction) {
        if constexpr (S <= 2) reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
        else {
#pragma unroll
            for (int s = 0; s < S; ++s) R[s] = 0.f;
        }
        return;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.f;
    for (int r = 0; r < n.nr; ++r) {
        float p = (float)n.rate[r];
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

__device__ __forceinline__ double relax(double f, double w, double rho, double om, double R) {
    return __dadd_rn(__dadd_rn(f, __dmul_rn(__dsub_rn(__dmul_rn(w, rho), f), om)), __dmul_rn(w, R));
}
__device__ __forceinline__ float relax(float f, float w, float rho, float om, float R) {
    return fmaf(1.f - om, f, w * (om * rho + R));
}
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return a + b; }

template <typename T, int Q, int S, int PHASE>
__global__ void __launch_bounds__(kBX) step_aa_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ AANet net;
    load_aanet(a.net, net);
    T *st = static_cast<T *>(a.dst);  // == a.src
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x = (tile - y * tiles_x) * kBX + threadIdx.x;
        if (x >= nx) continue;
        T f[S][Q], rho[S], R[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (PHASE == 0)
                    f[s][i] = st[(int64_t)(s * Q + i) * plane + wrap(y - L::ey(i), ny) * pitch + wrap(x - L::ex(i), nx)];
                else
                    f[s][i] = st[(int64_t)(s * Q + opp<Q>(i)) * plane + y * pitch + x];
            }
            T r = f[s][0];
#pragma unroll
            for (int i = 1; i < Q; ++i) r = radd(r, f[s][i]);
            rho[s] = r;
        }
        source<S>(a, net, rho, R);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const T om = (T)a.omega[s];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T post = relax(f[s][i], weight<Q, T>(i), rho[s], om, R[s]);
                if constexpr (PHASE == 0)
                    st[(int64_t)(s * Q + opp<Q>(i)) * plane + wrap(y + L::ey(i), ny) * pitch + wrap(x + L::ex(i), nx)] =
                        post;
                else
                    st[(int64_t)(s * Q + i) * plane + y * pitch + x] = post;
            }
            if (a.rho_out) static_cast<T *>(a.rho_out)[(int64_t)s * plane + y * pitch + x] = rho[s];
            acc[s] += (double)rho[s];
        }
    }
    if (a.mass_out) block_mass_reduce<S, kBX>(acc, a.partials, a.counter, a.mass_out);
}

// f*(t) of a pushed-and-swapped state (t odd) as packed FP64 [s][i][y][x]:
// f*_i(x) sits in slot opp(i) of x + e_i.
template <typename T, int Q>
__global__ void export_swapped_kernel(const T *st, int64_t nx, int64_t ny, int64_t pitch, int S, double *out) {
    using L = Lattice<Q>;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int si = blockIdx.z, s = si / Q, i = si - s * Q;
    if (x >= nx) return;
    int ex = 0, ey = 0, o = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (k == i) {
            ex = L::ex(k);
            ey = L::ey(k);
            o = opp<Q>(k);
        }
    const int64_t plane = ny * pitch;
    out[((int64_t)si * ny + y) * nx + x] = (double)st[(int64_t)(s * Q + o) * plane + wrap(y + ey, ny) * pitch + wrap(x + ex, nx)];
}

template <typename T, int Q, int S, int PHASE>
cudaError_t launch_aa(const StepArgs &a, cudaStream_t st) {
    const int64_t tiles_x = (a.nx + kBX - 1) / kBX, ntiles = tiles_x * a.ny;
    auto kern = step_aa_kernel<T, Q, S, PHASE>;
    const unsigned grid = persistent_blocks(kern, kBX, ntiles);
    kern<<<grid, kBX, 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <typename T, int PHASE>
cudaError_t dispatch_aa(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_aa<T, 9, 1, PHASE>(a, st);
            case 2: return launch_aa<T, 9, 2, PHASE>(a, st);
            case 3: return launch_aa<T, 9, 3, PHASE>(a, st);
            case 4: return launch_aa<T, 9, 4, PHASE>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_aa<T, 5, 1, PHASE>(a, st);
            case 2: return launch_aa<T, 5, 2, PHASE>(a, st);
            case 3: return launch_aa<T, 5, 3, PHASE>(a, st);
            case 4: return launch_aa<T, 5, 4, PHASE>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step_aa(int prec, int Q, int S, int phase, const StepArgs &a, cudaStream_t st) {
    if (a.src != a.dst) return cudaErrorInvalidValue;
    if (prec == 0) return phase ? dispatch_aa<double, 1>(Q, S, a, st) : dispatch_aa<double, 0>(Q, S, a, st);
    return phase ? dispatch_aa<float, 1>(Q, S, a, st) : dispatch_aa<float, 0>(Q, S, a, st);
}

cudaError_t launch_export_swapped(int prec, int Q, int S, const void *state, int64_t nx, int64_t ny, int64_t pitch,
                                  double *out, cudaStream_t st) {
    const dim3 g((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)(Q * S)), b(256);
    if (prec == 0) {
        if (Q == 9) export_swapped_kernel<double, 9><<<g, b, 0, st>>>(static_cast<const double *>(state), nx, ny, pitch, S, out);
        else export_swapped_kernel<double, 5><<<g, b, 0, st>>>(static_cast<const double *>(state), nx, ny, pitch, S, out);
    } else {
        if (Q == 9) export_swapped_kernel<float, 9><<<g, b, 0, st>>>(static_cast<const float *>(state), nx, ny, pitch, S, out);
        else export_swapped_kernel<float, 5><<<g, b, 0, st>>>(static_cast<const float *>(state), nx, ny, pitch, S, out);
    }
    return cudaGetLastError();
}

}  // namespace lbrd
