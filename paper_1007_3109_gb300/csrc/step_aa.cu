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
// both layouts give the same bits.  Persistent grid; one site per thread, or
// (FP32 launch variants) 2 or 4 consecutive sites per thread.
#include "step_aa_kernel.cuh"

namespace lbrd {

namespace {

using namespace aa;

constexpr int kBX = 128;

template <typename T, int Q, int S, int PHASE>
__global__ void __launch_bounds__(kBX) step_aa_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    __shared__ AANet net;
    load_net(a.net, net);
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x = (tile - y * tiles_x) * kBX + threadIdx.x;
        if (x < a.nx) site_aa<T, Q, S, PHASE>(a, net, x, y, acc);
    }
    if (a.mass_out) block_mass_reduce<S, kBX>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S, int V, int PHASE, int MINB>
__global__ void __launch_bounds__(kBX, MINB) step_aa_vec_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    __shared__ AANet net;
    load_net(a.net, net);
    const int lane = threadIdx.x & 31;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x0 = ((tile - y * tiles_x) * kBX + threadIdx.x) * V;
        tile_aa<Q, S, V, PHASE>(a, net, x0, y, lane, acc);
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

template <int Q, int S, int V, int PHASE, int MINB>
cudaError_t launch_aa_vec(const StepArgs &a, cudaStream_t st) {
    if (a.nx % V) return cudaErrorInvalidValue;
    const int64_t tiles_x = (a.nx / V + kBX - 1) / kBX, ntiles = tiles_x * a.ny;
    auto kern = step_aa_vec_kernel<Q, S, V, PHASE, MINB>;
    const unsigned grid = persistent_blocks(kern, kBX, ntiles);
    kern<<<grid, kBX, 0, st>>>(a, tiles_x, ntiles);
    return cudaGetLastError();
}

template <int V, int PHASE, int MINB>
cudaError_t dispatch_aa_vec(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9) {
        switch (S) {
            case 1: return launch_aa_vec<9, 1, V, PHASE, MINB>(a, st);
            case 2: return launch_aa_vec<9, 2, V, PHASE, MINB>(a, st);
            case 3: return launch_aa_vec<9, 3, V, PHASE, MINB>(a, st);
            case 4: return launch_aa_vec<9, 4, V, PHASE, MINB>(a, st);
        }
    } else if (Q == 5) {
        switch (S) {
            case 1: return launch_aa_vec<5, 1, V, PHASE, MINB>(a, st);
            case 2: return launch_aa_vec<5, 2, V, PHASE, MINB>(a, st);
            case 3: return launch_aa_vec<5, 3, V, PHASE, MINB>(a, st);
            case 4: return launch_aa_vec<5, 4, V, PHASE, MINB>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <int V, int MINB>
cudaError_t aa_vec(int Q, int S, int phase, const StepArgs &a, cudaStream_t st) {
    return phase ? dispatch_aa_vec<V, 1, MINB>(Q, S, a, st) : dispatch_aa_vec<V, 0, MINB>(Q, S, a, st);
}

}  // namespace

const GeneralVariant kAAVariants[] = {{"aa_1site", 1}, {"aa_2site", 2}, {"aa_4site", 4}, {"aa_4site_minb3", 4}};
const int kAAVariantCount = sizeof(kAAVariants) / sizeof(kAAVariants[0]);

cudaError_t launch_step_aa(int prec, int Q, int S, int phase, const StepArgs &a, cudaStream_t st, int variant) {
    if (a.src != a.dst) return cudaErrorInvalidValue;
    if (prec == 0) {
        if (variant != 0) return cudaErrorInvalidValue;
        return phase ? dispatch_aa<double, 1>(Q, S, a, st) : dispatch_aa<double, 0>(Q, S, a, st);
    }
    switch (variant) {
        case 0: return phase ? dispatch_aa<float, 1>(Q, S, a, st) : dispatch_aa<float, 0>(Q, S, a, st);
        case 1: return aa_vec<2, 4>(Q, S, phase, a, st);
        case 2: return aa_vec<4, 2>(Q, S, phase, a, st);
        case 3: return aa_vec<4, 3>(Q, S, phase, a, st);
        default: return cudaErrorInvalidValue;
    }
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
