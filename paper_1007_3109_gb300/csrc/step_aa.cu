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

// V sites at once: kinds other than mass action per site as above; the
// network with each step's constants read once for all V sites (per site
// the same operations in the same order).
template <int S, int V>
__device__ __forceinline__ void source_vec(const StepArgs &a, const AANet &n, const float (&rho)[S][V],
                                           float (&R)[S][V]) {
    if (a.rkind != kMassAction) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float rv[S], Rv[S];
#pragma unroll
            for (int s = 0; s < S; ++s) rv[s] = rho[s][v];
            source<S>(a, n, rv, Rv);
#pragma unroll
            for (int s = 0; s < S; ++s) R[s][v] = Rv[s];
        }
        return;
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int v = 0; v < V; ++v) R[s][v] = 0.f;
    for (int r = 0; r < n.nr; ++r) {
        float p[V];
        const float k = (float)n.rate[r];
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = k;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int o = n.order[r][j];
            for (int e = 0; e < o; ++e)
#pragma unroll
                for (int v = 0; v < V; ++v) p[v] *= rho[j][v];
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int c = n.change[r][s];
            if (c != 0) {
                const float cf = (float)c;
#pragma unroll
                for (int v = 0; v < V; ++v) R[s][v] += cf * p[v];
            }
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

// FP32, V = 2 or 4 consecutive sites per thread (nx % V == 0), plain
// coherent loads (never the read-only path: the kernel writes what it reads).
// Phase A loads the aligned V-vector of each pulled row and takes the +-1
// column from the neighbouring lane (edge lanes load it); its stores go to
// the pushed columns x + e_x, assembled into aligned vectors with a shuffle:
// for e_x = +1 a lane stores [left lane's site V-1, own sites 0 .. V-2], for
// e_x = -1 [own sites 1 .. V-1, right lane's site 0].  A lane at a warp or
// periodic edge cannot take the neighbour's value: it stores its own
// in-range values one by one, and the value that would cross the edge is
// stored, also as a scalar, by the lane that computed it.  Every slot is
// written once, by its own site's thread or by a lane of the same warp after
// a shuffle that follows that site's loads.  Phase B is site-local: aligned
// vector loads from slot opp(i), aligned vector stores to slot i.
template <int V>
__device__ __forceinline__ void ldv(const float *p, float (&v)[V]) {
    if constexpr (V == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
}

template <int V>
__device__ __forceinline__ void stv(float *p, const float (&v)[V]) {
    if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int Q, int S, int V, int PHASE, int MINB>
__global__ void __launch_bounds__(kBX, MINB) step_aa_vec_kernel(StepArgs a, int64_t tiles_x, int64_t ntiles) {
    using L = Lattice<Q>;
    __shared__ AANet net;
    load_aanet(a.net, net);
    float *st = static_cast<float *>(a.dst);  // == a.src
    const int lane = threadIdx.x & 31;
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_x, x0 = ((tile - y * tiles_x) * kBX + threadIdx.x) * V;
        const bool live = x0 < nx;
        const int64_t xc = live ? x0 : 0;
        const bool edge_l = lane == 0 || xc == 0;       // the left neighbour is not in this warp
        const bool edge_r = lane == 31 || xc + V >= nx; // the right neighbour is not in this warp
        const int64_t xl = xc == 0 ? nx - 1 : xc - 1;
        const int64_t xr = xc + V < nx ? xc + V : xc + V - nx;
        float f[S][Q][V], rho[S][V];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (PHASE == 1) {
                    float v[V];
                    ldv<V>(st + (int64_t)(s * Q + opp<Q>(i)) * plane + y * pitch + xc, v);
#pragma unroll
                    for (int j = 0; j < V; ++j) f[s][i][j] = v[j];
                } else {
                    const float *row = st + (int64_t)(s * Q + i) * plane + wrap(y - L::ey(i), ny) * pitch;
                    float v[V];
                    ldv<V>(row + xc, v);
                    if (L::ex(i) == 0) {
#pragma unroll
                        for (int j = 0; j < V; ++j) f[s][i][j] = v[j];
                    } else if (L::ex(i) == 1) {
                        float left = __shfl_up_sync(kFullMask, v[V - 1], 1);
                        if (edge_l) left = row[xl];
                        f[s][i][0] = left;
#pragma unroll
                        for (int j = 1; j < V; ++j) f[s][i][j] = v[j - 1];
                    } else {
                        float right = __shfl_down_sync(kFullMask, v[0], 1);
                        if (edge_r) right = row[xr];
#pragma unroll
                        for (int j = 0; j < V - 1; ++j) f[s][i][j] = v[j + 1];
                        f[s][i][V - 1] = right;
                    }
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
        float R[S][V];
        source_vec<S, V>(a, net, rho, R);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float om = (float)a.omega[s];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float o[V];
#pragma unroll
                for (int j = 0; j < V; ++j) o[j] = relax(f[s][i][j], weight<Q, float>(i), rho[s][j], om, R[s][j]);
                if constexpr (PHASE == 1) {
                    if (live) stv<V>(st + (int64_t)(s * Q + i) * plane + y * pitch + x0, o);
                } else {
                    float *row = st + (int64_t)(s * Q + opp<Q>(i)) * plane + wrap(y + L::ey(i), ny) * pitch;
                    if (L::ex(i) == 0) {
                        if (live) stv<V>(row + x0, o);
                    } else if (L::ex(i) == 1) {  // site j goes to column x0 + j + 1
                        const float from_left = __shfl_up_sync(kFullMask, o[V - 1], 1);
                        if (live) {
                            if (edge_l) {
#pragma unroll
                                for (int j = 0; j < V - 1; ++j) row[x0 + j + 1] = o[j];
                            } else {
                                float w[V];
                                w[0] = from_left;
#pragma unroll
                                for (int j = 1; j < V; ++j) w[j] = o[j - 1];
                                stv<V>(row + x0, w);
                            }
                            if (edge_r) row[xr] = o[V - 1];
                        }
                    } else {  // site j goes to column x0 + j - 1
                        const float from_right = __shfl_down_sync(kFullMask, o[0], 1);
                        if (live) {
                            if (edge_r) {
#pragma unroll
                                for (int j = 1; j < V; ++j) row[x0 + j - 1] = o[j];
                            } else {
                                float w[V];
#pragma unroll
                                for (int j = 0; j < V - 1; ++j) w[j] = o[j + 1];
                                w[V - 1] = from_right;
                                stv<V>(row + x0, w);
                            }
                            if (edge_l) row[xl] = o[0];
                        }
                    }
                }
            }
            if (live) {
                if (a.rho_out) stv<V>(static_cast<float *>(a.rho_out) + (int64_t)s * plane + y * pitch + x0, rho[s]);
                float part = 0.f;
#pragma unroll
                for (int j = 0; j < V; ++j) part += rho[s][j];
                acc[s] += (double)part;
            }
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
