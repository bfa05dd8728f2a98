// In-place (AA) step bodies shared by the single-simulation kernels
// (step_aa.cu) and the batched kernel (batch.cu).  The pattern, the phases
// and why the update is race-free in place are described in step_aa.cu.
#pragma once

#include "lbrd_kernels.h"
#include "site_math.cuh"

namespace lbrd {
namespace aa {

template <int Q>
__host__ __device__ constexpr int opp(int i) {
    for (int j = 0; j < Q; ++j)
        if (Lattice<Q>::ex(j) == -Lattice<Q>::ex(i) && Lattice<Q>::ey(j) == -Lattice<Q>::ey(i)) return j;
    return i;
}

using AANet = sm::NetSmem;
using sm::load_net;
using sm::radd;
using sm::relax;

// Reaction source with the arithmetic of the ping-pong kernels: the
// Gray-Scott and transformation sources of lbrd_common.cuh, or the network.
template <int S>
__device__ __forceinline__ void source(const StepArgs &a, const AANet &n, const double (&rho)[S], double (&R)[S]) {
    if (a.rkind == kMassAction) {
        sm::network_source<S>(n, rho, R);
    } else if constexpr (S <= 2) {
        reaction_f64<S>(a.rkind, a.kappa, a.F, a.k, rho, R);
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) R[s] = 0.0;
    }
}

template <int S>
__device__ __forceinline__ void source(const StepArgs &a, const AANet &n, const float (&rho)[S], float (&R)[S]) {
    if (a.rkind == kMassAction) {
        sm::network_source<S>(n, rho, R);
    } else if constexpr (S <= 2) {
        reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) R[s] = 0.f;
    }
}

// V sites at once (the network's constants read once for all of them).
template <int S, int V>
__device__ __forceinline__ void source_vec(const StepArgs &a, const AANet &n, const float (&rho)[S][V],
                                           float (&R)[S][V]) {
    if (a.rkind == kMassAction) {
        sm::network_source_vec<S, V>(n, rho, R);
        return;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        float rv[S], Rv[S];
#pragma unroll
        for (int s = 0; s < S; ++s) rv[s] = rho[s][v];
        source<S>(a, n, rv, Rv);
#pragma unroll
        for (int s = 0; s < S; ++s) R[s][v] = Rv[s];
    }
}

// The step of one site (x, y), one thread per site.
template <typename T, int Q, int S, int PHASE>
__device__ __forceinline__ void site_aa(const StepArgs &a, const AANet &net, int64_t x, int64_t y, double (&acc)[S]) {
    using L = Lattice<Q>;
    T *st = static_cast<T *>(a.dst);  // == a.src
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
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

// The step for the V sites (x0 .. x0 + V - 1, y) of the calling thread.
// Every lane of the warp must call it (shuffles); lanes with x0 >= nx or
// y >= ny load valid data but store nothing.  acc gathers the FP64 mass of the live sites.
template <int Q, int S, int V, int PHASE>
__device__ __forceinline__ void tile_aa(const StepArgs &a, const AANet &net, int64_t x0, int64_t y, int lane,
                                        double (&acc)[S]) {
    using L = Lattice<Q>;
    float *st = static_cast<float *>(a.dst);  // == a.src
    const int64_t nx = a.nx, ny = a.ny, pitch = a.pitch, plane = a.plane;
    // Dead lanes (x0 >= nx, or a row y >= ny of a multi-row tile) load a
    // valid row and column for the shuffles and store nothing.
    const bool live = x0 < nx && y < ny;
    const int64_t xc = x0 < nx ? x0 : 0;
    const int64_t yc = y < ny ? y : 0;
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
                ldv<V>(st + (int64_t)(s * Q + opp<Q>(i)) * plane + yc * pitch + xc, v);
#pragma unroll
                for (int j = 0; j < V; ++j) f[s][i][j] = v[j];
            } else {
                const float *row = st + (int64_t)(s * Q + i) * plane + wrap(yc - L::ey(i), ny) * pitch;
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
                float *row = st + (int64_t)(s * Q + opp<Q>(i)) * plane + wrap(yc + L::ey(i), ny) * pitch;
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

}  // namespace aa
}  // namespace lbrd
