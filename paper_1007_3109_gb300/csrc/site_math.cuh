// Per-site arithmetic shared by the general (N-species) and in-place step
// kernels: the mass-action source of a network copied to shared memory,
// the relaxation of one population and the ordered density sum.
//
// Network (Eq. reac_diff1 for N species): step r proceeds at
// rate_r = rate[r] prod_j rho_j^order[r][j] and changes species s by
// change[r][s]; evaluated as p = rate_r, p = p * rho_j (order[r][j] times,
// j ascending), R_s = R_s + change[r][s] * p (steps in order, zero changes
// skipped).  FP64 rounds every operation on its own; FP32 uses plain float
// arithmetic with the rate rounded to float once.
#pragma once

#include "lbrd_common.cuh"

namespace lbrd {
namespace sm {

struct NetSmem {
    int nr;
    double rate[kMaxReactions];
    float ratef[kMaxReactions];
    signed char order[kMaxReactions][kMaxSpecies];
    signed char change[kMaxReactions][kMaxSpecies];
};

// One thread of the block copies the network; every thread must call it.
__device__ __forceinline__ void load_net(const Network &n, NetSmem &sn) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
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
__device__ __forceinline__ void network_source(const NetSmem &n, const double (&rho)[S], double (&R)[S]) {
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
__device__ __forceinline__ void network_source(const NetSmem &n, const float (&rho)[S], float (&R)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.f;
    for (int r = 0; r < n.nr; ++r) {
        float p = n.ratef[r];
#pragma unroll
        for (int j = 0; j < S; ++j)
            for (int e = 0; e < n.order[r][j]; ++e) p = rn_mul(p, rho[j]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int c = n.change[r][s];
            if (c != 0) R[s] = rn_fma((float)c, p, R[s]);
        }
    }
}

// V sites at once: each step's constants read once for all V sites; per site
// the same operations in the same order as network_source.
template <int S, int V>
__device__ __forceinline__ void network_source_vec(const NetSmem &n, const float (&rho)[S][V], float (&R)[S][V]) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int v = 0; v < V; ++v) R[s][v] = 0.f;
    for (int r = 0; r < n.nr; ++r) {
        float p[V];
        const float k = n.ratef[r];
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = k;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int o = n.order[r][j];
            for (int e = 0; e < o; ++e)
#pragma unroll
                for (int v = 0; v < V; ++v) p[v] = rn_mul(p[v], rho[j][v]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int c = n.change[r][s];
            if (c != 0) {
                const float cf = (float)c;
#pragma unroll
                for (int v = 0; v < V; ++v) R[s][v] = rn_fma(cf, p[v], R[s][v]);
            }
        }
    }
}

// Post-collision value of one population (Eq. relax): FP64 in the oracle's
// order; FP32 as post = (1 - omega) f + w (omega rho + R).
__device__ __forceinline__ double relax(double f, double w, double rho, double om, double R) {
    return __dadd_rn(__dadd_rn(f, __dmul_rn(__dsub_rn(__dmul_rn(w, rho), f), om)), __dmul_rn(w, R));
}
__device__ __forceinline__ float relax(float f, float w, float rho, float om, float R) {
    return rn_fma(rn_sub(1.f, om), f, rn_mul(w, rn_fma(om, rho, R)));
}

// The density sum's additions (index order; FP64 never contracted).
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return rn_add(a, b); }

}  // namespace sm
}  // namespace lbrd
