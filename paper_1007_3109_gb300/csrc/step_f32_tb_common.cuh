// Per-site step and per-grid arguments shared by the multi-step FP32
// kernels (two steps per launch in step_f32_tb.cu, K steps per launch in
// step_f32_deep_kernel.cuh).  collide_site is the one-step kernels' arithmetic
// (density in index order, reaction, relaxation with source of Eq. relax in
// the FP32 form fma(1 - omega, f, w (omega rho + R))), so a multi-step launch
// gives the bits of as many single steps.
#pragma once

#include "step_f32_kernel.cuh"

namespace lbrd {
namespace tb {

// The fused step of one site from S * Q pulled values.
template <int Q, int S, typename Args>
__device__ __forceinline__ void collide_site(const Args &a, float (&f)[S][Q], float (&rho)[S]) {
    using L = Lattice<Q>;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i]);
        rho[s] = r;
    }
    float R[S];
    reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float om = (float)a.omega[s];
        const float c1 = rn_sub(1.f, om);
        const float t = rn_fma(om, rho[s], R[s]);
        float wt[L::kClasses];
#pragma unroll
        for (int c = 0; c < L::kClasses; ++c) wt[c] = rn_mul(L::template wc<float>(c), t);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = rn_fma(c1, f[s][i], wt[L::wclass(i)]);
    }
}

// collide_site for two sites at once: the two density sums side by side and
// one test of the reaction kind (RK >= 0: fixed at compile time), the same
// operations per site in the same order, so the same bits.  Two forms: one
// scalar instruction per operation and site, or the two sites' operands
// packed in pairs (FP32x2 instructions for the density sums and the
// relaxation, half the issue slots).  Packed operands must sit in aligned
// register pairs, which costs moves after the shifted pulls and, in kernels
// already at the register limit, spills: the packed form is taken where a
// level's carried state is small (S Q <= 10: D2Q5, or one D2Q9 species).
template <int Q, int S>
struct PackPair {
    static constexpr bool value = S * Q <= 10;
};

template <int Q, int S, int RK = -1, typename Args>
__device__ __forceinline__ void collide_pair(const Args &a, float (&f0)[S][Q], float (&f1)[S][Q], float (&rho0)[S],
                                             float (&rho1)[S]) {
    using L = Lattice<Q>;
    if constexpr (PackPair<Q, S>::value) {
        float2 r[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            r[s] = make_float2(f0[s][0], f1[s][0]);
#pragma unroll
            for (int i = 1; i < Q; ++i) r[s] = rn_add2(r[s], make_float2(f0[s][i], f1[s][i]));
            rho0[s] = r[s].x;
            rho1[s] = r[s].y;
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float r0 = f0[s][0], r1 = f1[s][0];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                r0 = rn_add(r0, f0[s][i]);
                r1 = rn_add(r1, f1[s][i]);
            }
            rho0[s] = r0;
            rho1[s] = r1;
        }
    }
    float R0[S], R1[S];
    reaction2_f32<S, RK>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho0, rho1, R0, R1);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float om = (float)a.omega[s];
        const float c1 = rn_sub(1.f, om);
        const float t0 = rn_fma(om, rho0[s], R0[s]), t1 = rn_fma(om, rho1[s], R1[s]);
        float wt0[L::kClasses], wt1[L::kClasses];
#pragma unroll
        for (int c = 0; c < L::kClasses; ++c) {
            wt0[c] = rn_mul(L::template wc<float>(c), t0);
            wt1[c] = rn_mul(L::template wc<float>(c), t1);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (PackPair<Q, S>::value) {
                const float2 v = rn_fma2(pair2(c1), make_float2(f0[s][i], f1[s][i]),
                                         make_float2(wt0[L::wclass(i)], wt1[L::wclass(i)]));
                f0[s][i] = v.x;
                f1[s][i] = v.y;
            } else {
                f0[s][i] = rn_fma(c1, f0[s][i], wt0[L::wclass(i)]);
                f1[s][i] = rn_fma(c1, f1[s][i], wt1[L::wclass(i)]);
            }
        }
    }
}

// The fields of one grid a multi-step segment needs, in registers (FP32 copies
// of the relaxation rates and reaction constants: the values the one-step
// kernels compute with).
struct SegArgs {
    const void *src;
    void *dst;
    void *rho_out;  // rho of the stored level ([s][y][pitch] float), or null
    int64_t nx, ny, pitch, plane;
    float omega[2];
    int rkind;
    float kappa, F, k;
};

__device__ __forceinline__ void load_seg(const StepArgs &a, SegArgs &g) {
    g.src = a.src;
    g.dst = a.dst;
    g.rho_out = a.rho_out;
    g.nx = a.nx;
    g.ny = a.ny;
    g.pitch = a.pitch;
    g.plane = a.plane;
    g.omega[0] = (float)a.omega[0];
    g.omega[1] = (float)a.omega[1];
    g.rkind = a.rkind;
    g.kappa = (float)a.kappa;
    g.F = (float)a.F;
    g.k = (float)a.k;
}

}  // namespace tb
}  // namespace lbrd
