// FP64 per-site update, shared by the single-simulation and batched kernels.
//
// One site: pull f_i(x, t + 1) = f*_i(x - e_i, t) (periodic), rho_s = sum_i f_i
// in index order, R_s(rho) from the reaction, then Eq. relax
//   post = f + (w_i rho - f) * omega + w_i R
// with every floating-point operation rounded on its own (__dadd_rn /
// __dmul_rn are never contracted into FMA), in that operation order, so the
// result is bit-reproducible against a plain FP64 implementation of the
// method.
#pragma once

#include "lbrd_common.cuh"

namespace lbrd {
namespace f64 {

template <int Q, int S>
__device__ __forceinline__ void site_f64(const StepArgs &a, int64_t x, int64_t y, double *acc) {
    using L = Lattice<Q>;
    const double *__restrict__ src = static_cast<const double *>(a.src);
    double *__restrict__ dst = static_cast<double *>(a.dst);
    double f[S][Q], rho[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int64_t xs = wrap(x - L::ex(i), a.nx);
            const int64_t ys = wrap(y - L::ey(i), a.ny);
            f[s][i] = src[(int64_t)(s * Q + i) * a.plane + ys * a.pitch + xs];
        }
        double r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = __dadd_rn(r, f[s][i]);
        rho[s] = r;
    }
    double R[S];
    reaction_f64<S>(a.rkind, a.kappa, a.F, a.k, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double om = a.omega[s];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double w = weight<Q, double>(i);
            const double feq = __dmul_rn(w, rho[s]);
            const double post =
                __dadd_rn(__dadd_rn(f[s][i], __dmul_rn(__dsub_rn(feq, f[s][i]), om)), __dmul_rn(w, R[s]));
            dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] = post;
        }
        if (a.rho_out) static_cast<double *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
        acc[s] = __dadd_rn(acc[s], rho[s]);
    }
}

}  // namespace f64
}  // namespace lbrd
