// FP32 step: launch variants (the autotuner picks one per grid), the default
// launch, the per-tile launch and the initialisation kernel.  The kernel body
// is in step_f32_kernel.cuh.
#include "step_f32_kernel.cuh"

namespace lbrd {

namespace {

template <int Q, int S>
__global__ void __launch_bounds__(256) init_f32_kernel(InitArgs a) {
    const int64_t x = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= a.nx) return;
    float f[S][Q], rho[S], R[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float r0 = (float)a.rho0[((int64_t)s * a.ny + y) * a.nx + x];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[s][i] = rn_mul(weight<Q, float>(i), r0);
        float r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i]);
        rho[s] = r;
    }
    reaction_f32<S>(a.rkind, (float)a.kappa, (float)a.F, (float)a.k, rho, R);
    float *dst = static_cast<float *>(a.dst);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float om = (float)a.omega[s];
        const float t = rn_fma(om, rho[s], R[s]);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] =
                rn_fma(rn_sub(1.f, om), f[s][i], rn_mul(weight<Q, float>(i), t));
        if (a.rho_out) static_cast<float *>(a.rho_out)[(int64_t)s * a.plane + y * a.pitch + x] = rho[s];
    }
}

}  // namespace

// Variant table: {threads along x, rows per tile, min blocks per SM, cache policy}.
const F32Variant kF32Variants[] = {
    {"64x2_minb4", 64, 2, 4, 0, 1, 1},
    {"64x2_minb5", 64, 2, 5, 0, 1, 1},
    {"64x2_minb2", 64, 2, 2, 0, 1, 1},
    {"32x4_minb4", 32, 4, 4, 0, 1, 1},
    {"128x1_minb4", 128, 1, 4, 0, 1, 1},
    {"64x2_minb4_stream", 64, 2, 4, 1, 1, 1},
    {"64x2_minb5_stream", 64, 2, 5, 1, 1, 1},
    {"128x2_minb2", 128, 2, 2, 0, 1, 1},
    // TMA bulk copies into a shared-memory ring (step_f32_bulk.cu): threads, stages
    {"bulk128_s4", 128, 1, 4, 2, 1, 4},
    {"bulk64_s4", 64, 1, 4, 2, 1, 4},
    {"bulk128_s3", 128, 1, 3, 2, 1, 4},
    {"bulk256_s2", 256, 1, 2, 2, 1, 4},
    {"bulk256_s3", 256, 1, 3, 2, 1, 4},
    {"bulk128_s2", 128, 1, 2, 2, 1, 4},
    // temporal blocking, two steps per launch (step_f32_tb.cu): threads, strip width, stages
    {"tb2_288x128_s8", 288, 128, 8, 3, 2, 128},
    {"tb2_288x128_s4x2", 288, 128, 4, 3, 2, 128},
    {"tb2_288x256_s6", 288, 256, 6, 3, 2, 256},
    {"tb2_352x512_s2", 352, 512, 2, 3, 2, 512},
    {"tb2_288x256_s2x2", 288, 256, 2, 3, 2, 256},
    {"tb2_544x512_s2", 544, 512, 2, 3, 2, 512},
    {"tb2i_288x256_s2x2", 288, 256, 2, 3, 2, 256},
    {"tb2i_544x512_s2", 544, 512, 2, 3, 2, 512},
    {"tb2i_160x128_s4x2", 160, 128, 4, 3, 2, 128},
    {"tb2i_288x256_s3", 288, 256, 3, 3, 2, 256},
    {"tb2w_288x256_s2x2", 288, 256, 2, 3, 2, 256},
    {"tb2w_288x256_s4", 288, 256, 4, 3, 2, 256},
    {"tb2w_160x128_s3x3", 160, 128, 3, 3, 2, 128},
    {"tb2w_544x512_s2", 544, 512, 2, 3, 2, 512},
    // temporal blocking to depth K, levels in registers (step_f32_deep_kernel.cuh): threads, K, min blocks
    // per SM; names deep<K>[v][p]_<threads>_minb<blocks>[_s<rows staged>]: v 16-byte staging (nx % 4 == 0),
    // p the pulls from earlier rows first, four staged rows unless _s5
    {"deep1_128_minb4", 128, 1, 4, 4, 1, 1},
    {"deep2_128_minb4", 128, 2, 4, 4, 2, 1},
    {"deep4_128_minb4", 128, 4, 4, 4, 4, 1},
    {"deep4_128_minb3", 128, 4, 3, 4, 4, 1},
    {"deep8_128_minb2", 128, 8, 2, 4, 8, 1},
    {"deep8_128_minb3", 128, 8, 3, 4, 8, 1},
    // 16-byte staging of the level-0 rows
    {"deep2v_128_minb4", 128, 2, 4, 4, 2, 4},
    {"deep4v_128_minb4", 128, 4, 4, 4, 4, 4},
    {"deep4v_128_minb3", 128, 4, 3, 4, 4, 4},
    {"deep8v_128_minb2", 128, 8, 2, 4, 8, 4},
    {"deep4v_128_minb3_s5", 128, 4, 3, 4, 4, 4},
    {"deep4v_192_minb2", 192, 4, 2, 4, 4, 4},
    {"deep4v_192_minb2_s5", 192, 4, 2, 4, 4, 4},
    {"deep4v_96_minb4", 96, 4, 4, 4, 4, 4},
    {"deep6v_128_minb2", 128, 6, 2, 4, 6, 4},
    {"deep8v_192_minb1", 192, 8, 1, 4, 8, 4},
    {"deep5v_128_minb2", 128, 5, 2, 4, 5, 4},
    {"deep5v_192_minb2", 192, 5, 2, 4, 5, 4},
    {"deep6v_192_minb2", 192, 6, 2, 4, 6, 4},
    {"deep6v_128_minb3_s5", 128, 6, 3, 4, 6, 4},
    // 16-byte staging, the pulls from earlier rows at the start of an iteration
    {"deep8vp_128_minb2", 128, 8, 2, 4, 8, 4},
    {"deep6vp_128_minb3_s5", 128, 6, 3, 4, 6, 4},
    {"deep6vp_128_minb2", 128, 6, 2, 4, 6, 4},
    {"deep5vp_192_minb2", 192, 5, 2, 4, 5, 4},
    {"deep7vp_128_minb2", 128, 7, 2, 4, 7, 4},
    {"deep6v_128_minb2_s5", 128, 6, 2, 4, 6, 4},
    {"deep6v_64_minb4", 64, 6, 4, 4, 6, 4},
    {"deep5v_64_minb4", 64, 5, 4, 4, 5, 4},
    {"deep6v_256_minb1", 256, 6, 1, 4, 6, 4},
    // three steps per launch (with the others, the last steps of a call)
    {"deep3v_128_minb3", 128, 3, 3, 4, 3, 4},
    {"deep3_128_minb3", 128, 3, 3, 4, 3, 1},
    // two columns per lane (step_f32_pair_kernel.cuh), 16-byte staging: deep<K>vw[p]_ (nx a multiple
    // of 4), deep<K>vw[p]a_ (any nx)
    {"deep4vw_128_minb2", 128, 4, 2, 4, 4, 4},
    {"deep4vwp_128_minb2", 128, 4, 2, 4, 4, 4},
    {"deep4vw_128_minb2_s5", 128, 4, 2, 4, 4, 4},
    {"deep4vwp_128_minb2_s5", 128, 4, 2, 4, 4, 4},
    {"deep5vw_128_minb2", 128, 5, 2, 4, 5, 4},
    {"deep5vwp_128_minb2", 128, 5, 2, 4, 5, 4},
    {"deep6vwp_128_minb1", 128, 6, 1, 4, 6, 4},
    {"deep4vwp_64_minb4_s5", 64, 4, 4, 4, 4, 4},
    {"deep3vwp_128_minb2_s5", 128, 3, 2, 4, 3, 4},
    {"deep5vwp_128_minb2_s5", 128, 5, 2, 4, 5, 4},
    {"deep5vw_128_minb2_s5", 128, 5, 2, 4, 5, 4},
    {"deep5vwpa_128_minb2", 128, 5, 2, 4, 5, 1},
    {"deep4vwa_128_minb2", 128, 4, 2, 4, 4, 1},
    {"deep6vwpa_128_minb1", 128, 6, 1, 4, 6, 1},
    {"deep3vwpa_128_minb2_s5", 128, 3, 2, 4, 3, 1},
    // two columns per lane, two or three rows staged ahead
    {"deep6vwp_128_minb1_s5", 128, 6, 1, 4, 6, 4},
    {"deep6vwp_128_minb1_s6", 128, 6, 1, 4, 6, 4},
    {"deep5vw_128_minb2_s6", 128, 5, 2, 4, 5, 4},
    {"deep5vw_256_minb1", 256, 5, 1, 4, 5, 4},
    {"deep6vwp_256_minb1_s5", 256, 6, 1, 4, 6, 4},
    {"deep5vwpa_256_minb1", 256, 5, 1, 4, 5, 1},
    // two columns per lane, a row staged as soon as level 1 has read the oldest one: deep<K>vw[p]e_
    {"deep6vwpe_128_minb1_s5", 128, 6, 1, 4, 6, 4},
};
const int kF32VariantCount = sizeof(kF32Variants) / sizeof(kF32Variants[0]);

cudaError_t launch_step_f32_variant_a(int v, int Q, int S, const StepArgs &a, cudaStream_t st, bool per_tile) {
    switch (v) {
        case 0: return f32::dispatch_shape<64, 2, 4, 0>(Q, S, a, st, per_tile);
        case 1: return f32::dispatch_shape<64, 2, 5, 0>(Q, S, a, st, per_tile);
        case 2: return f32::dispatch_shape<64, 2, 2, 0>(Q, S, a, st, per_tile);
        case 3: return f32::dispatch_shape<32, 4, 4, 0>(Q, S, a, st, per_tile);
        default: return launch_step_f32_variant_b(v, Q, S, a, st, per_tile);
    }
}

cudaError_t launch_step_f32_variant(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (v < 0 || v >= kF32VariantCount) return cudaErrorInvalidValue;
    return launch_step_f32_variant_a(v, Q, S, a, st, false);
}

StepShape step_shape_f32(int64_t, int64_t) { return {dim3(max_persistent_blocks()), dim3(64, 2)}; }

cudaError_t launch_step_f32(int Q, int S, const StepArgs &a, cudaStream_t st) {
    return launch_step_f32_variant_a(0, Q, S, a, st, false);
}

cudaError_t launch_init_f32(int Q, int S, const InitArgs &a, cudaStream_t st) {
    const dim3 g((unsigned)((a.nx + 255) / 256), (unsigned)a.ny), b(256);
    if (Q == 9 && S == 1) init_f32_kernel<9, 1><<<g, b, 0, st>>>(a);
    else if (Q == 9 && S == 2) init_f32_kernel<9, 2><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 1) init_f32_kernel<5, 1><<<g, b, 0, st>>>(a);
    else if (Q == 5 && S == 2) init_f32_kernel<5, 2><<<g, b, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// One block per tile instead of the persistent grid: the launch used by the
// allocation-free entry point, whose per-block scratch is sized from the grid.
int64_t step_tiles_f32(int64_t nx, int64_t ny) {
    int64_t tiles_x, ntiles;
    f32::tiles_for<64, 2>(nx, ny, &tiles_x, &ntiles);
    return ntiles;
}

cudaError_t launch_step_f32_per_tile(int Q, int S, const StepArgs &a, cudaStream_t st) {
    return launch_step_f32_variant_a(0, Q, S, a, st, true);
}

}  // namespace lbrd
