// Temporal blocking to depth K: the single-grid launch variants (the
// kernel, its staging and its arithmetic are in step_f32_deep_kernel.cuh).
#include "step_f32_deep_kernel.cuh"

namespace lbrd {

namespace {

template <int K, int NW, int NS, int MINB, bool V16 = false, bool PP = false>
cudaError_t dispatch_deep(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_deep<9, 1, K, NW, NS, MINB, V16, PP>(a, st);
    if (Q == 9 && S == 2) return launch_deep<9, 2, K, NW, NS, MINB, V16, PP>(a, st);
    if (Q == 5 && S == 1) return launch_deep<5, 1, K, NW, NS, MINB, V16, PP>(a, st);
    if (Q == 5 && S == 2) return launch_deep<5, 2, K, NW, NS, MINB, V16, PP>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace

// K time steps per launch (state t -> t + K).  v: depth and launch shape.
cudaError_t launch_step_f32_deep(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    switch (v) {
        case 0: return dispatch_deep<1, 4, 4, 4>(Q, S, a, st);
        case 1: return dispatch_deep<2, 4, 4, 4>(Q, S, a, st);
        case 2: return dispatch_deep<4, 4, 4, 4>(Q, S, a, st);
        case 3: return dispatch_deep<4, 4, 4, 3>(Q, S, a, st);
        case 4: return dispatch_deep<8, 4, 4, 2>(Q, S, a, st);
        case 5: return dispatch_deep<8, 4, 4, 3>(Q, S, a, st);
        case 6: return dispatch_deep<2, 4, 4, 4, true>(Q, S, a, st);
        case 7: return dispatch_deep<4, 4, 4, 4, true>(Q, S, a, st);
        case 8: return dispatch_deep<4, 4, 4, 3, true>(Q, S, a, st);
        case 9: return dispatch_deep<8, 4, 4, 2, true>(Q, S, a, st);
        case 10: return dispatch_deep<4, 4, 5, 3, true>(Q, S, a, st);
        case 11: return dispatch_deep<4, 6, 4, 2, true>(Q, S, a, st);
        case 12: return dispatch_deep<4, 6, 5, 2, true>(Q, S, a, st);
        case 13: return dispatch_deep<4, 3, 4, 4, true>(Q, S, a, st);
        case 14: return dispatch_deep<6, 4, 4, 2, true>(Q, S, a, st);
        case 15: return dispatch_deep<8, 6, 4, 1, true>(Q, S, a, st);
        case 16: return dispatch_deep<5, 4, 4, 2, true>(Q, S, a, st);
        case 17: return dispatch_deep<5, 6, 4, 2, true>(Q, S, a, st);
        case 18: return dispatch_deep<6, 6, 4, 2, true>(Q, S, a, st);
        case 19: return dispatch_deep<6, 4, 5, 3, true>(Q, S, a, st);
        // the pulls from earlier rows first (PP)
        case 20: return dispatch_deep<8, 4, 4, 2, true, true>(Q, S, a, st);
        case 21: return dispatch_deep<6, 4, 5, 3, true, true>(Q, S, a, st);
        case 22: return dispatch_deep<6, 4, 4, 2, true, true>(Q, S, a, st);
        case 23: return dispatch_deep<5, 6, 4, 2, true, true>(Q, S, a, st);
        case 24: return dispatch_deep<7, 4, 4, 2, true, true>(Q, S, a, st);
        case 25: return dispatch_deep<6, 4, 5, 2, true>(Q, S, a, st);
        case 26: return dispatch_deep<6, 2, 4, 4, true>(Q, S, a, st);
        case 27: return dispatch_deep<5, 2, 4, 4, true>(Q, S, a, st);
        case 28: return dispatch_deep<6, 8, 4, 1, true>(Q, S, a, st);
        case 29: return dispatch_deep<3, 4, 4, 3, true>(Q, S, a, st);
        case 30: return dispatch_deep<3, 4, 4, 3>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
