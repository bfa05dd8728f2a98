// 16-bit deviation storage with temporal blocking to depth K, two columns per
// lane: the single-grid launch variants (the kernel is in
// step_half_pair_kernel.cuh).
#include "step_half_pair_kernel.cuh"

namespace lbrd {

namespace {

template <int H, int K, int NW, int NS, int MINB>
cudaError_t dispatch_half_pair(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_half_pair<9, 1, H, K, NW, NS, MINB>(a, st);
    if (Q == 9 && S == 2) return launch_half_pair<9, 2, H, K, NW, NS, MINB>(a, st);
    if (Q == 5 && S == 1) return launch_half_pair<5, 1, H, K, NW, NS, MINB>(a, st);
    if (Q == 5 && S == 2) return launch_half_pair<5, 2, H, K, NW, NS, MINB>(a, st);
    return cudaErrorInvalidValue;
}

template <int H>
cudaError_t dispatch_v(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    switch (v) {
        case 0: return dispatch_half_pair<H, 4, 4, 4, 2>(Q, S, a, st);
        case 1: return dispatch_half_pair<H, 4, 4, 4, 3>(Q, S, a, st);
        case 2: return dispatch_half_pair<H, 5, 4, 4, 2>(Q, S, a, st);
        case 3: return dispatch_half_pair<H, 3, 4, 4, 3>(Q, S, a, st);
        case 4: return dispatch_half_pair<H, 6, 4, 4, 2>(Q, S, a, st);
        case 5: return dispatch_half_pair<H, 2, 4, 4, 4>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// K time steps per launch in 16-bit deviation storage, two columns per lane;
// v: depth and launch shape.  nx a multiple of 8.
cudaError_t launch_step_half_pair(int v, int Q, int S, int half_kind, const StepArgs &a, cudaStream_t st) {
    return half_kind ? dispatch_v<1>(v, Q, S, a, st) : dispatch_v<0>(v, Q, S, a, st);
}

}  // namespace lbrd
