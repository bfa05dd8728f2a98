// Temporal blocking to depth K with two columns per lane: the single-grid
// launch variants (the kernel is in step_f32_pair_kernel.cuh).
#include "step_f32_pair_kernel.cuh"

namespace lbrd {

namespace {

template <int K, int NW, int NS, int MINB, bool PP, bool ANY = false, bool EA = false>
cudaError_t dispatch_pair(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_pair<9, 1, K, NW, NS, MINB, PP, ANY, EA>(a, st);
    if (Q == 9 && S == 2) return launch_pair<9, 2, K, NW, NS, MINB, PP, ANY, EA>(a, st);
    if (Q == 5 && S == 1) return launch_pair<5, 1, K, NW, NS, MINB, PP, ANY, EA>(a, st);
    if (Q == 5 && S == 2) return launch_pair<5, 2, K, NW, NS, MINB, PP, ANY, EA>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace

// K time steps per launch, two columns per lane.  v: depth and launch shape.
cudaError_t launch_step_f32_pair(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    switch (v) {
        case 0: return dispatch_pair<4, 4, 4, 2, false>(Q, S, a, st);
        case 1: return dispatch_pair<4, 4, 4, 2, true>(Q, S, a, st);
        case 2: return dispatch_pair<4, 4, 5, 2, false>(Q, S, a, st);
        case 3: return dispatch_pair<4, 4, 5, 2, true>(Q, S, a, st);
        case 4: return dispatch_pair<5, 4, 4, 2, false>(Q, S, a, st);
        case 5: return dispatch_pair<5, 4, 4, 2, true>(Q, S, a, st);
        case 6: return dispatch_pair<6, 4, 4, 1, true>(Q, S, a, st);
        case 7: return dispatch_pair<4, 2, 5, 4, true>(Q, S, a, st);
        case 8: return dispatch_pair<3, 4, 5, 2, true>(Q, S, a, st);
        case 9: return dispatch_pair<5, 4, 5, 2, true>(Q, S, a, st);
        case 10: return dispatch_pair<5, 4, 5, 2, false>(Q, S, a, st);
        // any nx
        case 11: return dispatch_pair<5, 4, 4, 2, true, true>(Q, S, a, st);
        case 12: return dispatch_pair<4, 4, 4, 2, false, true>(Q, S, a, st);
        case 13: return dispatch_pair<6, 4, 4, 1, true, true>(Q, S, a, st);
        case 14: return dispatch_pair<3, 4, 5, 2, true, true>(Q, S, a, st);
        // more rows staged ahead (two or three): the smaller D2Q5 rows leave L1 its share
        case 15: return dispatch_pair<6, 4, 5, 1, true>(Q, S, a, st);
        case 16: return dispatch_pair<6, 4, 6, 1, true>(Q, S, a, st);
        case 17: return dispatch_pair<5, 4, 6, 2, false>(Q, S, a, st);
        // eight warps per block, one block per SM: the SM's warps walk eight adjacent strips
        case 18: return dispatch_pair<5, 8, 4, 1, false>(Q, S, a, st);
        case 19: return dispatch_pair<6, 8, 5, 1, true>(Q, S, a, st);
        case 20: return dispatch_pair<5, 8, 4, 1, true, true>(Q, S, a, st);
        // a row staged as soon as level 1 has read the oldest one (one more row in flight;
        // D2Q5: the D2Q9 forms are slower so)
        case 21: return dispatch_pair<6, 4, 5, 1, true, false, true>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
