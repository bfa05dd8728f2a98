// FP32 step: the remaining launch variants (compiled in their own
// translation unit so that the build runs in parallel).
#include "step_f32_kernel.cuh"

namespace lbrd {

cudaError_t launch_step_f32_variant_b(int v, int Q, int S, const StepArgs &a, cudaStream_t st, bool per_tile) {
    switch (v) {
        case 4: return f32::dispatch_shape<128, 1, 4, 0>(Q, S, a, st, per_tile);
        case 5: return f32::dispatch_shape<64, 2, 4, 1>(Q, S, a, st, per_tile);
        case 6: return f32::dispatch_shape<64, 2, 5, 1>(Q, S, a, st, per_tile);
        case 7: return f32::dispatch_shape<128, 2, 2, 0>(Q, S, a, st, per_tile);
        case 8: case 9: case 10: case 11: case 12: case 13:
            return per_tile ? cudaErrorInvalidValue : launch_step_f32_bulk(v - 8, Q, S, a, st);
        case 14: case 15: case 16: case 17: case 18: case 19: case 20: case 21: case 22: case 23:
        case 24: case 25: case 26: case 27:
            return per_tile ? cudaErrorInvalidValue : launch_step_f32_tb2(v - 14, Q, S, a, st);
        case 28: case 29: case 30: case 31: case 32: case 33: case 34: case 35: case 36: case 37:
        case 38: case 39: case 40: case 41: case 42: case 43: case 44: case 45: case 46: case 47:
        case 48: case 49: case 50: case 51: case 52: case 53: case 54: case 55: case 56: case 57: case 58:
            return per_tile ? cudaErrorInvalidValue : launch_step_f32_deep(v - 28, Q, S, a, st);
        case 59: case 60: case 61: case 62: case 63: case 64: case 65: case 66: case 67: case 68: case 69:
        case 70: case 71: case 72: case 73: case 74: case 75: case 76: case 77: case 78: case 79: case 80:
            return per_tile ? cudaErrorInvalidValue : launch_step_f32_pair(v - 59, Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
