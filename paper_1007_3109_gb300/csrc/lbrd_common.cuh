// Device-side building blocks shared by the step kernels: velocity sets,
// reaction sources, kernel parameter blocks and the FP64 block reduction
// used for the global mass diagnostic.
//
// Method: multi-species lattice BGK with a reaction source (Sec. II.A,
// Eq. relax), zero-velocity equilibrium f_eq = w_i rho_s (Eq. equili), D2Q9
// weights of Eq. Weights.  The velocity order (0,0),(1,0),(0,1),(-1,0),(0,-1),
// (1,1),(-1,1),(-1,-1),(1,-1) is fixed; rho is always summed in that order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbrd {

constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------------------
// Velocity sets (compile-time, fully unrolled loops fold them to constants)
// ---------------------------------------------------------------------------
template <int Q>
struct Lattice;

template <>
struct Lattice<9> {
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    // Weight class: 0 rest, 1 axis, 2 diagonal (Eq. Weights: 4/9, 1/9, 1/36).
    __host__ __device__ static constexpr int wclass(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }
    static constexpr int kClasses = 3;
    // Double: the correctly rounded 4/9, 1/9, 1/36.  Float: w1 one ulp below
    // the rounded 1/9, w2 = w1 / 4 and w0 = 1 - 5 w1, all exact in float, so
    // that the weights sum to exactly 1 (the correctly rounded floats sum to
    // 1 + 2e-8, which would drift the mass by that much every step).
    template <typename T>
    __host__ __device__ static constexpr T wc(int c) {
        if constexpr (sizeof(T) == 4)
            return c == 0 ? T(0x1.c71c74p-2f) : (c == 1 ? T(0x1.c71c70p-4f) : T(0x1.c71c70p-6f));
        else
            return c == 0 ? T(4) / T(9) : (c == 1 ? T(1) / T(9) : T(1) / T(36));
    }
};

template <>
struct Lattice<5> {
    __host__ __device__ static constexpr int ex(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int wclass(int i) { return i == 0 ? 0 : 1; }
    static constexpr int kClasses = 2;
    // D2Q5 (not in the paper): w0 = 1/3, w1..4 = 1/6, c_s^2 = 1/3.  Float:
    // w1 = rounded 1/6 and w0 = 1 - 4 w1 (exact), an exact partition of unity.
    template <typename T>
    __host__ __device__ static constexpr T wc(int c) {
        if constexpr (sizeof(T) == 4)
            return c == 0 ? T(0x1.555554p-2f) : T(0x1.555556p-3f);
        else
            return c == 0 ? T(1) / T(3) : T(1) / T(6);
    }
};

template <int Q, typename T>
__host__ __device__ constexpr T weight(int i) {
    return Lattice<Q>::template wc<T>(Lattice<Q>::wclass(i));
}

// ---------------------------------------------------------------------------
// Reactions (Sec. II.B and Sec. III)
// ---------------------------------------------------------------------------
enum ReactionKind : int { kNone = 0, kLinear = 1, kGrayScott = 2, kMassAction = 3 };

constexpr int kMaxSpecies = 4;     // species of one simulation
constexpr int kMaxReactions = 16;  // steps of a mass-action network

// Mass-action network: step r runs at rate[r] prod_j rho_j^order[r][j] and
// changes species s by change[r][s] (Eq. reac_diff1 for N species).
struct Network {
    int nr;
    double rate[kMaxReactions];
    signed char order[kMaxReactions][kMaxSpecies];
    signed char change[kMaxReactions][kMaxSpecies];
};

// FP32 operations rounded as written.  An FP32 multiply or add without an
// explicit rounding mode may be fused into an FMA by the compiler, and
// whether it is depends on the surrounding code; with these forms every
// kernel performs the same operations and so gives the same bits.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The same operations on pairs of floats, one packed FP32x2 instruction for
// two (sm_100 and later): each component is rounded as the scalar form
// above, so a pair gives the bits of the two scalar operations in half the
// issue slots.
__device__ __forceinline__ float2 rn_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 rn_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 rn_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pair2(float v) { return make_float2(v, v); }

// FP32 and faster paths: (u v) v;  fma(F, 1 - u, -uvv);  fma(-(F + k), v,
// uvv);  -kappa rho_A;  kappa rho_A.  RK >= 0 fixes the kind at compile time
// (the caller has checked that kind == RK).
template <int S, int RK = -1>
__device__ __forceinline__ void reaction_f32(int kind, float kappa, float F, float k, const float (&rho)[S],
                                             float (&R)[S]) {
    const int kd = RK >= 0 ? RK : kind;
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.f;
    if (kd == kLinear) {
        R[0] = rn_mul(-kappa, rho[0]);
        if (S == 2) R[S - 1] = rn_mul(kappa, rho[0]);
    } else if (kd == kGrayScott && S == 2) {
        const float u = rho[0], v = rho[S - 1];
        const float uvv = rn_mul(rn_mul(u, v), v);
        R[0] = rn_fma(F, rn_sub(1.f, u), -uvv);
        R[S - 1] = rn_fma(-rn_add(F, k), v, uvv);
    }
}

// The reactions of two sites under one test of the kind (the expressions of
// reaction_f32 site by site, so the same bits).  RK >= 0 fixes the kind at
// compile time (the caller has checked that kind == RK).
template <int S, int RK = -1>
__device__ __forceinline__ void reaction2_f32(int kind, float kappa, float F, float k, const float (&r0)[S],
                                              const float (&r1)[S], float (&R0)[S], float (&R1)[S]) {
    const int kd = RK >= 0 ? RK : kind;
#pragma unroll
    for (int s = 0; s < S; ++s) R0[s] = R1[s] = 0.f;
    if (kd == kLinear) {
        R0[0] = rn_mul(-kappa, r0[0]);
        R1[0] = rn_mul(-kappa, r1[0]);
        if (S == 2) {
            R0[S - 1] = rn_mul(kappa, r0[0]);
            R1[S - 1] = rn_mul(kappa, r1[0]);
        }
    } else if (kd == kGrayScott && S == 2) {
        const float u0 = r0[0], v0 = r0[S - 1], u1 = r1[0], v1 = r1[S - 1];
        const float uvv0 = rn_mul(rn_mul(u0, v0), v0), uvv1 = rn_mul(rn_mul(u1, v1), v1);
        const float fk = -rn_add(F, k);
        R0[0] = rn_fma(F, rn_sub(1.f, u0), -uvv0);
        R1[0] = rn_fma(F, rn_sub(1.f, u1), -uvv1);
        R0[S - 1] = rn_fma(fk, v0, uvv0);
        R1[S - 1] = rn_fma(fk, v1, uvv1);
    }
}

// FP64 path: every operation rounded on its own (no FMA), in the order
// (u v) v;  (-uvv) + F (1 - u);  uvv - (F + k) v;  -kappa rho_A;  kappa rho_A.
template <int S>
__device__ __forceinline__ void reaction_f64(int kind, double kappa, double F, double k, const double (&rho)[S],
                                             double (&R)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) R[s] = 0.0;
    if (kind == kLinear) {
        R[0] = -__dmul_rn(kappa, rho[0]);
        if (S == 2) R[S - 1] = __dmul_rn(kappa, rho[0]);
    } else if (kind == kGrayScott && S == 2) {
        const double u = rho[0], v = rho[S - 1];
        const double uvv = __dmul_rn(__dmul_rn(u, v), v);
        R[0] = __dadd_rn(-uvv, __dmul_rn(F, __dsub_rn(1.0, u)));
        R[S - 1] = __dsub_rn(uvv, __dmul_rn(__dadd_rn(F, k), v));
    }
}

// ---------------------------------------------------------------------------
// Kernel parameters
// ---------------------------------------------------------------------------
struct StepArgs {
    const void *src;    // f*(t): post-collision state, planes [s][i][y][pitch]
    void *dst;          // f*(t + 1)
    int64_t nx, ny;
    int64_t pitch;      // row pitch in elements (a multiple of 32)
    int64_t plane;      // ny * pitch
    double omega[kMaxSpecies];  // 1 / tau_s
    int rkind;
    double kappa, F, k;
    Network net;        // kMassAction only
    void *rho_out;      // optional rho(t + 1), [s][y][pitch] in the compute type
    double *partials;   // optional per-block mass partials [nblocks][S]
    unsigned int *counter;  // arrival counter for the last-block finalisation
    double *mass_out;   // optional sum_x rho_s(t + 1), S doubles
    int *status;        // optional error word: a kernel whose bounded wait gave up writes its status here
    int inject_timeout; // test switch: block 0's first stage waits for 16 bytes that never come
};

// Initialisation: f_i = w_i rho0, then the collision of step 0 at every site,
// stored in place (the state is always the post-collision f*(t)).
struct InitArgs {
    const double *rho0;  // [S][ny][nx]
    void *dst;
    int64_t nx, ny, pitch, plane;
    double omega[kMaxSpecies];
    int rkind;
    double kappa, F, k;
    Network net;
    void *rho_out;       // rho(0), [s][y][pitch]
};

// ---------------------------------------------------------------------------
// Global FP64 sum: per-block partial, then the last block to arrive adds the
// partials in block order.  Deterministic for a given launch shape.
// ---------------------------------------------------------------------------
template <int S, int NT>
__device__ __forceinline__ void block_mass_reduce(double (&acc)[S], double *partials, unsigned int *counter,
                                                  double *mass_out) {
    __shared__ double red[NT / 32][S];
    __shared__ bool last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.x + blockIdx.y * gridDim.x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double v = acc[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
        if (lane == 0) red[warp][s] = v;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            double v = 0.0;
            for (int w = 0; w < NT / 32; ++w) v += red[w][s];
            partials[(size_t)bid * S + s] = v;
        }
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v[S];
#pragma unroll
    for (int s = 0; s < S; ++s) v[s] = 0.0;
    for (unsigned b = tid; b < nblocks; b += NT) {
#pragma unroll
        for (int s = 0; s < S; ++s) v[s] += __ldcg(&partials[(size_t)b * S + s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(kFullMask, v[s], o);
        if (lane == 0) red[warp][s] = v[s];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            double m = 0.0;
            for (int w = 0; w < NT / 32; ++w) m += red[w][s];
            mass_out[s] = m;
        }
        *counter = 0u;  // ready for the next launch on this stream
    }
}

__host__ __device__ inline int64_t wrap(int64_t a, int64_t n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

}  // namespace lbrd
