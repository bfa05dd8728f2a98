// Temporal blocking to depth K over a list of grids (batches and server
// ticks): the launch shape per K, the (band, strip) plan of the list and the
// launch (the kernel is in step_f32_deep_kernel.cuh).
#include "step_f32_deep_kernel.cuh"
#include "step_f32_pair_kernel.cuh"

namespace lbrd {

namespace {

// Two columns per lane (step_f32_pair_kernel.cuh) where that form is the
// faster one: depths whose carried levels fit the register file without
// heavy spills (K <= 5 for D2Q9, K <= 6 for D2Q5); its any-nx form unless
// every grid has nx a multiple of 4.  Four warps, the pulls from earlier rows
// first, five staged rows below K = 5 and for D2Q5 (whose smaller rows leave
// L1 its share with two rows staged ahead).
template <int Q, int K, bool V16>
struct UsePair {
    static constexpr bool value = Q == 9 ? K <= 5 : K <= 6;
};
template <int Q, int S, int K, bool V16, int RK = -1>
struct PairShape
    : PairKernel<Q, S, K, 4, (K < 5 || Q == 5 ? 5 : 4), (K == 6 ? 1 : 2), true, true, !V16, RK> {
    static constexpr int NW = 4, NS = K < 5 || Q == 5 ? 5 : 4, MINB = K == 6 ? 1 : 2;
};

// Batched launch shapes per K: the single-grid choices (K = 4, 5: six warps,
// two blocks per SM; K = 6, 7, 8: four warps, two blocks per SM; K = 5, 7, 8
// with the pulls from earlier rows first; K = 2, 3, which cover the last steps
// of a call or a tick: four warps, four and three blocks per SM).
template <int Q, int S, int K, bool V16>
struct BatchShape;
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 2, V16> : DeepKernel<Q, S, 2, 4, 4, 4, V16, true> {
    static constexpr int NW = 4;
    static constexpr int MINB = 4;
    static constexpr bool PP = false;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 3, V16> : DeepKernel<Q, S, 3, 4, 4, 3, V16, true> {
    static constexpr int NW = 4;
    static constexpr int MINB = 3;
    static constexpr bool PP = false;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 4, V16> : DeepKernel<Q, S, 4, 6, 4, 2, V16, true> {
    static constexpr int NW = 6;
    static constexpr int MINB = 2;
    static constexpr bool PP = false;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 5, V16> : DeepKernel<Q, S, 5, 6, 4, 2, V16, true, true> {
    static constexpr int NW = 6;
    static constexpr int MINB = 2;
    static constexpr bool PP = true;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 6, V16> : DeepKernel<Q, S, 6, 4, 4, 2, V16, true> {
    static constexpr int NW = 4;
    static constexpr int MINB = 2;
    static constexpr bool PP = false;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 7, V16> : DeepKernel<Q, S, 7, 4, 4, 2, V16, true, true> {
    static constexpr int NW = 4;
    static constexpr int MINB = 2;
    static constexpr bool PP = true;
};
template <int Q, int S, bool V16>
struct BatchShape<Q, S, 8, V16> : DeepKernel<Q, S, 8, 4, 4, 2, V16, true, true> {
    static constexpr int NW = 4;
    static constexpr int MINB = 2;
    static constexpr bool PP = true;
};

template <int Q, int S, int K, bool V16>
int64_t plan_batch(DeepItem *items, int n) {
    constexpr bool pair = UsePair<Q, K, V16>::value;
    constexpr int WO = pair ? PairGeom<K>::WO : 34 - 2 * K;
    int NW = 0;
    unsigned full = 0;
    cudaError_t ge;
    if constexpr (pair) {  // only the kernels a list can run are instantiated
        NW = PairShape<Q, S, K, V16>::NW;
        ge = PairShape<Q, S, K, V16>::get(&full);
    } else {
        NW = BatchShape<Q, S, K, V16>::NW;
        ge = BatchShape<Q, S, K, V16>::get(&full);
    }
    if (ge != cudaSuccess) return -1;
    for (int i = 0; i < n; ++i) items[i].nstrips = (items[i].a.nx + WO - 1) / WO;
    const int64_t h = choose_band_height(K, items, n, (int64_t)full * NW);
    int64_t units = 0;
    for (int i = 0; i < n; ++i) {
        items[i].band = h;
        items[i].unit_begin = units;
        units += items[i].nstrips * ((items[i].a.ny + h - 1) / h);
    }
    return units;
}

template <int Q, int S, int K, bool V16, int RK>
cudaError_t launch_pair_list(const DeepItem *items, int n, int64_t total_units, bool emit, cudaStream_t st) {
    using PS = PairShape<Q, S, K, V16, RK>;
    unsigned full = 0;
    cudaError_t e = PS::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nwarps = (int64_t)full * PS::NW;
    const unsigned grid = total_units < nwarps ? (unsigned)((total_units + PS::NW - 1) / PS::NW) : full;
    step_pair_kernel<Q, S, K, PS::NW, PS::NS, PS::MINB, true, true, !V16, RK>
        <<<grid, PS::NW * 32, PS::smem, st>>>(StepArgs{}, 0, 0, 0, items, n, total_units, emit ? 1 : 0);
    return cudaGetLastError();
}

// rk: the reaction kind of every grid of the list, or -1 (mixed); two-species
// Gray-Scott lists of grids with nx a multiple of 4 run the two-column form
// with the reaction fixed at compile time (in the any-nx list form that
// instantiation spilled more and ran K = 5 at 0.6x the speed of the other).
template <int Q, int S, int K, bool V16>
cudaError_t launch_batch(const DeepItem *items, int n, int64_t total_units, bool emit, int rk, cudaStream_t st) {
    if constexpr (UsePair<Q, K, V16>::value) {
        if constexpr (S == 2 && V16)
            if (rk == kGrayScott) return launch_pair_list<Q, S, K, V16, kGrayScott>(items, n, total_units, emit, st);
        return launch_pair_list<Q, S, K, V16, -1>(items, n, total_units, emit, st);
    } else {
        using BS = BatchShape<Q, S, K, V16>;
        unsigned full = 0;
        cudaError_t e = BS::get(&full);
        if (e != cudaSuccess) return e;
        const int64_t nwarps = (int64_t)full * BS::NW;
        const unsigned grid = total_units < nwarps ? (unsigned)((total_units + BS::NW - 1) / BS::NW) : full;
        step_deep_kernel<Q, S, K, BS::NW, 4, BS::MINB, V16, true, BS::PP>
            <<<grid, BS::NW * 32, BS::smem, st>>>(StepArgs{}, 0, 0, 0, items, n, total_units, emit ? 1 : 0);
        return cudaGetLastError();
    }
}

template <int K, bool V16>
int64_t plan_qs(int Q, int S, DeepItem *items, int n) {
    if (Q == 9 && S == 1) return plan_batch<9, 1, K, V16>(items, n);
    if (Q == 9 && S == 2) return plan_batch<9, 2, K, V16>(items, n);
    if (Q == 5 && S == 1) return plan_batch<5, 1, K, V16>(items, n);
    if (Q == 5 && S == 2) return plan_batch<5, 2, K, V16>(items, n);
    return -1;
}

template <int K, bool V16>
cudaError_t launch_qs(int Q, int S, const DeepItem *items, int n, int64_t total_units, bool emit, int rk,
                      cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_batch<9, 1, K, V16>(items, n, total_units, emit, rk, st);
    if (Q == 9 && S == 2) return launch_batch<9, 2, K, V16>(items, n, total_units, emit, rk, st);
    if (Q == 5 && S == 1) return launch_batch<5, 1, K, V16>(items, n, total_units, emit, rk, st);
    if (Q == 5 && S == 2) return launch_batch<5, 2, K, V16>(items, n, total_units, emit, rk, st);
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t launch_v(int Q, int S, bool v16, const DeepItem *items, int n, int64_t total_units, bool emit, int rk,
                     cudaStream_t st) {
    return v16 ? launch_qs<K, true>(Q, S, items, n, total_units, emit, rk, st)
               : launch_qs<K, false>(Q, S, items, n, total_units, emit, rk, st);
}

}  // namespace

bool batch_deep_depth_ok(int K) { return K >= 2 && K <= 8; }

int batch_deep_default_k(int Q) { return Q == 9 ? 5 : 6; }

int64_t batch_deep_plan(int K, int Q, int S, bool v16, DeepItem *items, int n) {
    switch (K) {
        case 2: return v16 ? plan_qs<2, true>(Q, S, items, n) : plan_qs<2, false>(Q, S, items, n);
        case 3: return v16 ? plan_qs<3, true>(Q, S, items, n) : plan_qs<3, false>(Q, S, items, n);
        case 4: return v16 ? plan_qs<4, true>(Q, S, items, n) : plan_qs<4, false>(Q, S, items, n);
        case 5: return v16 ? plan_qs<5, true>(Q, S, items, n) : plan_qs<5, false>(Q, S, items, n);
        case 6: return v16 ? plan_qs<6, true>(Q, S, items, n) : plan_qs<6, false>(Q, S, items, n);
        case 7: return v16 ? plan_qs<7, true>(Q, S, items, n) : plan_qs<7, false>(Q, S, items, n);
        case 8: return v16 ? plan_qs<8, true>(Q, S, items, n) : plan_qs<8, false>(Q, S, items, n);
        default: return -1;
    }
}

cudaError_t launch_batch_deep(int K, int Q, int S, bool v16, const DeepItem *items, int n, int64_t total_units,
                              bool emit, int rk, cudaStream_t st) {
    switch (K) {
        case 2: return launch_v<2>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 3: return launch_v<3>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 4: return launch_v<4>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 5: return launch_v<5>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 6: return launch_v<6>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 7: return launch_v<7>(Q, S, v16, items, n, total_units, emit, rk, st);
        case 8: return launch_v<8>(Q, S, v16, items, n, total_units, emit, rk, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
