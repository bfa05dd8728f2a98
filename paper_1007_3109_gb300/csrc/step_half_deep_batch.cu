// 16-bit deviation storage with temporal blocking to depth K over a list of
// grids (batches and server ticks): launch shapes per K, the (band, strip)
// plan of the list and the launch.  Lists whose grids all have nx a multiple
// of 8 run the two-column kernel (step_half_pair_kernel.cuh), the others the
// one-column kernel (step_half_deep_kernel.cuh).
#include "step_half_deep_kernel.cuh"
#include "step_half_pair_kernel.cuh"

namespace lbrd {

namespace {

// Four warps per block; resident blocks per SM by the depth's registers.
template <int K>
struct HalfShape {
    static constexpr int NW = 4, NS = 4, MINB = K <= 2 ? 4 : (K <= 4 ? 3 : 2);
};
// The two-column kernel: the single-grid choices (two blocks per SM, three
// at K = 3, four at K = 2).
template <int K>
struct HalfPairShape {
    static constexpr int NW = 4, NS = 4, MINB = K <= 2 ? 4 : (K == 3 ? 3 : 2);
};

template <int Q, int S, int H, int K>
int64_t plan_half_batch(DeepItem *items, int n) {
    const bool v8 = list_nx8(items, n);
    int NW = 0, WO = 0;
    unsigned full = 0;
    if (v8) {
        using PS = HalfPairShape<K>;
        if (HalfPairKernel<Q, S, H, K, PS::NW, PS::NS, PS::MINB, true>::get(&full) != cudaSuccess) return -1;
        NW = PS::NW;
        WO = PairGeom<K>::WO;
    } else {
        using HS = HalfShape<K>;
        if (HalfDeepKernel<Q, S, H, K, HS::NW, HS::NS, HS::MINB, true>::get(&full) != cudaSuccess) return -1;
        NW = HS::NW;
        WO = 34 - 2 * K;
    }
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

template <int Q, int S, int H, int K, int RK>
cudaError_t launch_half_batch_rk(const DeepItem *items, int n, int64_t total_units, bool emit, cudaStream_t st) {
    using HS = HalfShape<K>;
    using HK = HalfDeepKernel<Q, S, H, K, HS::NW, HS::NS, HS::MINB, true, RK>;
    unsigned full = 0;
    cudaError_t e = HK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nwarps = (int64_t)full * HS::NW;
    const unsigned grid = total_units < nwarps ? (unsigned)((total_units + HS::NW - 1) / HS::NW) : full;
    step_half_deep_kernel<Q, S, H, K, HS::NW, HS::NS, HS::MINB, true, RK>
        <<<grid, HS::NW * 32, HK::smem, st>>>(StepArgs{}, 0, 0, 0, items, n, total_units, emit ? 1 : 0);
    return cudaGetLastError();
}

template <int Q, int S, int H, int K, int RK>
cudaError_t launch_half_pair_list(const DeepItem *items, int n, int64_t total_units, bool emit, cudaStream_t st) {
    using PS = HalfPairShape<K>;
    using HK = HalfPairKernel<Q, S, H, K, PS::NW, PS::NS, PS::MINB, true, RK>;
    unsigned full = 0;
    cudaError_t e = HK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nwarps = (int64_t)full * PS::NW;
    const unsigned grid = total_units < nwarps ? (unsigned)((total_units + PS::NW - 1) / PS::NW) : full;
    step_half_pair_kernel<Q, S, H, K, PS::NW, PS::NS, PS::MINB, true, RK>
        <<<grid, PS::NW * 32, HK::smem, st>>>(StepArgs{}, 0, 0, 0, items, n, total_units, emit ? 1 : 0);
    return cudaGetLastError();
}

// rk: the reaction kind of every grid of the list, or -1 (mixed); v8: every
// grid has nx a multiple of 8 (the plan chose the two-column kernel).
template <int Q, int S, int H, int K>
cudaError_t launch_half_batch(const DeepItem *items, int n, int64_t total_units, bool emit, int rk, bool v8,
                              cudaStream_t st) {
    if (v8) {
        if constexpr (S == 2)
            if (rk == kGrayScott)
                return launch_half_pair_list<Q, S, H, K, kGrayScott>(items, n, total_units, emit, st);
        return launch_half_pair_list<Q, S, H, K, -1>(items, n, total_units, emit, st);
    }
    if constexpr (S == 2)
        if (rk == kGrayScott) return launch_half_batch_rk<Q, S, H, K, kGrayScott>(items, n, total_units, emit, st);
    return launch_half_batch_rk<Q, S, H, K, -1>(items, n, total_units, emit, st);
}

template <int H, int K>
int64_t plan_qs(int Q, int S, DeepItem *items, int n) {
    if (Q == 9 && S == 1) return plan_half_batch<9, 1, H, K>(items, n);
    if (Q == 9 && S == 2) return plan_half_batch<9, 2, H, K>(items, n);
    if (Q == 5 && S == 1) return plan_half_batch<5, 1, H, K>(items, n);
    if (Q == 5 && S == 2) return plan_half_batch<5, 2, H, K>(items, n);
    return -1;
}

template <int H, int K>
cudaError_t launch_qs(int Q, int S, const DeepItem *items, int n, int64_t total_units, bool emit, int rk, bool v8,
                      cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_half_batch<9, 1, H, K>(items, n, total_units, emit, rk, v8, st);
    if (Q == 9 && S == 2) return launch_half_batch<9, 2, H, K>(items, n, total_units, emit, rk, v8, st);
    if (Q == 5 && S == 1) return launch_half_batch<5, 1, H, K>(items, n, total_units, emit, rk, v8, st);
    if (Q == 5 && S == 2) return launch_half_batch<5, 2, H, K>(items, n, total_units, emit, rk, v8, st);
    return cudaErrorInvalidValue;
}

template <int H>
int64_t plan_k(int K, int Q, int S, DeepItem *items, int n) {
    switch (K) {
        case 2: return plan_qs<H, 2>(Q, S, items, n);
        case 3: return plan_qs<H, 3>(Q, S, items, n);
        case 4: return plan_qs<H, 4>(Q, S, items, n);
        case 5: return plan_qs<H, 5>(Q, S, items, n);
        default: return -1;
    }
}

template <int H>
cudaError_t launch_k(int K, int Q, int S, const DeepItem *items, int n, int64_t total_units, bool emit, int rk,
                     bool v8, cudaStream_t st) {
    switch (K) {
        case 2: return launch_qs<H, 2>(Q, S, items, n, total_units, emit, rk, v8, st);
        case 3: return launch_qs<H, 3>(Q, S, items, n, total_units, emit, rk, v8, st);
        case 4: return launch_qs<H, 4>(Q, S, items, n, total_units, emit, rk, v8, st);
        case 5: return launch_qs<H, 5>(Q, S, items, n, total_units, emit, rk, v8, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int batch_half_default_k() { return 4; }

int64_t batch_half_deep_plan(int K, int Q, int S, int half_kind, DeepItem *items, int n) {
    return half_kind ? plan_k<1>(K, Q, S, items, n) : plan_k<0>(K, Q, S, items, n);
}

cudaError_t launch_batch_half_deep(int K, int Q, int S, int half_kind, const DeepItem *items, int n,
                                   int64_t total_units, bool emit, int rk, bool v8, cudaStream_t st) {
    return half_kind ? launch_k<1>(K, Q, S, items, n, total_units, emit, rk, v8, st)
                     : launch_k<0>(K, Q, S, items, n, total_units, emit, rk, v8, st);
}

}  // namespace lbrd
