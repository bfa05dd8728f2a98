// FP32 step, bulk-copy variant: the same arithmetic as step_f32_kernel.cuh,
// with the pulled rows staged in shared memory by the TMA engine.
//
// Work unit: one row y of one strip of TX = 4 * NT columns.  For every
// species s and velocity i the unit needs row y - e_iy of plane (s, i) at
// columns x - e_ix; one elected thread copies those row segments (with the
// periodic halo column on the side e_ix points to) from HBM into a
// shared-memory stage with cp.async.bulk, completing on the stage's mbarrier.
// STAGES units are in flight per block, so HBM sees several stages of copies
// outstanding while the threads compute the current one from shared memory
// (aligned 128-bit shared loads, the +-1 column shift by warp shuffle, the
// warp-edge lanes read the halo word).  Results go to HBM with 128-bit
// stores.  One block per SM walks the units in row-major order with a
// grid-stride loop.
//
// Stage layout: S * Q slots of TX + 8 floats; slot index k holds column
// x0 - 4 + k.  Copies: e_ix = 0 -> columns [x0, x_end) at k = 4;
// e_ix = +1 -> [x0 - 4, x_end) at k = 0 (x0 = 0 takes [nx - 4, nx) for the
// halo); e_ix = -1 -> [x0, x_end + 4) at k = 4 (past nx it takes [0, 4)).
// Every copy starts on a 16-byte boundary and moves a multiple of 16 bytes
// (nx % 4 == 0, pitch % 32 == 0).
//
// Every mbarrier wait is bounded (about 2^31 clock cycles, ~1 s): on timeout
// the block records LB_RD_ETIMEOUT in the status word, waits (again bounded)
// for its own copies still in flight and returns.
#include <atomic>

#include "step_f32_kernel.cuh"
#include "lb_rd.h"

namespace lbrd {

namespace {

constexpr long long kWaitCycles = 1ll << 31;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

template <int Q, int S, int NT>
struct BulkGeom {
    static constexpr int TX = 4 * NT;
    static constexpr int kSlot = TX + 8;                 // floats per slot
    static constexpr int kStageFloats = S * Q * kSlot;  // floats per stage
};

// Issue the copies of unit u into stage buffer `st`.  Called by all 32 lanes
// of one warp: lane 0 posts the expected bytes, lane p < S * Q issues plane
// p's copies (a negative transaction count before the arrival is allowed).
template <int Q, int S, int NT>
__device__ __forceinline__ void issue_unit(const StepArgs &a, int64_t u, int64_t nstrips, float *st, unsigned bar,
                                           unsigned extra_tx = 0) {
    using L = Lattice<Q>;
    using G = BulkGeom<Q, S, NT>;
    const int lane = threadIdx.x & 31;
    const int64_t y = u / nstrips;
    const int64_t x0 = (u - y * nstrips) * G::TX;
    const int64_t xe = x0 + G::TX < a.nx ? x0 + G::TX : a.nx;
    const float *src = static_cast<const float *>(a.src);
    if (lane == 0) {
        unsigned total = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) total += (unsigned)((xe - x0) + (L::ex(i) != 0 ? 4 : 0)) * 4u;
        mbar_expect_tx(bar, total * S + extra_tx);
    }
    __syncwarp();
    if (lane >= S * Q) return;
    const int s = lane / Q, i = lane - s * Q;
    int ex = 0, ey = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (q == i) {
            ex = L::ex(q);
            ey = L::ey(q);
        }
    const int64_t yr = wrap(y - ey, a.ny);
    const float *row = src + (int64_t)(s * Q + i) * a.plane + yr * a.pitch;
    float *slot = st + (s * Q + i) * G::kSlot;
    if (ex == 0) {
        bulk_copy(smem_u32(slot + 4), row + x0, (unsigned)(xe - x0) * 4u, bar);
    } else if (ex == 1) {
        if (x0 == 0) {
            bulk_copy(smem_u32(slot), row + a.nx - 4, 16u, bar);
            bulk_copy(smem_u32(slot + 4), row, (unsigned)xe * 4u, bar);
        } else {
            bulk_copy(smem_u32(slot), row + x0 - 4, (unsigned)(xe - x0 + 4) * 4u, bar);
        }
    } else {
        if (xe == a.nx) {
            bulk_copy(smem_u32(slot + 4), row + x0, (unsigned)(xe - x0) * 4u, bar);
            bulk_copy(smem_u32(slot + 4 + (xe - x0)), row, 16u, bar);
        } else {
            bulk_copy(smem_u32(slot + 4), row + x0, (unsigned)(xe - x0 + 4) * 4u, bar);
        }
    }
}

template <int Q, int S, int NT, int STAGES>
__global__ void __launch_bounds__(NT, 1) step_bulk_kernel(StepArgs a, int64_t nstrips, int64_t nunits) {
    using L = Lattice<Q>;
    using G = BulkGeom<Q, S, NT>;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) unsigned long long bars[STAGES];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t nx = a.nx;

    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();

    // units of this block: u_j = blockIdx.x + j * gridDim.x
    const int64_t nmine = blockIdx.x < nunits ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid < 32) {
        for (int k = 0; k < STAGES && k < nmine; ++k)
            issue_unit<Q, S, NT>(a, blockIdx.x + (int64_t)k * gridDim.x, nstrips, smem + k * G::kStageFloats,
                                 smem_u32(&bars[k]), (a.inject_timeout && blockIdx.x == 0 && k == 0) ? 16u : 0u);
    }
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    float *__restrict__ dst = static_cast<float *>(a.dst);

    int64_t j = 0;
    for (; j < nmine; ++j) {
        const int stage = (int)(j % STAGES);
        const unsigned parity = (unsigned)((j / STAGES) & 1);
        if (!mbar_wait(smem_u32(&bars[stage]), parity)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        const int64_t u = blockIdx.x + j * gridDim.x;
        const int64_t y = u / nstrips;
        const int64_t x0s = (u - y * nstrips) * G::TX;
        const int64_t x0 = x0s + 4 * tid;
        const bool live = x0 < nx;
        const float *st = smem + stage * G::kStageFloats;

        float f[S][Q][4];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float *slot = st + (s * Q + i) * G::kSlot;
                const float4 v = *reinterpret_cast<const float4 *>(slot + 4 + 4 * tid);
                const int ex = L::ex(i);
                if (ex == 0) {
                    f[s][i][0] = v.x; f[s][i][1] = v.y; f[s][i][2] = v.z; f[s][i][3] = v.w;
                } else if (ex == 1) {
                    float left = __shfl_up_sync(kFullMask, v.w, 1);
                    if (lane == 0) left = slot[3 + 4 * tid];
                    f[s][i][0] = left; f[s][i][1] = v.x; f[s][i][2] = v.y; f[s][i][3] = v.z;
                } else {
                    float right = __shfl_down_sync(kFullMask, v.x, 1);
                    if (lane == 31) right = slot[8 + 4 * tid];
                    f[s][i][0] = v.y; f[s][i][1] = v.z; f[s][i][2] = v.w; f[s][i][3] = right;
                }
            }
        }
        // all reads of this stage are done: refill it with unit j + STAGES
        __syncthreads();
        if (tid < 32 && j + STAGES < nmine) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_unit<Q, S, NT>(a, blockIdx.x + (j + STAGES) * gridDim.x, nstrips, smem + stage * G::kStageFloats,
                                 smem_u32(&bars[stage]));
        }

        float rho[S][4];
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                float r = f[s][0][jj];
#pragma unroll
                for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i][jj]);
                rho[s][jj] = r;
            }
        }
        float R[S][4];
        const float kappa = (float)a.kappa, F = (float)a.F, k = (float)a.k;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float rj[S], Rj[S];
#pragma unroll
            for (int s = 0; s < S; ++s) rj[s] = rho[s][jj];
            reaction_f32<S>(a.rkind, kappa, F, k, rj, Rj);
#pragma unroll
            for (int s = 0; s < S; ++s) R[s][jj] = Rj[s];
        }
        if (live) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float om = (float)a.omega[s];
                const float c1 = rn_sub(1.f, om);
                float wt[L::kClasses][4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float t = rn_fma(om, rho[s][jj], R[s][jj]);
#pragma unroll
                    for (int c = 0; c < L::kClasses; ++c) wt[c][jj] = rn_mul(L::template wc<float>(c), t);
                }
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int c = L::wclass(i);
                    float4 o;
                    o.x = rn_fma(c1, f[s][i][0], wt[c][0]);
                    o.y = rn_fma(c1, f[s][i][1], wt[c][1]);
                    o.z = rn_fma(c1, f[s][i][2], wt[c][2]);
                    o.w = rn_fma(c1, f[s][i][3], wt[c][3]);
                    *reinterpret_cast<float4 *>(dst + (int64_t)(s * Q + i) * a.plane + y * a.pitch + x0) = o;
                }
                if (a.rho_out)
                    *reinterpret_cast<float4 *>(static_cast<float *>(a.rho_out) + (int64_t)s * a.plane + y * a.pitch +
                                                x0) = make_float4(rho[s][0], rho[s][1], rho[s][2], rho[s][3]);
                if (a.mass_out)  // FP32 over the four sites, one FP64 add per unit
                    acc[s] += (double)((rho[s][0] + rho[s][1]) + (rho[s][2] + rho[s][3]));
            }
        }
    }
    if (abort_flag) {
        // record the timeout, then wait (bounded) for this block's copies that
        // are still in flight before the block's shared memory goes away
        if (tid == 0) {
            if (a.status) atomicExch(a.status, LB_RD_ETIMEOUT);
            for (int64_t jj = j; jj < nmine && jj < j + STAGES; ++jj)
                mbar_wait(smem_u32(&bars[jj % STAGES]), (unsigned)((jj / STAGES) & 1));
        }
        __syncthreads();
        return;
    }
    if (a.mass_out) block_mass_reduce<S, NT>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S, int NT, int STAGES>
cudaError_t launch_bulk(const StepArgs &a, cudaStream_t st, bool per_unit) {
    using G = BulkGeom<Q, S, NT>;
    if (a.nx % 4) return cudaErrorInvalidValue;
    const int64_t nstrips = (a.nx + G::TX - 1) / G::TX;
    const int64_t nunits = nstrips * a.ny;
    const size_t smem = (size_t)STAGES * G::kStageFloats * sizeof(float);
    auto kern = step_bulk_kernel<Q, S, NT, STAGES>;
    static std::atomic<bool> configured[64] = {};  // per device ordinal (handles on several threads)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev].store(true);
    }
    const unsigned grid = per_unit ? (unsigned)nunits : persistent_blocks(kern, NT, nunits, smem);
    kern<<<grid, NT, smem, st>>>(a, nstrips, nunits);
    return cudaGetLastError();
}

template <int NT, int STAGES>
cudaError_t dispatch_bulk(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_bulk<9, 1, NT, STAGES>(a, st, false);
    if (Q == 9 && S == 2) return launch_bulk<9, 2, NT, STAGES>(a, st, false);
    if (Q == 5 && S == 1) return launch_bulk<5, 1, NT, STAGES>(a, st, false);
    if (Q == 5 && S == 2) return launch_bulk<5, 2, NT, STAGES>(a, st, false);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step_f32_bulk(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    switch (v) {
        case 0: return dispatch_bulk<128, 4>(Q, S, a, st);
        case 1: return dispatch_bulk<64, 4>(Q, S, a, st);
        case 2: return dispatch_bulk<128, 3>(Q, S, a, st);
        case 3: return dispatch_bulk<256, 2>(Q, S, a, st);
        case 4: return dispatch_bulk<256, 3>(Q, S, a, st);
        case 5: return dispatch_bulk<128, 2>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
