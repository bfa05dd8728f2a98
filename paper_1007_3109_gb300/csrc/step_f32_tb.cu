// FP32 temporal blocking: two time steps of Eq. relax per pass over HBM.
//
// Work: strips of TX columns; each block takes a contiguous range of the
// (strip, row) pairs (one or a few row segments) and walks it row by row
// (2.5-D streaming):
//   * level 0 (the stored state f*(t)) arrives by TMA bulk copy: for the
//     level-1 row r, plane (s, i) row r - e_iy, columns [x0 - 4, x0 + TX + 4)
//     (periodic wrap), into a stage of a shared-memory pipeline (NS stages);
//   * level 1 (f*(t + 1)) is computed on columns [x0 - 1, x0 + TX + 1) into
//     a ring of four rows in shared memory;
//   * level 2 (f*(t + 2)) of row r - 2 is computed from level-1 rows r - 3,
//     r - 2, r - 1 (finished in earlier iterations) in the same thread loop
//     as level 1 of row r, and written to HBM: one barrier per row.
// Each level is the fused step of the FP32 kernels (pull, rho in index
// order, reaction, BGK + source), so the result is bitwise that of two
// single steps.  HBM sees one read and one write of the state per two steps
// plus the halos (8 columns per strip and two rows per segment).  Needs
// nx % TX == 0.
//
// Threads map to consecutive columns (column = thread + NT * j), so shared
// loads and stores of a warp touch consecutive words (no bank conflicts) and
// global stores are coalesced 128-byte rows.  Every mbarrier wait is bounded
// as in the bulk-copy kernel (status word, drain, return).
#include <atomic>

#include "step_f32_tb_common.cuh"
#include "lb_rd.h"

namespace lbrd {

namespace {

using namespace tb;

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

template <int Q, int S, int TX>
struct TbGeom {
    static constexpr int W0 = TX + 8;   // level-0 slot: columns [x0 - 4, x0 + TX + 4)
    static constexpr int W1 = TX + 8;   // level-1 slot: columns [x0 - 4, x0 + TX + 4) (x0 - 1 .. x0 + TX used)
    static constexpr int kStage = S * Q * W0;
    static constexpr int kRow1 = S * Q * W1;
};

// Copy [c0, c1) of a periodic row (c0 may be < 0, c1 may be > nx; c1 - c0 <= nx
// + 8) into dst, in up to three 16-byte aligned pieces.  Returns the bytes.
__device__ __forceinline__ unsigned copy_periodic(float *dst, const float *row, int64_t c0, int64_t c1, int64_t nx,
                                                  unsigned bar, bool issue) {
    unsigned bytes = 0;
    int64_t c = c0;
    float *d = dst;
    while (c < c1) {
        const int64_t cw = c < 0 ? c + nx : (c >= nx ? c - nx : c);  // wrapped start
        int64_t len = c1 - c;
        if (cw + len > nx) len = nx - cw;
        if (issue) bulk_copy(smem_u32(d), row + cw, (unsigned)len * 4u, bar);
        bytes += (unsigned)len * 4u;
        c += len;
        d += len;
    }
    return bytes;
}

// Issue the level-0 copies for level-1 row r.  Called by all 32 lanes of one
// warp: lane 0 posts the expected bytes, lane p < S * Q issues plane p's
// pieces (a negative transaction count before the arrival is allowed).
template <int Q, int S, int TX, typename Args>
__device__ __forceinline__ void issue_row(const Args &a, int64_t r, int64_t x0, float *st, unsigned bar,
                                          unsigned extra_tx = 0) {
    using L = Lattice<Q>;
    using G = TbGeom<Q, S, TX>;
    const int lane = threadIdx.x & 31;
    const float *src = static_cast<const float *>(a.src);
    if (lane == 0) {
        const unsigned per_plane = copy_periodic(st, src, x0 - 4, x0 + TX + 4, a.nx, bar, false);
        mbar_expect_tx(bar, per_plane * S * Q + extra_tx);
    }
    __syncwarp();
    if (lane < S * Q) {
        const int s = lane / Q, i = lane - s * Q;
        const int ey = (Q == 9) ? Lattice<9>::ey(i) : Lattice<5>::ey(i);
        const int64_t yr = wrap(wrap(r, a.ny) - ey, a.ny);
        const float *row = src + (int64_t)lane * a.plane + yr * a.pitch;
        copy_periodic(st + lane * G::W0, row, x0 - 4, x0 + TX + 4, a.nx, bar, true);
    }
    (void)sizeof(L);
}

// IL = 1 (needs NT >= TX + 2): thread t computes level-1 site t and level-2
// site t of the iteration in one straight-line block (both sets of shared
// loads issued before either collision, from clamped valid addresses; the
// stores are predicated), instead of the items one after the other.  The
// arithmetic of every site is unchanged.
template <int Q, int S, int NT, int TX, int NS, int MINB, int IL>
__global__ void __launch_bounds__(NT, MINB) step_tb2_kernel(StepArgs a, int64_t nstrips) {
    using L = Lattice<Q>;
    using G = TbGeom<Q, S, TX>;
    constexpr int kL1 = TX + 2;       // level-1 columns x0 - 1 .. x0 + TX (slot index 3 .. TX + 4)
    constexpr int kItems = kL1 + TX;  // level-1 and level-2 sites of one iteration
    extern __shared__ __align__(128) float smem[];
    float *stages = smem;                 // NS level-0 stages
    float *ring = smem + NS * G::kStage;  // 4 level-1 rows
    __shared__ __align__(8) unsigned long long bars[NS];
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    float *__restrict__ dst = static_cast<float *>(a.dst);

    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(smem_u32(&bars[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    int64_t ticket = 0;  // level-0 stages consumed by this block so far (stage = ticket % NS)

    // Balanced split: the (strip, row) pairs in strip-major order are cut into
    // gridDim.x contiguous ranges; a range covers one or a few row segments.
    const int64_t total = nstrips * a.ny;
    const int64_t u_end = total * (blockIdx.x + 1) / gridDim.x;
    for (int64_t u = total * blockIdx.x / gridDim.x; u < u_end && !abort_flag;) {
        const int64_t strip = u / a.ny;
        const int64_t y0 = u - strip * a.ny;
        const int64_t ly = (a.ny - y0 < u_end - u) ? a.ny - y0 : u_end - u;
        u += ly;
        const int64_t x0 = strip * TX;
        const int64_t nrows = ly + 2;  // level-1 rows y0 - 1 .. y0 + ly (index j <-> row y0 - 1 + j)
        if (tid < 32)
            for (int64_t j = 0; j < NS && j < nrows; ++j) {
                const int64_t tk = ticket + j;
                issue_row<Q, S, TX>(a, y0 - 1 + j, x0, stages + (tk % NS) * G::kStage, smem_u32(&bars[tk % NS]),
                                    (a.inject_timeout && blockIdx.x == 0 && tk == 0) ? 16u : 0u);
            }
        float sum[S];
#pragma unroll
        for (int s = 0; s < S; ++s) sum[s] = 0.f;
        // Iteration j computes level-1 row j (if j < nrows) and, from level-1
        // rows j - 3 .. j - 1 finished in earlier iterations, level-2 row
        // y = y0 + j - 3 (if 3 <= j <= nrows); one barrier per iteration.
        for (int64_t j = 0; j <= nrows; ++j) {
            const bool do1 = j < nrows, do2 = j >= 3;
            const int64_t tk = ticket + j;
            const int sidx = (int)(tk % NS);
            if (do1 && !mbar_wait(smem_u32(&bars[sidx]), (unsigned)((tk / NS) & 1))) abort_flag = 1;
            const float *st = stages + sidx * G::kStage;
            const unsigned jm = (unsigned)j & 3u;  // j >= 0: j % 4 without a 64-bit division
            float *r1 = ring + jm * G::kRow1;
            // level-1 rows y - 1, y, y + 1 (indices j - 3, j - 2, j - 1) for level 2
            const float *rows1[3] = {ring + ((jm + 1u) & 3u) * G::kRow1, ring + ((jm + 2u) & 3u) * G::kRow1,
                                     ring + ((jm + 3u) & 3u) * G::kRow1};
            const int64_t y = y0 + j - 3;
            if constexpr (IL == 1) {
                static_assert(NT >= kL1, "interleaved items need a thread per level-1 site");
                const bool a1 = do1 && tid < kL1, a2 = do2 && tid < TX;
                const int k1 = (tid < kL1 ? tid : kL1 - 1) + 3;
                const int k2 = tid < TX ? tid : TX - 1;
                float f1[S][Q], f2[S][Q], rho1[S], rho2[S];
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        f1[s][i] = st[(s * Q + i) * G::W0 + k1 - L::ex(i)];
                        f2[s][i] = rows1[1 - L::ey(i)][(s * Q + i) * G::W1 + k2 + 4 - L::ex(i)];
                    }
                collide_site<Q, S>(a, f1, rho1);
                collide_site<Q, S>(a, f2, rho2);
                if (a1) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) r1[(s * Q + i) * G::W1 + k1] = f1[s][i];
                }
                if (a2) {
                    const int64_t x = x0 + k2;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] = f2[s][i];
                        sum[s] += rho2[s];
                    }
                }
            }
            for (int it = tid; IL == 0 && it < kItems; it += NT) {
                float f[S][Q], rho[S];
                if (it < kL1) {
                    if (!do1) continue;
                    const int k1 = it + 3;  // level-1 slot index, column x0 - 4 + k1
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) f[s][i] = st[(s * Q + i) * G::W0 + k1 - L::ex(i)];
                    collide_site<Q, S>(a, f, rho);
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) r1[(s * Q + i) * G::W1 + k1] = f[s][i];
                } else {
                    if (!do2) continue;
                    const int k2 = it - kL1;  // column x0 + k2
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i)  // level-1 row y - e_iy
                            f[s][i] = rows1[1 - L::ey(i)][(s * Q + i) * G::W1 + k2 + 4 - L::ex(i)];
                    collide_site<Q, S>(a, f, rho);
                    const int64_t x = x0 + k2;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) dst[(int64_t)(s * Q + i) * a.plane + y * a.pitch + x] = f[s][i];
                        sum[s] += rho[s];
                    }
                }
            }
            __syncthreads();  // level-1 row j complete, stage consumed, ring slot (j + 1) % 4 free
            if (abort_flag) {
                if (tid == 0) {
                    if (a.status) atomicExch(a.status, LB_RD_ETIMEOUT);
                    for (int64_t jj = j; jj < nrows && jj < j + NS; ++jj)
                        mbar_wait(smem_u32(&bars[(ticket + jj) % NS]), (unsigned)(((ticket + jj) / NS) & 1));
                }
                break;
            }
            if (tid < 32 && do1 && j + NS < nrows) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_row<Q, S, TX>(a, y0 - 1 + j + NS, x0, stages + sidx * G::kStage, smem_u32(&bars[sidx]));
            }
        }
        if (a.mass_out) {
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] += (double)sum[s];
        }
        ticket += nrows;
    }
    if (abort_flag) return;
    if (a.mass_out) block_mass_reduce<S, NT>(acc, a.partials, a.counter, a.mass_out);
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Level-0 row r for the warp-decoupled kernel, by the producer warp.  An
// interior strip (halos inside the row) takes one bulk copy of
// [x0 - 4, x0 + TX + 4) per plane.  A strip at the periodic edge takes one
// bulk copy of [x0, x0 + TX) (16-byte aligned: x0 and nx are multiples of TX)
// and its wrapped halos [x0 - 4, x0), [x0 + TX, x0 + TX + 4) by plain 16-byte
// loads stored into the stage (HALO_LOADS; otherwise by three bulk copies,
// which keep the producer asynchronous: single grids, where the edge strips
// are a few blocks' whole share and would otherwise lag).  Then lane 0
// arrives on the stage's full barrier (count 2 with the expect_tx arrival)
// after a __syncwarp that orders the lanes' halo stores before it.  Grids one
// strip wide (batched 256^2 instances) thus take one copy per plane instead
// of three.
template <int Q, int S, int TX, bool HALO_LOADS, typename Args>
__device__ __forceinline__ void issue_row_tbw(const Args &a, int64_t r, int64_t x0, float *st, unsigned bar,
                                              unsigned extra_tx) {
    using G = TbGeom<Q, S, TX>;
    const int lane = threadIdx.x & 31;
    const float *src = static_cast<const float *>(a.src);
    const bool interior = x0 >= 4 && x0 + TX + 4 <= a.nx;  // the halos do not wrap: one copy per plane
    const bool loads = HALO_LOADS && !interior;
    const unsigned per_plane = (unsigned)(loads ? TX : TX + 8) * 4u;
    if (lane == 0) mbar_expect_tx(bar, per_plane * S * Q + extra_tx);
    __syncwarp();
    if (lane < S * Q) {
        const int i = lane % Q;
        const int ey = (Q == 9) ? Lattice<9>::ey(i) : Lattice<5>::ey(i);
        const int64_t yr = wrap(wrap(r, a.ny) - ey, a.ny);
        const float *row = src + (int64_t)lane * a.plane + yr * a.pitch;
        float *d = st + lane * G::W0;
        if (interior) {
            bulk_copy(smem_u32(d), row + x0 - 4, per_plane, bar);
        } else if (!loads) {
            copy_periodic(d, row, x0 - 4, x0 + TX + 4, a.nx, bar, true);
        } else {
            bulk_copy(smem_u32(d + 4), row + x0, per_plane, bar);
            const int64_t xl = x0 == 0 ? a.nx - 4 : x0 - 4;
            const int64_t xr = x0 + TX == a.nx ? 0 : x0 + TX;
            const float4 hl = *reinterpret_cast<const float4 *>(row + xl);
            const float4 hr = *reinterpret_cast<const float4 *>(row + xr);
            *reinterpret_cast<float4 *>(d) = hl;
            *reinterpret_cast<float4 *>(d + TX + 4) = hr;
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

// Warp-decoupled two-step kernel: W consumer warps and one producer warp.
// The block's strip is TX = 32 W columns; consumer warp w owns the 32
// columns c0 = x0 + 32 w ... and computes level 1 on its 34 columns
// [c0 - 1, c0 + 33) (recomputing the two halo columns its neighbours also
// compute) into a ring of three level-1 rows private to the warp, and level
// 2 of its 32 columns from that ring, so the warp synchronises only with
// itself: each iteration loads everything it needs (the level-0 stage and
// ring rows j - 3 .. j - 1), passes __syncwarp, and only then overwrites the
// ring slot of row j - 3 with level-1 row j.  Level-0 rows arrive by TMA bulk
// copy into NS block-shared stages: the producer warp refills stage k once
// every consumer warp has arrived on its "empty" barrier (count W) and the
// copies complete on its "full" barrier.  Every wait is bounded (status
// word, drain, return); the arithmetic of every site is the one-step
// kernels'.  BATCH: the (strip, row) units of a list of grids (TbwItem, one
// per batched instance, all with nx % TX == 0) instead of one grid; a
// segment never crosses from one grid to the next.
template <int Q, int S, int W, int NS, int MINB, bool BATCH>
__global__ void __launch_bounds__((W + 1) * 32, MINB)
    step_tbw_kernel(StepArgs a, int64_t nstrips, const TbwItem *__restrict__ items, int nitems, int64_t total_units) {
    using L = Lattice<Q>;
    constexpr int TX = 32 * W;
    using G = TbGeom<Q, S, TX>;
    constexpr int RW = 34;                // ring row width: the warp's 34 level-1 columns
    constexpr int kRing = S * Q * RW;     // one level-1 row of one warp
    extern __shared__ __align__(128) float smem[];
    float *stages = smem;                 // NS level-0 stages of the strip
    float *rings = smem + NS * G::kStage; // [W][3] level-1 rows
    __shared__ __align__(8) unsigned long long full[NS], empty[NS];
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) {
            mbar_init(smem_u32(&full[k]), 2);  // expect_tx arrival + halo arrival
            mbar_init(smem_u32(&empty[k]), W);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    int64_t ticket = 0;  // level-0 rows (stages) used by this block so far
    int64_t issued = 0;  // producer: rows issued
    const int64_t total = BATCH ? total_units : nstrips * a.ny;
    const int64_t u_end = total * (blockIdx.x + 1) / gridDim.x;
    float *ring = rings + (w < W ? w : 0) * 3 * kRing;
    int it = 0;  // BATCH: the grid of unit u (a block's units only increase)
    for (int64_t u = total * blockIdx.x / gridDim.x; u < u_end;) {
        SegArgs g;
        int64_t local;
        if constexpr (BATCH) {
            while (it + 1 < nitems && items[it + 1].unit_begin <= u) ++it;
            load_seg(items[it].a, g);
            local = u - items[it].unit_begin;
        } else {
            load_seg(a, g);
            local = u;
        }
        const int64_t strip = local / g.ny;
        const int64_t y0 = local - strip * g.ny;
        const int64_t ly = (g.ny - y0 < u_end - u) ? g.ny - y0 : u_end - u;
        u += ly;
        const int64_t x0 = strip * TX;
        const int64_t nrows = ly + 2;
        float *__restrict__ dst = static_cast<float *>(g.dst);
        // Every decision below is warp-uniform (__any_sync / __all_sync), so the
        // lanes of a warp always take the same path to each __syncwarp.
        if (w == W) {  // producer
            for (int64_t j = 0; j < nrows; ++j) {
                if (__any_sync(kFullMask, abort_flag != 0)) break;
                const int64_t tk = ticket + j;
                const int sk = (int)(tk % NS);
                const bool ok = tk < NS || mbar_wait(smem_u32(&empty[sk]), (unsigned)(((tk / NS) - 1) & 1));
                if (!__all_sync(kFullMask, ok)) {
                    abort_flag = 1;
                    break;
                }
                // the consumers' reads of this stage (generic proxy) before the copies into it (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_row_tbw<Q, S, TX, BATCH>(g, y0 - 1 + j, x0, stages + sk * G::kStage, smem_u32(&full[sk]),
                                    (a.inject_timeout && blockIdx.x == 0 && tk == 0) ? 16u : 0u);
                issued = tk + 1;
            }
        } else {  // consumer warp w
            const int64_t c0 = x0 + 32 * w;
            const int k1 = 32 * w + 3 + lane;  // stage slot of ring column `lane` (column c0 - 1 + lane)
            float sum[S];
#pragma unroll
            for (int s = 0; s < S; ++s) sum[s] = 0.f;
            int m3 = 0;  // j % 3
            for (int64_t j = 0; j <= nrows; ++j, m3 = m3 == 2 ? 0 : m3 + 1) {
                if (__any_sync(kFullMask, abort_flag != 0)) break;
                const bool do1 = j < nrows, do2 = j >= 3;
                const int64_t tk = ticket + j;
                const int sk = (int)(tk % NS);
                const bool ok = !do1 || mbar_wait(smem_u32(&full[sk]), (unsigned)((tk / NS) & 1));
                if (!__all_sync(kFullMask, ok)) {
                    abort_flag = 1;
                    break;
                }
                const float *st = stages + sk * G::kStage;
                // ring slots: row j (written) and rows j - 3, j - 2, j - 1 (read) are j % 3, j % 3, +1, +2
                float *r1 = ring + m3 * kRing;
                const float *rows1[3] = {ring + m3 * kRing, ring + (m3 == 2 ? 0 : m3 + 1) * kRing,
                                         ring + (m3 == 0 ? 2 : m3 - 1) * kRing};
                const int64_t y = y0 + j - 3;
                float f1[S][Q], f2[S][Q], rho1[S], rho2[S];
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        f1[s][i] = st[(s * Q + i) * G::W0 + k1 - L::ex(i)];
                        f2[s][i] = rows1[1 - L::ey(i)][(s * Q + i) * RW + lane + 1 - L::ex(i)];
                    }
                __syncwarp();  // every lane has read ring row j - 3 before it is overwritten
                collide_site<Q, S>(g, f1, rho1);
                collide_site<Q, S>(g, f2, rho2);
                if (do1) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) r1[(s * Q + i) * RW + lane] = f1[s][i];
                    if (lane < 2) {  // ring columns 32, 33: columns c0 + 31, c0 + 32
#pragma unroll
                        for (int s = 0; s < S; ++s)
#pragma unroll
                            for (int i = 0; i < Q; ++i) f1[s][i] = st[(s * Q + i) * G::W0 + k1 + 32 - L::ex(i)];
                        collide_site<Q, S>(g, f1, rho1);
#pragma unroll
                        for (int s = 0; s < S; ++s)
#pragma unroll
                            for (int i = 0; i < Q; ++i) r1[(s * Q + i) * RW + lane + 32] = f1[s][i];
                    }
                }
                if (do2) {
                    const int64_t x = c0 + lane;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) dst[(int64_t)(s * Q + i) * g.plane + y * g.pitch + x] = f2[s][i];
                        sum[s] += rho2[s];
                    }
                }
                __syncwarp();  // stage reads and ring writes of this row are done
                if (do1 && lane == 0) mbar_arrive(smem_u32(&empty[sk]));
            }
            if (a.mass_out) {
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] += (double)sum[s];
            }
        }
        ticket += nrows;
        if (__any_sync(kFullMask, abort_flag != 0)) break;
    }
    if (w == W && abort_flag) {  // wait (bounded) for the copies that may still be in flight
        for (int64_t tk = issued - NS > 0 ? issued - NS : 0; tk < issued; ++tk)
            mbar_wait(smem_u32(&full[tk % NS]), (unsigned)((tk / NS) & 1));
    }
    __syncthreads();
    if (abort_flag) {
        if (tid == 0 && a.status) atomicExch(a.status, LB_RD_ETIMEOUT);
        return;
    }
    if (a.mass_out) block_mass_reduce<S, (W + 1) * 32>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S, int W, int NS, int MINB>
cudaError_t launch_tbw(const StepArgs &a, cudaStream_t st) {
    constexpr int TX = 32 * W;
    using G = TbGeom<Q, S, TX>;
    if (a.nx % TX != 0) return cudaErrorInvalidValue;
    const int64_t nstrips = a.nx / TX;
    const size_t smem = ((size_t)NS * G::kStage + (size_t)W * 3 * S * Q * 34) * sizeof(float);
    auto kern = step_tbw_kernel<Q, S, W, NS, MINB, false>;
    static std::atomic<bool> configured[64] = {};  // per device ordinal (handles on several threads)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev].store(true);
    }
    const int64_t work = nstrips * a.ny / 16 > 0 ? nstrips * a.ny / 16 : 1;
    const unsigned grid = persistent_blocks(kern, (W + 1) * 32, work, smem);
    kern<<<grid, (W + 1) * 32, smem, st>>>(a, nstrips, nullptr, 0, 0);
    return cudaGetLastError();
}

// Batched form: the same kernel over the units of a list of grids.
template <int Q, int S, int W, int NS, int MINB>
cudaError_t launch_tbw_batch(const TbwItem *items, int n, int64_t total_units, cudaStream_t st) {
    constexpr int TX = 32 * W;
    using G = TbGeom<Q, S, TX>;
    const size_t smem = ((size_t)NS * G::kStage + (size_t)W * 3 * S * Q * 34) * sizeof(float);
    auto kern = step_tbw_kernel<Q, S, W, NS, MINB, true>;
    static std::atomic<bool> configured[64] = {};  // per device ordinal (handles on several threads)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev].store(true);
    }
    const int64_t work = total_units / 16 > 0 ? total_units / 16 : 1;
    const unsigned grid = persistent_blocks(kern, (W + 1) * 32, work, smem);
    kern<<<grid, (W + 1) * 32, smem, st>>>(StepArgs{}, 0, items, n, total_units);
    return cudaGetLastError();
}

template <int W, int NS, int MINB>
cudaError_t dispatch_tbw(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tbw<9, 1, W, NS, MINB>(a, st);
    if (Q == 9 && S == 2) return launch_tbw<9, 2, W, NS, MINB>(a, st);
    if (Q == 5 && S == 1) return launch_tbw<5, 1, W, NS, MINB>(a, st);
    if (Q == 5 && S == 2) return launch_tbw<5, 2, W, NS, MINB>(a, st);
    return cudaErrorInvalidValue;
}

template <int Q, int S, int NT, int TX, int NS, int MINB, int IL>
cudaError_t launch_tb(const StepArgs &a, cudaStream_t st) {
    using G = TbGeom<Q, S, TX>;
    if (a.nx % TX != 0) return cudaErrorInvalidValue;
    const int64_t nstrips = a.nx / TX;
    const size_t smem = ((size_t)NS * G::kStage + 4 * (size_t)G::kRow1) * sizeof(float);
    auto kern = step_tb2_kernel<Q, S, NT, TX, NS, MINB, IL>;
    static std::atomic<bool> configured[64] = {};  // per device ordinal (handles on several threads)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev].store(true);
    }
    // at least 16 rows per block so that the two halo rows stay a small overhead
    const int64_t work = nstrips * a.ny / 16 > 0 ? nstrips * a.ny / 16 : 1;
    const unsigned grid = persistent_blocks(kern, NT, work, smem);
    kern<<<grid, NT, smem, st>>>(a, nstrips);
    return cudaGetLastError();
}

template <int NT, int TX, int NS, int MINB, int IL = 0>
cudaError_t dispatch_tb(int Q, int S, const StepArgs &a, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tb<9, 1, NT, TX, NS, MINB, IL>(a, st);
    if (Q == 9 && S == 2) return launch_tb<9, 2, NT, TX, NS, MINB, IL>(a, st);
    if (Q == 5 && S == 1) return launch_tb<5, 1, NT, TX, NS, MINB, IL>(a, st);
    if (Q == 5 && S == 2) return launch_tb<5, 2, NT, TX, NS, MINB, IL>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace

// Batched two steps per launch (tb2w_288x256_s2x2 shape: strips of 256).
int batch_tb2_strip() { return 256; }

cudaError_t launch_batch_tb2(const TbwItem *items, int n, int64_t total_units, int Q, int S, cudaStream_t st) {
    if (Q == 9 && S == 1) return launch_tbw_batch<9, 1, 8, 2, 2>(items, n, total_units, st);
    if (Q == 9 && S == 2) return launch_tbw_batch<9, 2, 8, 2, 2>(items, n, total_units, st);
    if (Q == 5 && S == 1) return launch_tbw_batch<5, 1, 8, 2, 2>(items, n, total_units, st);
    if (Q == 5 && S == 2) return launch_tbw_batch<5, 2, 8, 2, 2>(items, n, total_units, st);
    return cudaErrorInvalidValue;
}

// Two time steps per launch (state t -> t + 2).  v: launch shape.
cudaError_t launch_step_f32_tb2(int v, int Q, int S, const StepArgs &a, cudaStream_t st) {
    // threads, strip width, stages, blocks per SM: threads ~ (2 TX + 2) / rounds
    switch (v) {
        case 0: return dispatch_tb<288, 128, 8, 1>(Q, S, a, st);
        case 1: return dispatch_tb<288, 128, 4, 2>(Q, S, a, st);
        case 2: return dispatch_tb<288, 256, 6, 1>(Q, S, a, st);
        case 3: return dispatch_tb<352, 512, 2, 1>(Q, S, a, st);
        case 4: return dispatch_tb<288, 256, 2, 2>(Q, S, a, st);
        case 5: return dispatch_tb<544, 512, 2, 1>(Q, S, a, st);
        case 6: return dispatch_tb<288, 256, 2, 2, 1>(Q, S, a, st);
        case 7: return dispatch_tb<544, 512, 2, 1, 1>(Q, S, a, st);
        case 8: return dispatch_tb<160, 128, 4, 2, 1>(Q, S, a, st);
        case 9: return dispatch_tb<288, 256, 3, 1, 1>(Q, S, a, st);
        case 10: return dispatch_tbw<8, 2, 2>(Q, S, a, st);
        case 11: return dispatch_tbw<8, 4, 1>(Q, S, a, st);
        case 12: return dispatch_tbw<4, 3, 3>(Q, S, a, st);
        case 13: return dispatch_tbw<16, 2, 1>(Q, S, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbrd
