// FP32 temporal blocking to depth K: K time steps of Eq. relax per pass over
// HBM, the intermediate time levels held in registers.
//
// Each warp owns a strip of columns and walks it down a band of rows (2.5-D
// streaming); lane l holds column xb + l, xb = (first output column) - (K - 1).
//   * level 0 (the stored state f*(t)) is staged per warp: row by row, each
//     lane copies its column of every plane (lanes 0 and 1 also the two
//     columns past the warp's 32) into a ring of NS rows in shared memory with
//     cp.async, P = NS - 3 rows ahead of use (waits on the warp's own copy
//     groups: nothing to time out);
//   * level 1 (f*(t + 1)) of row r pulls from staged rows r - 1, r, r + 1
//     (shared loads at column offset -e_ix);
//   * level m > 1 pulls from level m - 1: the row that level computed in this
//     iteration (directions with e_iy = -1), the row of the previous
//     iteration (e_iy = 0) and the one before (e_iy = +1), kept in registers
//     (only the components a later pull reads), shifted in x by warp shuffles;
//   * level K is stored to HBM.
// Level m is valid on lanes m - 1 .. 32 - m (one halo column lost on each
// side per level), so a warp writes 34 - 2K columns, and from iteration 2K of
// its band on (the first 2K iterations fill the pipeline).  With `emit` set
// the launch also writes rho(t + K) = sum_i f_i,s of level K (the pre-collision
// density of Eq. relax at the new time) to the grid's density plane, 4 bytes
// per species and site: the last launch of a call leaves the density cache
// current without a separate pass.  Each level is the
// fused step of the one-step kernels (tb::collide_site): K levels give the
// bits of K single steps.  PP variants take the pulls of levels 2 .. K from
// the rows of earlier iterations (e_iy >= 0) at the start of an iteration,
// so the carried values die before the new rows are produced (fewer register
// moves; which form is faster depends on the depth and the lattice).
//
// Work units are (band, strip) pairs, strips fastest, dealt to the warps
// round-robin: consecutive warps walk adjacent strips of one band at about
// the same pace, so the 2K columns two neighbouring strips both read are
// mostly L2 (or L1) hits.  HBM moves one read and one write of the state per
// K steps, plus 2K halo rows per band.  Any nx, ny >= 1 (periodic wrap with a
// true modulo; the last strip may be ragged).
#pragma once

#include <atomic>
#include <cstdint>

#include "step_f32_tb_common.cuh"
#include "lb_rd.h"

namespace lbrd {

namespace {

using namespace tb;

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(unsigned dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ __forceinline__ int64_t wrap_mod(int64_t a, int64_t n) {
    const int64_t r = a % n;
    return r < 0 ? r + n : r;
}

// V16: level-0 rows staged in 16-byte chunks (needs nx and the row pitch to
// be multiples of 4): the warp's columns xb - 1 .. xb + 32 lie in the ten
// aligned chunks [a0, a0 + 40), a0 = xb - 1 rounded down to a multiple of 4
// (a chunk never straddles the periodic seam); lane 10 q + c (q < 3, c < 10)
// copies chunk c of planes q, q + 3, q + 6, ... (lanes 30, 31 idle).
// Otherwise 4-byte copies: lane l copies column xb - 1 + l of every plane,
// lanes 0 and 1 also columns xb + 31, xb + 32.
// BATCH: the units of a list of grids (DeepItem, sorted by unit_begin; each
// with its own strips and band height) instead of one grid.
template <int Q, int S, int K, int NW, int NS, int MINB, bool V16, bool BATCH, bool PP>
__global__ void __launch_bounds__(NW * 32, MINB)
    step_deep_kernel(StepArgs a, int64_t nstrips, int64_t nbands, int64_t band, const DeepItem *__restrict__ items,
                     int nitems, int64_t total_units, int emit) {
    using L = Lattice<Q>;
    constexpr int SQ = S * Q;
    constexpr int CW = V16 ? 40 : 34;  // staged columns of a warp row
    constexpr int kRow = SQ * CW;      // one staged row, all planes
    constexpr int P = NS - 3;          // rows staged ahead of use
    constexpr int WO = 34 - 2 * K;     // output columns per warp
    constexpr int KC = K > 1 ? K - 1 : 1;
    static_assert(K >= 1 && K <= 8 && NS >= 4, "depth 1 .. 8, at least four staged rows");
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *ring = smem + (size_t)w * NS * kRow;
    const unsigned ring_s = static_cast<unsigned>(__cvta_generic_to_shared(ring));
    SegArgs g;
    if (!BATCH) {
        load_seg(a, g);
        if (!emit) g.rho_out = nullptr;
    }
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t units = BATCH ? total_units : nstrips * nbands;
    const int cq = lane / 10, cc = lane - 10 * cq;  // V16 copy role: plane residue, chunk
    int it = 0;  // BATCH: the item of unit u (a warp's units only increase)
    for (int64_t u = (int64_t)blockIdx.x * NW + w; u < units; u += nwarps) {
        int64_t local = u, ns = nstrips, bh = band;
        if constexpr (BATCH) {
            while (it + 1 < nitems && items[it + 1].unit_begin <= u) ++it;
            load_seg(items[it].a, g);
            if (!emit) g.rho_out = nullptr;
            local = u - items[it].unit_begin;
            ns = items[it].nstrips;
            bh = items[it].band;
        }
        const float *__restrict__ src = static_cast<const float *>(g.src);
        float *__restrict__ dst = static_cast<float *>(g.dst);
        const int64_t b = local / ns, strip = local - b * ns;
        const int64_t y0 = b * bh;
        const int64_t ly = g.ny - y0 < bh ? g.ny - y0 : bh;
        const int64_t xb = strip * WO - (K - 1);  // column of lane 0
        const int64_t a0 = V16 ? (xb - 1) - wrap_mod(xb - 1, 4) : xb - 1;
        const int o = (int)(xb - 1 - a0);         // staged column of xb - 1
        // source offsets of this lane's copies (elements, row excluded)
        const int64_t offA = V16 ? (int64_t)cq * g.plane + wrap_mod(a0 + 4 * cc, g.nx) : wrap_mod(xb - 1 + lane, g.nx);
        const int64_t offB = V16 ? 0 : wrap_mod(xb + 31 + lane, g.nx);
        const int64_t nrows = ly + 2 * K;  // iterations: level-0 rows y0 - K .. y0 + ly + K - 1
        int64_t yl = wrap_mod(y0 - K, g.ny);  // next level-0 row to stage
        // stage level-0 row j into ring slot `slot`; one commit group per row (empty past the band)
        auto stage = [&](int64_t j, int slot) {
            if (j < nrows) {
                const float *row = src + yl * g.pitch;
                if constexpr (V16) {
                    if (lane < 30) {
                        const unsigned d = ring_s + (unsigned)(slot * kRow + cq * CW + 4 * cc) * 4u;
                        const float *sp = row + offA;
#pragma unroll
                        for (int r = 0; r < (SQ + 2) / 3; ++r)
                            if (cq + 3 * r < SQ) cp_async16(d + (unsigned)(3 * r * CW * 4), sp + 3 * r * g.plane);
                    }
                } else {
                    float *d = ring + slot * kRow;
#pragma unroll
                    for (int p = 0; p < SQ; ++p) {
                        cp_async4(d + p * CW + lane, row + p * g.plane + offA);
                        if (lane < 2) cp_async4(d + p * CW + 32 + lane, row + p * g.plane + offB);
                    }
                }
            }
            yl = yl + 1 == g.ny ? 0 : yl + 1;
            cp_async_commit();
        };
#pragma unroll
        for (int jj = 0; jj < P; ++jj) stage(jj, jj);
        // carried rows of levels 1 .. K - 1: E0 the previous row's e_iy = 0
        // components, P1 / P2 the e_iy = +1 components of the previous row
        // and of the one before
        float E0[KC][S][Q], P1[KC][S][Q], P2[KC][S][Q];
#pragma unroll
        for (int m = 0; m < KC; ++m)
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) E0[m][s][i] = P1[m][s][i] = P2[m][s][i] = 0.f;
        float sum[S];
#pragma unroll
        for (int s = 0; s < S; ++s) sum[s] = 0.f;
        int sl = 0;  // j % NS
        for (int64_t j = 0; j < nrows; ++j) {
            stage(j + P, sl + P >= NS ? sl + P - NS : sl + P);
            cp_async_wait<P>();  // this lane's copies of rows <= j have landed
            __syncwarp();        // ... and every other lane's
            const int s1 = sl == 0 ? NS - 1 : sl - 1, s2 = s1 == 0 ? NS - 1 : s1 - 1;
            // staged rows of iterations j - 2, j - 1, j: pulled with e_iy = +1, 0, -1
            const float *rows0[3] = {ring + s2 * kRow + o + lane + 1, ring + s1 * kRow + o + lane + 1,
                                     ring + sl * kRow + o + lane + 1};
            float f[S][Q], rho[S];
            float hp[KC][S][Q];
            if constexpr (PP) {
                // Pulls of levels 2 .. K from the rows of earlier iterations
                // (e_iy >= 0) first: the carried values then die before the new
                // rows are computed, so each level's new e_iy >= 0 components
                // can be produced in the carried registers themselves.
#pragma unroll
                for (int m = 1; m < K; ++m)
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i)
                            if (L::ey(i) >= 0) {
                                const float v = L::ey(i) == 0 ? E0[m - 1][s][i] : P2[m - 1][s][i];
                                hp[m - 1][s][i] = L::ex(i) > 0   ? __shfl_up_sync(kFullMask, v, 1)
                                                  : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v, 1)
                                                                 : v;
                                if (L::ey(i) > 0) P2[m - 1][s][i] = P1[m - 1][s][i];
                            }
            }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) f[s][i] = rows0[1 - L::ey(i)][(s * Q + i) * CW - L::ex(i)];
            collide_site<Q, S>(g, f, rho);
            if constexpr (PP) {
#pragma unroll
                for (int m = 1; m < K; ++m) {  // level m + 1 from level m (carried index m - 1)
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (L::ey(i) > 0) P1[m - 1][s][i] = f[s][i];
                            else if (L::ey(i) == 0) E0[m - 1][s][i] = f[s][i];
                            f[s][i] = L::ey(i) >= 0 ? hp[m - 1][s][i]
                                      : L::ex(i) > 0 ? __shfl_up_sync(kFullMask, f[s][i], 1)
                                      : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, f[s][i], 1)
                                                     : f[s][i];
                        }
                    collide_site<Q, S>(g, f, rho);
                }
            } else {
#pragma unroll
                for (int m = 1; m < K; ++m) {  // level m + 1 from level m (carried index m - 1)
                    float h[S][Q];
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            const float v =
                                L::ey(i) < 0 ? f[s][i] : (L::ey(i) == 0 ? E0[m - 1][s][i] : P2[m - 1][s][i]);
                            h[s][i] = L::ex(i) > 0   ? __shfl_up_sync(kFullMask, v, 1)
                                      : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v, 1)
                                                     : v;
                        }
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (L::ey(i) > 0) {
                                P2[m - 1][s][i] = P1[m - 1][s][i];
                                P1[m - 1][s][i] = f[s][i];
                            } else if (L::ey(i) == 0) {
                                E0[m - 1][s][i] = f[s][i];
                            }
                            f[s][i] = h[s][i];
                        }
                    collide_site<Q, S>(g, f, rho);
                }
            }
            if (j >= 2 * K) {  // level K of row y0 + j - 2K
                const int64_t x = xb + lane;
                if (lane >= K - 1 && lane <= 32 - K && x < g.nx) {
                    const int64_t y = y0 + j - 2 * K;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) dst[(int64_t)(s * Q + i) * g.plane + y * g.pitch + x] = f[s][i];
                        if (g.rho_out) static_cast<float *>(g.rho_out)[(int64_t)s * g.plane + y * g.pitch + x] = rho[s];
                        sum[s] += rho[s];
                    }
                }
            }
            __syncwarp();  // every lane has read slot j - 2 before iteration j + 1 stages into it
            sl = sl + 1 == NS ? 0 : sl + 1;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] += (double)sum[s];
    }
    cp_async_wait<0>();
    if (a.mass_out) block_mass_reduce<S, NW * 32>(acc, a.partials, a.counter, a.mass_out);
}

// Bands: the count nb of bands per grid whose round-robin deal of
// nb x nstrips units (ny rows each grid) to nwarps warps takes the least
// time, rounds x (rows per band + 2K pipeline-fill iterations).
int64_t choose_bands(int K, int64_t nstrips, int64_t ny, int64_t nwarps) {
    int64_t nb = 1, best = INT64_MAX;
    for (int64_t r = 1; r <= 64; ++r) {
        for (int64_t c = r * nwarps / nstrips; c <= r * nwarps / nstrips + 1; ++c) {
            const int64_t n = c < 1 ? 1 : (c > ny ? ny : c);
            const int64_t rows = (ny + n - 1) / n;
            const int64_t rounds = (n * nstrips + nwarps - 1) / nwarps;
            const int64_t cost = rounds * (rows + 2 * K);
            if (cost < best) {
                best = cost;
                nb = n;
            }
        }
    }
    return nb;
}

// Band height (rows) for a list of grids (items with nstrips and a.ny set):
// every grid is cut into bands of h rows (its last band shorter), one height
// for the whole list, so that a small grid is not cut into bands of a few
// rows that each pay the 2K pipeline-fill rows.  The height minimises the
// estimated time of the round-robin deal of the units to nwarps warps: the
// rows each warp walks on average (every band of a grid adds 2K) plus one
// unit for the last round's imbalance.
int64_t choose_band_height(int K, const DeepItem *items, int n, int64_t nwarps) {
    static const int64_t kCand[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768,
                                    1024, 1536, 2048, 3072, 4096, 6144, 8192, 16384, 32768, 65536};
    int64_t maxny = 1;
    for (int i = 0; i < n; ++i) maxny = items[i].a.ny > maxny ? items[i].a.ny : maxny;
    int64_t best_h = maxny;
    double best = 1e300;
    for (int64_t h : kCand) {
        const int64_t hh = h < maxny ? h : maxny;
        double rows = 0.0;
        for (int i = 0; i < n; ++i) {
            const int64_t nb = (items[i].a.ny + hh - 1) / hh;
            rows += (double)items[i].nstrips * (double)(items[i].a.ny + 2 * K * nb);
        }
        const double cost = rows / (double)nwarps + (double)(hh + 2 * K);
        if (cost < best) {
            best = cost;
            best_h = hh;
        }
        if (h >= maxny) break;
    }
    return best_h;
}

template <int Q, int S, int K, int NW, int NS, int MINB, bool V16, bool BATCH, bool PP = false>
struct DeepKernel {
    static constexpr size_t smem = (size_t)NW * NS * S * Q * (V16 ? 40 : 34) * sizeof(float);
    // the kernel, its shared-memory attribute set once per device, and its full persistent grid
    static cudaError_t get(unsigned *full) {
        auto kern = step_deep_kernel<Q, S, K, NW, NS, MINB, V16, BATCH, PP>;
        static std::atomic<bool> configured[64] = {};  // per device ordinal (handles on several threads)
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !configured[dev].load()) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            configured[dev].store(true);
        }
        *full = persistent_blocks(kern, NW * 32, INT64_MAX, smem);
        return cudaSuccess;
    }
};

template <int Q, int S, int K, int NW, int NS, int MINB, bool V16, bool PP>
cudaError_t launch_deep(const StepArgs &a, cudaStream_t st) {
    constexpr int WO = 34 - 2 * K;
    if (V16 && (a.nx % 4 != 0 || a.pitch % 4 != 0)) return cudaErrorInvalidValue;
    using DK = DeepKernel<Q, S, K, NW, NS, MINB, V16, false, PP>;
    unsigned full = 0;
    cudaError_t e = DK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nstrips = (a.nx + WO - 1) / WO;
    const int64_t nwarps = (int64_t)full * NW;
    const int64_t nb = choose_bands(K, nstrips, a.ny, nwarps);
    const int64_t band = (a.ny + nb - 1) / nb, nbands = (a.ny + band - 1) / band;
    const int64_t units = nstrips * nbands;
    const unsigned grid = units < nwarps ? (unsigned)((units + NW - 1) / NW) : full;
    step_deep_kernel<Q, S, K, NW, NS, MINB, V16, false, PP>
        <<<grid, NW * 32, DK::smem, st>>>(a, nstrips, nbands, band, nullptr, 0, 0, a.rho_out != nullptr);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbrd
