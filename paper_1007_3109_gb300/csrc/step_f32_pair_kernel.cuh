// FP32 temporal blocking to depth K with two columns per lane: the depth-K
// scheme of step_f32_deep_kernel.cuh (K time steps of Eq. relax per pass over
// HBM, intermediate levels in registers, a warp walking a strip of columns
// down a band of rows) on a 64-column warp window.
//
// Lane l holds the adjacent columns xb + 2l and xb + 2l + 1.  A pull from the
// left neighbour (e_ix = +1) takes the lane's own first column for its second
// one and the second column of lane l - 1 (a warp shuffle) for its first one;
// e_ix = -1 mirrors it.  So a level costs one shuffle per shifted direction
// for two sites, and each level loses one column per side of a 64-column
// window instead of a 32-column one: with the left halo HL (K rounded up to
// an even count) a warp writes 64 - 2 HL columns, e.g. 56 of 64 at K = 4
// against 26 of 32 for one column per lane.  The price is twice the carried
// registers per level, which bounds K.
//
//   * level 0 (f*(t)): rows staged per warp by cp.async in 16-byte chunks
//     (the row pitch is a multiple of 32): the window's 64 columns start at
//     xb (even), inside the 17 aligned chunks from a0 = xb rounded down to a
//     multiple of 4; lanes 0-15 copy chunk `lane` of the even planes, lanes
//     16-31 chunk `lane - 16` of the odd planes, lane p < S Q chunk 16 of
//     plane p.  nx a multiple of 4: no chunk straddles the periodic seam.
//     The ANY form takes any nx: a chunk that reaches past the seam (edge
//     strips only) is copied column by column with wrapped indices; kept
//     apart because the extra paths slow the loop body down even where they
//     never run.  Waits only on the warp's own copy groups.
//   * level 1 pulls the lane's column pair of every plane from the staged row
//     of its e_iy (one 8-byte shared load) and shifts it like the levels
//     above; level m > 1 pulls from level m - 1 carried in registers (the row
//     of this iteration for e_iy = -1, the previous one for e_iy = 0, the one
//     before for e_iy = +1), exactly as the one-column kernel.
//   * level 1 is valid on window columns 1 .. 62 and level m on m .. 63 - m;
//     level K is stored for columns HL .. 63 - HL (8-byte stores; the last
//     column of an odd nx alone in the ANY form), and with `emit` rho(t + K)
//     of level K too.
// Each level collides the lane's two columns together (tb::collide_pair: the
// operations of tb::collide_site per column, one test of the reaction kind
// for both, or none with the kind fixed at compile time): K levels give the
// bits of K single steps.  Units, bands, the periodic wrap and the FP64 mass
// reduction are those of the one-column kernel.
#pragma once

#include "step_f32_deep_kernel.cuh"

namespace lbrd {

namespace {

// Periodic wrap of a column index in 32-bit arithmetic (inlined, unlike a
// 64-bit remainder, which would put a call into the row loop).
__device__ __forceinline__ int wrap32(int a, int n) {
    const int r = a % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async4s(unsigned dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}

// Volatile shared-memory loads: a list's grid parameters are read from the
// warp's shared copy where they are used (never hoisted into registers).
__device__ __forceinline__ unsigned long long lds_v64(const void *p) {
    unsigned long long v;
    asm volatile("ld.volatile.shared.u64 %0, [%1];\n" : "=l"(v) : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
    return v;
}
__device__ __forceinline__ unsigned lds_v32(const void *p) {
    unsigned v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
    return v;
}

template <int K>
struct PairGeom {
    static constexpr int HL = (K + 1) / 2 * 2;  // left (and right) halo columns of the window, even
    static constexpr int WO = 64 - 2 * HL;      // output columns per warp, even
};

// ANY: grids of any nx (the seam chunks copied column by column, the last
// column of an odd nx stored alone); otherwise nx must be a multiple of 4.
// RK >= 0: the grid's reaction kind, fixed at compile time.  EA: a row is
// staged as soon as level 1 has read the oldest staged row, whose slot it
// takes: NS - 2 rows in flight instead of NS - 3, in the same ring.
template <int Q, int S, int K, int NW, int NS, int MINB, bool BATCH, bool PP, bool ANY = false, int RK = -1,
          bool EA = false>
__global__ void __launch_bounds__(NW * 32, MINB)
    step_pair_kernel(StepArgs a, int64_t nstrips, int64_t nbands, int64_t band, const DeepItem *__restrict__ items,
                     int nitems, int64_t total_units, int emit) {
    using L = Lattice<Q>;
    constexpr int SQ = S * Q;
    constexpr int CW = 68;          // staged columns of a warp row: 17 chunks of four
    constexpr int kRow = SQ * CW;   // one staged row, all planes
    constexpr int P = EA ? NS - 2 : NS - 3;  // rows staged ahead of use
    constexpr int HL = PairGeom<K>::HL;
    constexpr int WO = PairGeom<K>::WO;
    constexpr int KC = K > 1 ? K - 1 : 1;
    static_assert(K >= 1 && K <= 8 && NS >= 4 && WO > 0, "depth 1 .. 8, at least four staged rows");
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *ring = smem + (size_t)w * NS * kRow;
    const unsigned ring_s = static_cast<unsigned>(__cvta_generic_to_shared(ring));
    SegArgs g;
    if (!BATCH) {
        load_seg(a, g);
        if (!emit) g.rho_out = nullptr;
    }
    // BATCH: the unit's grid parameters, one copy per warp, read where they
    // are used so that they hold no registers across the row loop (a single
    // grid reads them from the kernel's parameter space)
    __shared__ SegArgs seg_sh[BATCH ? NW : 1];
    SegArgs &gs = seg_sh[BATCH ? w : 0];
    auto p_src = [&]() -> const float * {
        if constexpr (BATCH) return reinterpret_cast<const float *>(lds_v64(&gs.src));
        else return static_cast<const float *>(a.src);
    };
    auto p_dst = [&]() -> float * {
        if constexpr (BATCH) return reinterpret_cast<float *>(lds_v64(&gs.dst));
        else return static_cast<float *>(a.dst);
    };
    auto p_rho = [&]() -> float * {
        if constexpr (BATCH) return reinterpret_cast<float *>(lds_v64(&gs.rho_out));
        else return emit ? static_cast<float *>(a.rho_out) : nullptr;
    };
    auto p_pitch = [&]() -> int64_t {
        if constexpr (BATCH) return (int64_t)lds_v64(&gs.pitch);
        else return a.pitch;
    };
    auto p_plane = [&]() -> int64_t {
        if constexpr (BATCH) return (int64_t)lds_v64(&gs.plane);
        else return a.plane;
    };
    // relaxation and reaction constants of the collisions
    auto p_coll = [&]() -> SegArgs {
        if constexpr (BATCH) {
            SegArgs c;
            c.omega[0] = __uint_as_float(lds_v32(&gs.omega[0]));
            c.omega[1] = __uint_as_float(lds_v32(&gs.omega[1]));
            c.rkind = (int)lds_v32(&gs.rkind);
            c.kappa = __uint_as_float(lds_v32(&gs.kappa));
            c.F = __uint_as_float(lds_v32(&gs.F));
            c.k = __uint_as_float(lds_v32(&gs.k));
            return c;
        } else {
            return g;
        }
    };
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t units = BATCH ? total_units : nstrips * nbands;
    const int cch = lane & 15, cpar = lane >> 4;  // copy role: chunk, plane parity
    int it = 0;
    for (int64_t u = (int64_t)blockIdx.x * NW + w; u < units; u += nwarps) {
        int64_t local = u, ns = nstrips, bh = band;
        if constexpr (BATCH) {
            while (it + 1 < nitems && items[it + 1].unit_begin <= u) ++it;
            load_seg(items[it].a, g);
            if (!emit) g.rho_out = nullptr;
            local = u - items[it].unit_begin;
            ns = items[it].nstrips;
            bh = items[it].band;
            __syncwarp();  // the previous unit's reads of gs are done
            if (lane == 0) gs = g;
            __syncwarp();
        }
        // rows and columns fit 32 bits (sides <= 65535); plane offsets need 64
        const int nx = (int)g.nx, ny = (int)g.ny;
        const int64_t b = local / ns, strip = local - b * ns;
        const int y0 = (int)(b * bh);
        const int ly = ny - y0 < (int)bh ? ny - y0 : (int)bh;
        const int xb = (int)(strip * WO) - HL;  // first window column (even)
        const int a0 = xb - (int)wrap_mod(xb, 4);  // first staged column
        const int o = xb - a0;                     // staged column of xb: 0 or 2
        // this lane's chunks start at columns cA and cB; a chunk that reaches past the
        // periodic seam (edge strips only, nx not a multiple of 4) is copied column by
        // column with wrapped indices, the others in one 16-byte copy
        const int cA = a0 + 4 * cch, cB = a0 + 64;
        const bool cleanA = !ANY || (cA >= 0 && cA + 4 <= nx), cleanB = !ANY || (cB >= 0 && cB + 4 <= nx);
        const int64_t offA = (int64_t)cpar * g.plane + (ANY ? (cleanA ? cA : 0) : wrap_mod(cA, nx));
        const int64_t offB = (int64_t)(lane < SQ ? lane : 0) * g.plane + (ANY ? (cleanB ? cB : 0) : wrap_mod(cB, nx));
        const int nrows = ly + 2 * K;
        int yl = (int)wrap_mod(y0 - K, ny);
        auto stage = [&](int j, int slot) {
            if (j < nrows) {
                const float *row = p_src() + (int64_t)yl * p_pitch();
                const unsigned d = ring_s + (unsigned)(slot * kRow + cpar * CW + 4 * cch) * 4u;
                const float *sp = row + offA;
                int64_t pl2 = 2 * p_plane();
                asm volatile("" : "+l"(pl2));  // no plane multiples kept live across the row loop
                if (!ANY || cleanA) {
#pragma unroll
                    for (int r = 0; r < (SQ + 1) / 2; ++r)
                        if (cpar + 2 * r < SQ) cp_async16(d + (unsigned)(2 * r * CW * 4), sp + r * pl2);
                } else if constexpr (ANY) {
                    for (int r = 0; r < (SQ + 1) / 2; ++r)
                        if (cpar + 2 * r < SQ)
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                cp_async4s(d + (unsigned)((2 * r * CW + e) * 4), sp + r * pl2 + wrap32(cA + e, nx));
                }
                if (lane < SQ) {
                    const unsigned db = ring_s + (unsigned)(slot * kRow + lane * CW + 64) * 4u;
                    if (!ANY || cleanB) {
                        cp_async16(db, row + offB);
                    } else if constexpr (ANY) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) cp_async4s(db + 4u * e, row + offB + wrap32(cB + e, nx));
                    }
                }
            }
            yl = yl + 1 == ny ? 0 : yl + 1;
            cp_async_commit();
        };
#pragma unroll
        for (int jj = 0; jj < P; ++jj) stage(jj, jj);
        // carried levels 1 .. K - 1, both columns: E0 the previous row's
        // e_iy = 0 components, P1 / P2 the e_iy = +1 components of the
        // previous row and of the one before
        float E0[KC][2][S][Q], P1[KC][2][S][Q], P2[KC][2][S][Q];
#pragma unroll
        for (int m = 0; m < KC; ++m)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int i = 0; i < Q; ++i) E0[m][c][s][i] = P1[m][c][s][i] = P2[m][c][s][i] = 0.f;
        float sum[S];
#pragma unroll
        for (int s = 0; s < S; ++s) sum[s] = 0.f;
        int sl = 0;
        for (int j = 0; j < nrows; ++j) {
            if constexpr (!EA) stage(j + P, sl + P >= NS ? sl + P - NS : sl + P);
            cp_async_wait<EA ? P - 1 : P>();  // this lane's copies of row j have landed
            __syncwarp();
            const int s1 = sl == 0 ? NS - 1 : sl - 1, s2 = s1 == 0 ? NS - 1 : s1 - 1;
            // staged rows of iterations j - 2, j - 1, j: pulled with e_iy = +1, 0, -1
            const float *rows0[3] = {ring + s2 * kRow + o + 2 * lane, ring + s1 * kRow + o + 2 * lane,
                                     ring + sl * kRow + o + 2 * lane};
            float f0[S][Q], f1[S][Q], rho0[S], rho1[S];
            float hp0[KC][S][Q], hp1[KC][S][Q];
            if constexpr (PP) {
#pragma unroll
                for (int m = 1; m < K; ++m)
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i)
                            if (L::ey(i) >= 0) {
                                const float v0 = L::ey(i) == 0 ? E0[m - 1][0][s][i] : P2[m - 1][0][s][i];
                                const float v1 = L::ey(i) == 0 ? E0[m - 1][1][s][i] : P2[m - 1][1][s][i];
                                hp0[m - 1][s][i] = L::ex(i) > 0   ? __shfl_up_sync(kFullMask, v1, 1)
                                                   : L::ex(i) < 0 ? v1
                                                                  : v0;
                                hp1[m - 1][s][i] = L::ex(i) > 0   ? v0
                                                   : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v0, 1)
                                                                  : v1;
                                if (L::ey(i) > 0) {
                                    P2[m - 1][0][s][i] = P1[m - 1][0][s][i];
                                    P2[m - 1][1][s][i] = P1[m - 1][1][s][i];
                                }
                            }
            }
            // level 1 from the staged rows
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float2 v = *reinterpret_cast<const float2 *>(rows0[1 - L::ey(i)] + (s * Q + i) * CW);
                    f0[s][i] = L::ex(i) > 0 ? __shfl_up_sync(kFullMask, v.y, 1) : (L::ex(i) < 0 ? v.y : v.x);
                    f1[s][i] = L::ex(i) > 0 ? v.x : (L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v.x, 1) : v.y);
                }
            if constexpr (EA) {  // every lane has read row j - 2: its slot takes row j + P
                __syncwarp();
                stage(j + P, sl + P >= NS ? sl + P - NS : sl + P);
            }
            {
                const SegArgs cg = p_coll();
                collide_pair<Q, S, RK>(cg, f0, f1, rho0, rho1);
            }
#pragma unroll
            for (int m = 1; m < K; ++m) {  // level m + 1 from level m (carried index m - 1)
                if constexpr (PP) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (L::ey(i) > 0) {
                                P1[m - 1][0][s][i] = f0[s][i];
                                P1[m - 1][1][s][i] = f1[s][i];
                            } else if (L::ey(i) == 0) {
                                E0[m - 1][0][s][i] = f0[s][i];
                                E0[m - 1][1][s][i] = f1[s][i];
                            }
                            const float v0 = f0[s][i], v1 = f1[s][i];
                            f0[s][i] = L::ey(i) >= 0 ? hp0[m - 1][s][i]
                                       : L::ex(i) > 0 ? __shfl_up_sync(kFullMask, v1, 1)
                                       : L::ex(i) < 0 ? v1
                                                      : v0;
                            f1[s][i] = L::ey(i) >= 0 ? hp1[m - 1][s][i]
                                       : L::ex(i) > 0 ? v0
                                       : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v0, 1)
                                                      : v1;
                        }
                } else {
                    float h0[S][Q], h1[S][Q];
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            const float v0 = L::ey(i) < 0    ? f0[s][i]
                                             : L::ey(i) == 0 ? E0[m - 1][0][s][i]
                                                             : P2[m - 1][0][s][i];
                            const float v1 = L::ey(i) < 0    ? f1[s][i]
                                             : L::ey(i) == 0 ? E0[m - 1][1][s][i]
                                                             : P2[m - 1][1][s][i];
                            h0[s][i] = L::ex(i) > 0 ? __shfl_up_sync(kFullMask, v1, 1) : (L::ex(i) < 0 ? v1 : v0);
                            h1[s][i] = L::ex(i) > 0 ? v0 : (L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v0, 1) : v1);
                        }
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (L::ey(i) > 0) {
                                P2[m - 1][0][s][i] = P1[m - 1][0][s][i];
                                P2[m - 1][1][s][i] = P1[m - 1][1][s][i];
                                P1[m - 1][0][s][i] = f0[s][i];
                                P1[m - 1][1][s][i] = f1[s][i];
                            } else if (L::ey(i) == 0) {
                                E0[m - 1][0][s][i] = f0[s][i];
                                E0[m - 1][1][s][i] = f1[s][i];
                            }
                            f0[s][i] = h0[s][i];
                            f1[s][i] = h1[s][i];
                        }
                }
                const SegArgs cg = p_coll();
                collide_pair<Q, S, RK>(cg, f0, f1, rho0, rho1);
            }
            if (j >= 2 * K) {  // level K of row y0 + j - 2K: window columns HL .. 63 - HL
                const int x = xb + 2 * lane;
                if (lane >= HL / 2 && lane < (HL + WO) / 2 && x < nx) {
                    const int y = y0 + j - 2 * K;
                    int64_t pl = p_plane();
                    asm volatile("" : "+l"(pl));  // no plane multiples kept live across the row loop
                    const int64_t yx = (int64_t)y * p_pitch() + x;
                    float *dp = p_dst() + yx;
                    float *rp = p_rho();
                    if (!ANY || x + 1 < nx) {  // both columns (x is even: 8-byte stores)
#pragma unroll
                        for (int s = 0; s < S; ++s) {
#pragma unroll
                            for (int i = 0; i < Q; ++i)
                                *reinterpret_cast<float2 *>(dp + (s * Q + i) * pl) = make_float2(f0[s][i], f1[s][i]);
                            if (rp) *reinterpret_cast<float2 *>(rp + s * pl + yx) = make_float2(rho0[s], rho1[s]);
                            sum[s] += rho0[s] + rho1[s];
                        }
                    } else if constexpr (ANY) {  // the last column of an odd nx
#pragma unroll
                        for (int s = 0; s < S; ++s) {
#pragma unroll
                            for (int i = 0; i < Q; ++i) dp[(s * Q + i) * pl] = f0[s][i];
                            if (rp) rp[s * pl + yx] = rho0[s];
                            sum[s] += rho0[s];
                        }
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

template <int Q, int S, int K, int NW, int NS, int MINB, bool BATCH, bool PP = false, bool ANY = false, int RK = -1,
          bool EA = false>
struct PairKernel {
    static constexpr size_t smem = (size_t)NW * NS * S * Q * 68 * sizeof(float);
    static cudaError_t get(unsigned *full) {
        auto kern = step_pair_kernel<Q, S, K, NW, NS, MINB, BATCH, PP, ANY, RK, EA>;
        static std::atomic<bool> configured[64] = {};
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

template <int Q, int S, int K, int NW, int NS, int MINB, bool PP, bool ANY, int RK, bool EA>
cudaError_t launch_pair_rk(const StepArgs &a, cudaStream_t st) {
    constexpr int WO = PairGeom<K>::WO;
    using PK = PairKernel<Q, S, K, NW, NS, MINB, false, PP, ANY, RK, EA>;
    unsigned full = 0;
    cudaError_t e = PK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nstrips = (a.nx + WO - 1) / WO;
    const int64_t nwarps = (int64_t)full * NW;
    const int64_t nb = choose_bands(K, nstrips, a.ny, nwarps);
    const int64_t band = (a.ny + nb - 1) / nb, nbands = (a.ny + band - 1) / band;
    const int64_t units = nstrips * nbands;
    const unsigned grid = units < nwarps ? (unsigned)((units + NW - 1) / NW) : full;
    step_pair_kernel<Q, S, K, NW, NS, MINB, false, PP, ANY, RK, EA>
        <<<grid, NW * 32, PK::smem, st>>>(a, nstrips, nbands, band, nullptr, 0, 0, a.rho_out != nullptr);
    return cudaGetLastError();
}

// Two-species Gray-Scott grids run the form with the reaction fixed at
// compile time (no test of the kind in the row loop); the others test it.
template <int Q, int S, int K, int NW, int NS, int MINB, bool PP, bool ANY = false, bool EA = false>
cudaError_t launch_pair(const StepArgs &a, cudaStream_t st) {
    if ((!ANY && a.nx % 4 != 0) || a.pitch % 4 != 0) return cudaErrorInvalidValue;
    if constexpr (S == 2)
        if (a.rkind == kGrayScott) return launch_pair_rk<Q, S, K, NW, NS, MINB, PP, ANY, kGrayScott, EA>(a, st);
    return launch_pair_rk<Q, S, K, NW, NS, MINB, PP, ANY, -1, EA>(a, st);
}

}  // namespace
}  // namespace lbrd
