// 16-bit deviation storage with temporal blocking to depth K: K time steps of
// Eq. relax per pass over HBM for the storage of step_half_kernel.cuh (per
// species and site the FP32 post-collision mass rho* = rho + R and the Q - 1
// deviations g_i = (1 - 1/tau)(f_i - w_i rho) rounded to bf16 or fp16).
//
// A single step stores the rounded deviations and the next step reads them
// back, so K steps give the bits of K single steps only if every level holds
// its post-collision state in that same form: rho* in FP32 and the deviations
// already rounded to 16 bits (kept as the floats they convert to).  The pull
// of the next level is then exactly the single step's:
//   f_i(x) = w_i rho*(x - e_i) + g_i(x - e_i)          (i >= 1, one FMA)
//   f_0(x) = w_0 rho*(x) - sum_{i >= 1} g_i(x)          (sum in index order)
// with the sum of a row's own deviations formed when the row is produced.
//
// Scheme of step_f32_deep_kernel.cuh (one column per lane, a warp walking a
// strip of 34 - 2K output columns down a band of rows, levels in registers):
//   * level 0 rows staged per warp by cp.async into a ring of NS rows: per
//     species rho* in 16-byte chunks of four floats and every deviation plane
//     in 8-byte chunks of four 16-bit values, the ten aligned chunks from
//     a0 = xb - 1 rounded down to a multiple of 4 (nx and the pitch are
//     multiples of 4, so no chunk straddles the periodic seam);
//   * level m > 1 pulls from level m - 1: the row of this iteration
//     (e_iy = -1), the previous row (e_iy = 0: its deviations of those
//     directions and its own-deviation sum, E0) and the one before (e_iy = +1:
//     P2), rho* of both earlier rows carried with the e_iy = +1 deviations
//     (P1 -> P2); shifts in x by warp shuffles;
//   * level K is stored: rho* as float, the deviations as 16-bit values, and
//     with `emit` rho(t + K) of level K.
// Work units, bands, the periodic wrap and the FP64 mass reduction are those
// of the FP32 depth-K kernel.  No waits but the warp's own copy groups.
#pragma once

#include "step_f32_deep_kernel.cuh"
#include "step_half_kernel.cuh"

namespace lbrd {

namespace {

__device__ __forceinline__ void cp_async8(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}

// Collision of one site in the stored form: rho_s = sum_i f_i (index order),
// R, rho*_s = rho_s + R_s and the deviations g_i rounded to 16 bits (as the
// floats they convert back to), with their sum over i >= 1 in index order.
// The arithmetic of half::tile_half; RK >= 0: the reaction kind fixed at
// compile time.
template <int Q, int S, int H, int RK = -1>
__device__ __forceinline__ void collide_half(const tb::SegArgs &g, const float (&f)[S][Q], float (&rho)[S],
                                             float (&rstar)[S], float (&gh)[S][Q], float (&gsum)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float r = f[s][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) r = rn_add(r, f[s][i]);
        rho[s] = r;
    }
    float R[S];
    reaction_f32<S, RK>(g.rkind, g.kappa, g.F, g.k, rho, R);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        rstar[s] = rn_add(rho[s], R[s]);
        const float c1 = rn_sub(1.f, g.omega[s]);
        float gs = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float hv = rn_mul(c1, rn_fma(-weight<Q, float>(i), rho[s], f[s][i]));
            gh[s][i] = half::h2f<H>(half::f2h<H>(hv));
            gs = rn_add(gs, gh[s][i]);
        }
        gsum[s] = gs;
    }
}

template <int Q, int S, int H, int K, int NW, int NS, int MINB, bool BATCH, int RK = -1>
__global__ void __launch_bounds__(NW * 32, MINB)
    step_half_deep_kernel(StepArgs a, int64_t nstrips, int64_t nbands, int64_t band,
                          const DeepItem *__restrict__ items, int nitems, int64_t total_units, int emit) {
    using L = Lattice<Q>;
    constexpr int QD = Q - 1;                 // deviation planes per species
    constexpr int CW = 40;                    // staged columns of a warp row: ten chunks of four
    constexpr int kSp = CW * 4 + QD * CW * 2; // staged bytes per species: rho* then the deviations
    constexpr int kRow = S * kSp;             // staged bytes per row
    constexpr int P = NS - 3;                 // rows staged ahead of use
    constexpr int WO = 34 - 2 * K;
    constexpr int KC = K > 1 ? K - 1 : 1;
    constexpr int NCP = S * Q;                // staged planes per row (rho* and QD deviations per species)
    static_assert(K >= 1 && K <= 8 && NS >= 4 && kSp % 16 == 0, "depth 1 .. 8, at least four staged rows");
    extern __shared__ __align__(16) unsigned char hsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *ring = hsm + (size_t)w * NS * kRow;
    const unsigned ring_s = static_cast<unsigned>(__cvta_generic_to_shared(ring));
    tb::SegArgs g;
    if (!BATCH) {
        tb::load_seg(a, g);
        if (!emit) g.rho_out = nullptr;
    }
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t units = BATCH ? total_units : nstrips * nbands;
    const int cq = lane / 10, cc = lane - 10 * cq;  // copy role: plane residue (planes cq, cq + 3, ...), chunk
    int it = 0;
    for (int64_t u = (int64_t)blockIdx.x * NW + w; u < units; u += nwarps) {
        int64_t local = u, ns = nstrips, bh = band;
        if constexpr (BATCH) {
            while (it + 1 < nitems && items[it + 1].unit_begin <= u) ++it;
            tb::load_seg(items[it].a, g);
            if (!emit) g.rho_out = nullptr;
            local = u - items[it].unit_begin;
            ns = items[it].nstrips;
            bh = items[it].band;
        }
        const unsigned char *__restrict__ src = static_cast<const unsigned char *>(g.src);
        unsigned char *__restrict__ dst = static_cast<unsigned char *>(g.dst);
        const int nx = (int)g.nx, ny = (int)g.ny;
        const int64_t plane = g.plane, pitch = g.pitch;
        const int64_t sp_bytes = plane * (4 + 2 * QD);  // one species' planes in global memory
        const int64_t b = local / ns, strip = local - b * ns;
        const int y0 = (int)(b * bh);
        const int ly = ny - y0 < (int)bh ? ny - y0 : (int)bh;
        const int xb = (int)(strip * WO) - (K - 1);  // column of lane 0
        const int a0 = (xb - 1) - (int)wrap_mod(xb - 1, 4);
        const int o = xb - 1 - a0;                   // staged column of xb - 1
        const int col = (int)wrap_mod(a0 + 4 * cc, nx);  // this lane's chunk column in global memory
        const int nrows = ly + 2 * K;
        int yl = (int)wrap_mod(y0 - K, ny);
        auto stage = [&](int j, int slot) {
            if (j < nrows && lane < 30) {
                const unsigned dslot = ring_s + (unsigned)(slot * kRow);
#pragma unroll
                for (int r = 0; r < (NCP + 2) / 3; ++r) {
                    const int p = cq + 3 * r;  // staged plane: species p / Q, plane p % Q (0: rho*)
                    if (p < NCP) {
                        const int s = p / Q, k = p - (p / Q) * Q;
                        if (k == 0) {
                            const unsigned char *gp = src + s * sp_bytes + ((int64_t)yl * pitch + col) * 4;
                            cp_async16(dslot + (unsigned)(s * kSp + cc * 16), reinterpret_cast<const float *>(gp));
                        } else {
                            const unsigned char *gp =
                                src + s * sp_bytes + plane * (4 + 2 * (k - 1)) + ((int64_t)yl * pitch + col) * 2;
                            cp_async8(dslot + (unsigned)(s * kSp + CW * 4 + (k - 1) * CW * 2 + cc * 8), gp);
                        }
                    }
                }
            }
            yl = yl + 1 == ny ? 0 : yl + 1;
            cp_async_commit();
        };
#pragma unroll
        for (int jj = 0; jj < P; ++jj) stage(jj, jj);
        // carried rows of levels 1 .. K - 1 (index m - 1 for level m):
        // P1 / P2 rho* and the e_iy = +1 deviations of the previous row and
        // of the one before, E0 the e_iy = 0 deviations and the own-deviation
        // sum of the previous row
        float P1r[KC][S], P2r[KC][S], E0s[KC][S];
        float P1g[KC][S][Q], P2g[KC][S][Q], E0g[KC][S][Q];
#pragma unroll
        for (int m = 0; m < KC; ++m)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                P1r[m][s] = P2r[m][s] = E0s[m][s] = 0.f;
#pragma unroll
                for (int i = 0; i < Q; ++i) P1g[m][s][i] = P2g[m][s][i] = E0g[m][s][i] = 0.f;
            }
        float sum[S];
#pragma unroll
        for (int s = 0; s < S; ++s) sum[s] = 0.f;
        int sl = 0;
        for (int j = 0; j < nrows; ++j) {
            stage(j + P, sl + P >= NS ? sl + P - NS : sl + P);
            cp_async_wait<P>();
            __syncwarp();
            const int s1 = sl == 0 ? NS - 1 : sl - 1, s2 = s1 == 0 ? NS - 1 : s1 - 1;
            // staged rows of iterations j - 2, j - 1, j: pulled with e_iy = +1, 0, -1
            const unsigned char *rows0[3] = {ring + s2 * kRow, ring + s1 * kRow, ring + sl * kRow};
            float f[S][Q], rho[S], rstar[S], gh[S][Q], gsum[S];
            // level 1 from the staged rows: the single step's pulls and own-deviation sum
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const unsigned char *own = rows0[1] + s * kSp;
                float gs = 0.f;
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const unsigned char *rs = rows0[1 - L::ey(i)] + s * kSp;
                    const int c = o + 1 + lane - L::ex(i);
                    const float rp = reinterpret_cast<const float *>(rs)[c];
                    const float gp = half::h2f<H>(reinterpret_cast<const unsigned short *>(rs + CW * 4 + (i - 1) * CW * 2)[c]);
                    f[s][i] = rn_fma(weight<Q, float>(i), rp, gp);
                    gs = rn_add(gs, half::h2f<H>(reinterpret_cast<const unsigned short *>(own + CW * 4 + (i - 1) * CW * 2)[o + 1 + lane]));
                }
                f[s][0] = rn_fma(weight<Q, float>(0), reinterpret_cast<const float *>(own)[o + 1 + lane], -gs);
            }
            collide_half<Q, S, H, RK>(g, f, rho, rstar, gh, gsum);
#pragma unroll
            for (int m = 1; m < K; ++m) {  // level m + 1 from level m (carried index m - 1)
                float nf[S][Q];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    // rho* of the three source rows at x - 1, x, x + 1
                    const float rr[3] = {P2r[m - 1][s], P1r[m - 1][s], rstar[s]};  // e_iy = +1, 0, -1
                    float rsh[3][3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        rsh[d][0] = __shfl_up_sync(kFullMask, rr[d], 1);    // x - 1 (e_ix = +1)
                        rsh[d][1] = rr[d];                                   // x
                        rsh[d][2] = __shfl_down_sync(kFullMask, rr[d], 1);  // x + 1 (e_ix = -1)
                    }
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const float v = L::ey(i) < 0 ? gh[s][i] : (L::ey(i) == 0 ? E0g[m - 1][s][i] : P2g[m - 1][s][i]);
                        const float gp = L::ex(i) > 0   ? __shfl_up_sync(kFullMask, v, 1)
                                         : L::ex(i) < 0 ? __shfl_down_sync(kFullMask, v, 1)
                                                        : v;
                        nf[s][i] = rn_fma(weight<Q, float>(i), rsh[1 - L::ey(i)][1 - L::ex(i)], gp);
                    }
                    nf[s][0] = rn_fma(weight<Q, float>(0), P1r[m - 1][s], -E0s[m - 1][s]);
                }
                // level m's rows move down: this row becomes the previous one
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    P2r[m - 1][s] = P1r[m - 1][s];
                    P1r[m - 1][s] = rstar[s];
                    E0s[m - 1][s] = gsum[s];
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        if (L::ey(i) > 0) {
                            P2g[m - 1][s][i] = P1g[m - 1][s][i];
                            P1g[m - 1][s][i] = gh[s][i];
                        } else if (L::ey(i) == 0) {
                            E0g[m - 1][s][i] = gh[s][i];
                        }
                    }
                }
                collide_half<Q, S, H, RK>(g, nf, rho, rstar, gh, gsum);
            }
            if (j >= 2 * K) {  // level K of row y0 + j - 2K
                const int x = xb + lane;
                if (lane >= K - 1 && lane <= 32 - K && x < nx) {
                    const int y = y0 + j - 2 * K;
                    const int64_t yx = (int64_t)y * pitch + x;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        unsigned char *base = dst + s * sp_bytes;
                        reinterpret_cast<float *>(base)[yx] = rstar[s];
                        unsigned short *gd = reinterpret_cast<unsigned short *>(base + plane * 4);
#pragma unroll
                        for (int i = 1; i < Q; ++i) gd[(int64_t)(i - 1) * plane + yx] = (unsigned short)half::f2h<H>(gh[s][i]);
                        if (g.rho_out) static_cast<float *>(g.rho_out)[s * plane + yx] = rho[s];
                        sum[s] += rho[s];
                    }
                }
            }
            __syncwarp();
            sl = sl + 1 == NS ? 0 : sl + 1;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] += (double)sum[s];
    }
    cp_async_wait<0>();
    if (a.mass_out) block_mass_reduce<S, NW * 32>(acc, a.partials, a.counter, a.mass_out);
}

template <int Q, int S, int H, int K, int NW, int NS, int MINB, bool BATCH, int RK = -1>
struct HalfDeepKernel {
    static constexpr size_t smem = (size_t)NW * NS * S * (40 * 4 + (Q - 1) * 40 * 2);
    static cudaError_t get(unsigned *full) {
        auto kern = step_half_deep_kernel<Q, S, H, K, NW, NS, MINB, BATCH, RK>;
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

template <int Q, int S, int H, int K, int NW, int NS, int MINB, int RK>
cudaError_t launch_half_deep_rk(const StepArgs &a, cudaStream_t st) {
    constexpr int WO = 34 - 2 * K;
    using HK = HalfDeepKernel<Q, S, H, K, NW, NS, MINB, false, RK>;
    unsigned full = 0;
    cudaError_t e = HK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nstrips = (a.nx + WO - 1) / WO;
    const int64_t nwarps = (int64_t)full * NW;
    const int64_t nb = choose_bands(K, nstrips, a.ny, nwarps);
    const int64_t band = (a.ny + nb - 1) / nb, nbands = (a.ny + band - 1) / band;
    const int64_t units = nstrips * nbands;
    const unsigned grid = units < nwarps ? (unsigned)((units + NW - 1) / NW) : full;
    step_half_deep_kernel<Q, S, H, K, NW, NS, MINB, false, RK>
        <<<grid, NW * 32, HK::smem, st>>>(a, nstrips, nbands, band, nullptr, 0, 0, a.rho_out != nullptr);
    return cudaGetLastError();
}

// Two-species Gray-Scott grids run the form with the reaction fixed at
// compile time; the others test the kind per site.
template <int Q, int S, int H, int K, int NW, int NS, int MINB>
cudaError_t launch_half_deep(const StepArgs &a, cudaStream_t st) {
    if (a.nx % 4 != 0 || a.pitch % 4 != 0) return cudaErrorInvalidValue;
    if constexpr (S == 2)
        if (a.rkind == kGrayScott) return launch_half_deep_rk<Q, S, H, K, NW, NS, MINB, kGrayScott>(a, st);
    return launch_half_deep_rk<Q, S, H, K, NW, NS, MINB, -1>(a, st);
}

}  // namespace
}  // namespace lbrd
