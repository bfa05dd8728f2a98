// 16-bit deviation storage with temporal blocking to depth K, two columns per
// lane: the scheme of step_half_deep_kernel.cuh (K time steps of Eq. relax per
// pass over HBM, every level holding rho* in FP32 and the deviations rounded
// to 16 bits as a single step stores them, so that K levels give the bits of
// K single steps) on the 64-column warp window of step_f32_pair_kernel.cuh:
// lane l holds the adjacent columns xb + 2l and xb + 2l + 1, a pull shifted
// in x takes one warp shuffle for the two sites, and with HL = K rounded up
// to an even count a warp writes 64 - 2 HL columns.
//
//   * The two columns' deviations of a plane are rounded by one paired
//     conversion (the bits of two single ones) and kept packed, one 32-bit
//     word per plane: the carried rows hold half the registers of floats, a
//     shift moves both columns' values with one shuffle, and level K stores a
//     plane's pair with one 4-byte store.
//   * Level 0 rows are staged per warp by 16-byte cp.async: per species rho*
//     for the 72 columns from a0 (xb rounded down to a multiple of 8) and
//     each deviation plane for the same columns (nine chunks of eight 16-bit
//     values).  nx is a multiple of 8, so no chunk straddles the periodic
//     seam.  Lanes 0-17 copy the rho* chunks, lanes 0-26 the deviation chunks
//     (chunk lane % 9 of the planes lane / 9, lane / 9 + 3, ...).
//   * Level 1 is valid on window columns 1 .. 62 and level m on m .. 63 - m
//     (a lane's outer neighbours come by shuffle; the window's own edges have
//     none); level K is stored for columns HL .. 63 - HL.
//   * Level 1 reads each lane's column pair from the staged rows (an 8-byte
//     load of rho*, a 4-byte load of a deviation plane) and sums the middle
//     row's own deviations for f_0; level m > 1 pulls from level m - 1 in
//     registers: the row of this iteration (e_iy = -1), the previous row
//     (e_iy = 0: its deviations and own-deviation sum, E0) and the one before
//     (e_iy = +1), rho* of both earlier rows carried with them.
// Work units, bands, the periodic wrap and the FP64 mass reduction are those
// of the FP32 depth-K kernels.  No waits but the warp's own copy groups.
#pragma once

#include "step_f32_pair_kernel.cuh"
#include "step_half_deep_kernel.cuh"

namespace lbrd {

namespace {

// The two halves of a packed pair as the floats they convert to.
template <int H>
__device__ __forceinline__ float lo16(unsigned w) {
    return half::h2f<H>(w);
}
template <int H>
__device__ __forceinline__ float hi16(unsigned w) {
    return half::h2f<H>(w >> 16);
}

// f = fma(w, rho*, g) of the lane's two sites: one packed FP32x2
// instruction (PK) or two scalar ones, the same bits.
template <bool PK>
__device__ __forceinline__ void pull_pair(float w, float r0, float r1, float g0, float g1, float &f0, float &f1) {
    if constexpr (PK) {
        const float2 v = rn_fma2(pair2(w), make_float2(r0, r1), make_float2(g0, g1));
        f0 = v.x;
        f1 = v.y;
    } else {
        f0 = rn_fma(w, r0, g0);
        f1 = rn_fma(w, r1, g1);
    }
}

// Collision of the lane's two sites in the stored form (collide_half's
// operations per site): rho_s = sum_i f_i (index order), R, rho*_s = rho_s +
// R_s, the deviations g_i = (1 - omega) fma(-w_i, rho, f_i) rounded to 16 bits
// (both columns in one paired conversion, kept packed in gp) and their sum
// over i >= 1 in index order.  PK: the two sites' operands packed in pairs
// (FP32x2 instructions, each component rounded as the scalar operation, half
// the issue slots; the constant pairs take registers, so it is the form of
// the launch bounds that leave room for them).  RK >= 0: the reaction kind
// fixed at compile time.
template <int Q, int S, int H, int RK, bool PK>
__device__ __forceinline__ void collide_half_pair(const tb::SegArgs &g, const float (&f0)[S][Q],
                                                  const float (&f1)[S][Q], float (&rho0)[S], float (&rho1)[S],
                                                  float (&rs0)[S], float (&rs1)[S], unsigned (&gp)[S][Q],
                                                  float (&gs0)[S], float (&gs1)[S]) {
    if constexpr (PK) {
        float2 r[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            r[s] = make_float2(f0[s][0], f1[s][0]);
#pragma unroll
            for (int i = 1; i < Q; ++i) r[s] = rn_add2(r[s], make_float2(f0[s][i], f1[s][i]));
            rho0[s] = r[s].x;
            rho1[s] = r[s].y;
        }
        float R0[S], R1[S];
        reaction2_f32<S, RK>(g.rkind, g.kappa, g.F, g.k, rho0, rho1, R0, R1);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float2 rs = rn_add2(r[s], make_float2(R0[s], R1[s]));
            rs0[s] = rs.x;
            rs1[s] = rs.y;
            const float2 c1 = pair2(rn_sub(1.f, g.omega[s]));
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float2 d =
                    rn_mul2(c1, rn_fma2(pair2(-weight<Q, float>(i)), r[s], make_float2(f0[s][i], f1[s][i])));
                const unsigned p = half::f2h2<H>(d.x, d.y);
                gp[s][i] = p;
                acc = rn_add2(acc, make_float2(lo16<H>(p), hi16<H>(p)));
            }
            gs0[s] = acc.x;
            gs1[s] = acc.y;
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float r0 = f0[s][0], r1 = f1[s][0];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                r0 = rn_add(r0, f0[s][i]);
                r1 = rn_add(r1, f1[s][i]);
            }
            rho0[s] = r0;
            rho1[s] = r1;
        }
        float R0[S], R1[S];
        reaction2_f32<S, RK>(g.rkind, g.kappa, g.F, g.k, rho0, rho1, R0, R1);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            rs0[s] = rn_add(rho0[s], R0[s]);
            rs1[s] = rn_add(rho1[s], R1[s]);
            const float c1 = rn_sub(1.f, g.omega[s]);
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float w = weight<Q, float>(i);
                const unsigned p = half::f2h2<H>(rn_mul(c1, rn_fma(-w, rho0[s], f0[s][i])),
                                                 rn_mul(c1, rn_fma(-w, rho1[s], f1[s][i])));
                gp[s][i] = p;
                a0 = rn_add(a0, lo16<H>(p));
                a1 = rn_add(a1, hi16<H>(p));
            }
            gs0[s] = a0;
            gs1[s] = a1;
        }
    }
}

template <int K>
using HalfPairGeom = PairGeom<K>;

template <int Q, int S, int H, int K, int NW, int NS, int MINB, bool BATCH, int RK = -1>
__global__ void __launch_bounds__(NW * 32, MINB)
    step_half_pair_kernel(StepArgs a, int64_t nstrips, int64_t nbands, int64_t band,
                          const DeepItem *__restrict__ items, int nitems, int64_t total_units, int emit) {
    using L = Lattice<Q>;
    constexpr int QD = Q - 1;                  // deviation planes per species
    constexpr int CW = 72;                     // staged columns of a warp row
    constexpr int kSp = CW * 4 + QD * CW * 2;  // staged bytes per species: rho* then the deviations
    constexpr int kRow = S * kSp;              // staged bytes per row
    constexpr int NDP = S * QD;                // deviation planes of all species
    constexpr int P = NS - 3;                  // rows staged ahead of use
    constexpr int HL = HalfPairGeom<K>::HL;
    constexpr int WO = HalfPairGeom<K>::WO;
    constexpr int KC = K > 1 ? K - 1 : 1;
    constexpr bool PK = MINB <= 2;  // packed pairs where the launch bounds allow 255 registers
    static_assert(K >= 1 && K <= 8 && NS >= 4 && WO > 0 && kSp % 16 == 0, "depth 1 .. 8, four staged rows");
    extern __shared__ __align__(16) unsigned char hps[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *ring = hps + (size_t)w * NS * kRow;
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
    const int cq = lane / 9, cc = lane - 9 * (lane / 9);  // deviation copies: planes cq, cq + 3, ..., chunk cc
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
        // rows and columns fit 32 bits (sides <= 65535); plane offsets need 64
        const int nx = (int)g.nx, ny = (int)g.ny;
        const int64_t plane = g.plane, pitch = g.pitch;
        const int64_t sp_bytes = plane * (4 + 2 * QD);  // one species' planes in global memory
        const int64_t b = local / ns, strip = local - b * ns;
        const int y0 = (int)(b * bh);
        const int ly = ny - y0 < (int)bh ? ny - y0 : (int)bh;
        const int xb = (int)(strip * WO) - HL;             // first window column (even)
        const int a0 = xb - (int)wrap_mod(xb, 8);  // first staged column (a multiple of 8)
        const int t0 = xb - a0 + 2 * lane;         // staged column of this lane's first column (even)
        const int colr = wrap32(a0 + 4 * (lane < 18 ? lane : 0), nx);  // rho* chunk column
        const int cold = wrap32(a0 + 8 * cc, nx);                      // deviation chunk column
        const int nrows = ly + 2 * K;
        int yl = (int)wrap_mod(y0 - K, ny);
        auto stage = [&](int j, int slot) {
            if (j < nrows) {
                const unsigned dslot = ring_s + (unsigned)(slot * kRow);
                const int64_t yrow = (int64_t)yl * pitch;
                if (lane < 18) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        cp_async16(dslot + (unsigned)(s * kSp + 16 * lane),
                                   reinterpret_cast<const float *>(src + s * sp_bytes + (yrow + colr) * 4));
                }
                if (lane < 27) {
#pragma unroll
                    for (int r = 0; r < (NDP + 2) / 3; ++r) {
                        const int pd = cq + 3 * r;  // deviation plane over all species: species pd / QD
                        if (pd < NDP) {
                            const int s = pd / QD, p = pd - (pd / QD) * QD;
                            const int64_t off = plane * (int64_t)(s * (4 + 2 * QD) + 4 + 2 * p) + (yrow + cold) * 2;
                            cp_async16(dslot + (unsigned)(s * kSp + CW * 4 + p * CW * 2 + 16 * cc),
                                       reinterpret_cast<const float *>(src + off));
                        }
                    }
                }
            }
            yl = yl + 1 == ny ? 0 : yl + 1;
            cp_async_commit();
        };
#pragma unroll
        for (int jj = 0; jj < P; ++jj) stage(jj, jj);
        // carried rows of levels 1 .. K - 1 (index m - 1 for level m), both
        // columns: rho* of the previous row and of the one before (P1r / P2r),
        // the previous row's own-deviation sums (E0s); the packed deviations
        // of the e_iy = +1 directions of those two rows (P1g / P2g) and of the
        // e_iy = 0 directions of the previous row (E0g)
        float P1r[KC][2][S], P2r[KC][2][S], E0s[KC][2][S];
        unsigned P1g[KC][S][Q], P2g[KC][S][Q], E0g[KC][S][Q];
#pragma unroll
        for (int m = 0; m < KC; ++m)
#pragma unroll
            for (int s = 0; s < S; ++s) {
#pragma unroll
                for (int c = 0; c < 2; ++c) P1r[m][c][s] = P2r[m][c][s] = E0s[m][c][s] = 0.f;
#pragma unroll
                for (int i = 0; i < Q; ++i) P1g[m][s][i] = P2g[m][s][i] = E0g[m][s][i] = 0u;
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
            float f0[S][Q], f1[S][Q], rho0[S], rho1[S], rs0[S], rs1[S], gs0[S], gs1[S];
            unsigned gp[S][Q];
            // level 1 from the staged rows: the single step's pulls and the middle
            // row's own-deviation sums
#pragma unroll
            for (int s = 0; s < S; ++s) {
                float rsh[3][2][3];  // rho* of row d at columns x - 1, x, x + 1 of column c
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float2 v = *reinterpret_cast<const float2 *>(rows0[d] + s * kSp + 4 * t0);
                    const float l = __shfl_up_sync(kFullMask, v.y, 1), r = __shfl_down_sync(kFullMask, v.x, 1);
                    rsh[d][0][0] = l;
                    rsh[d][0][1] = v.x;
                    rsh[d][0][2] = v.y;
                    rsh[d][1][0] = v.x;
                    rsh[d][1][1] = v.y;
                    rsh[d][1][2] = r;
                }
                float2 own = make_float2(0.f, 0.f);  // the middle row's own-deviation sums
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int dv = s * kSp + CW * 4 + (i - 1) * CW * 2 + 2 * t0;  // the lane's pair of plane i
                    const unsigned wsrc = *reinterpret_cast<const unsigned *>(rows0[1 - L::ey(i)] + dv);
                    const unsigned wown = L::ey(i) == 0 ? wsrc : *reinterpret_cast<const unsigned *>(rows0[1] + dv);
                    float g0, g1;
                    if (L::ex(i) > 0) {
                        g0 = hi16<H>(__shfl_up_sync(kFullMask, wsrc, 1));
                        g1 = lo16<H>(wsrc);
                    } else if (L::ex(i) < 0) {
                        g0 = hi16<H>(wsrc);
                        g1 = lo16<H>(__shfl_down_sync(kFullMask, wsrc, 1));
                    } else {
                        g0 = lo16<H>(wsrc);
                        g1 = hi16<H>(wsrc);
                    }
                    pull_pair<PK>(weight<Q, float>(i), rsh[1 - L::ey(i)][0][1 - L::ex(i)],
                                  rsh[1 - L::ey(i)][1][1 - L::ex(i)], g0, g1, f0[s][i], f1[s][i]);
                    if constexpr (PK) {
                        own = rn_add2(own, make_float2(lo16<H>(wown), hi16<H>(wown)));
                    } else {
                        own.x = rn_add(own.x, lo16<H>(wown));
                        own.y = rn_add(own.y, hi16<H>(wown));
                    }
                }
                f0[s][0] = rn_fma(weight<Q, float>(0), rsh[1][0][1], -own.x);
                f1[s][0] = rn_fma(weight<Q, float>(0), rsh[1][1][1], -own.y);
            }
            collide_half_pair<Q, S, H, RK, PK>(g, f0, f1, rho0, rho1, rs0, rs1, gp, gs0, gs1);
#pragma unroll
            for (int m = 1; m < K; ++m) {  // level m + 1 from level m (carried index m - 1)
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    // rho* of the three source rows (e_iy = +1, 0, -1) at x - 1, x, x + 1
                    const float rr[3][2] = {{P2r[m - 1][0][s], P2r[m - 1][1][s]},
                                            {P1r[m - 1][0][s], P1r[m - 1][1][s]},
                                            {rs0[s], rs1[s]}};
                    float rsh[3][2][3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float l = __shfl_up_sync(kFullMask, rr[d][1], 1);
                        const float r = __shfl_down_sync(kFullMask, rr[d][0], 1);
                        rsh[d][0][0] = l;
                        rsh[d][0][1] = rr[d][0];
                        rsh[d][0][2] = rr[d][1];
                        rsh[d][1][0] = rr[d][0];
                        rsh[d][1][1] = rr[d][1];
                        rsh[d][1][2] = r;
                    }
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const unsigned wsrc =
                            L::ey(i) < 0 ? gp[s][i] : (L::ey(i) == 0 ? E0g[m - 1][s][i] : P2g[m - 1][s][i]);
                        float g0, g1;
                        if (L::ex(i) > 0) {
                            g0 = hi16<H>(__shfl_up_sync(kFullMask, wsrc, 1));
                            g1 = lo16<H>(wsrc);
                        } else if (L::ex(i) < 0) {
                            g0 = hi16<H>(wsrc);
                            g1 = lo16<H>(__shfl_down_sync(kFullMask, wsrc, 1));
                        } else {
                            g0 = lo16<H>(wsrc);
                            g1 = hi16<H>(wsrc);
                        }
                        pull_pair<PK>(weight<Q, float>(i), rsh[1 - L::ey(i)][0][1 - L::ex(i)],
                                      rsh[1 - L::ey(i)][1][1 - L::ex(i)], g0, g1, f0[s][i], f1[s][i]);
                    }
                    f0[s][0] = rn_fma(weight<Q, float>(0), P1r[m - 1][0][s], -E0s[m - 1][0][s]);
                    f1[s][0] = rn_fma(weight<Q, float>(0), P1r[m - 1][1][s], -E0s[m - 1][1][s]);
                }
                // level m's rows move down: this row becomes the previous one
#pragma unroll
                for (int s = 0; s < S; ++s) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        P2r[m - 1][c][s] = P1r[m - 1][c][s];
                        P1r[m - 1][c][s] = c ? rs1[s] : rs0[s];
                        E0s[m - 1][c][s] = c ? gs1[s] : gs0[s];
                    }
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        if (L::ey(i) > 0) {
                            P2g[m - 1][s][i] = P1g[m - 1][s][i];
                            P1g[m - 1][s][i] = gp[s][i];
                        } else if (L::ey(i) == 0) {
                            E0g[m - 1][s][i] = gp[s][i];
                        }
                    }
                }
                collide_half_pair<Q, S, H, RK, PK>(g, f0, f1, rho0, rho1, rs0, rs1, gp, gs0, gs1);
            }
            if (j >= 2 * K) {  // level K of row y0 + j - 2K: window columns HL .. 63 - HL
                const int x = xb + 2 * lane;
                if (lane >= HL / 2 && lane < (HL + WO) / 2 && x < nx) {  // nx even: x + 1 < nx too
                    const int y = y0 + j - 2 * K;
                    const int64_t yx = (int64_t)y * pitch + x;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        unsigned char *base = dst + s * sp_bytes;
                        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(base) + yx) = make_float2(rs0[s], rs1[s]);
                        unsigned short *gd = reinterpret_cast<unsigned short *>(base + plane * 4);
#pragma unroll
                        for (int i = 1; i < Q; ++i)
                            *reinterpret_cast<unsigned *>(gd + (int64_t)(i - 1) * plane + yx) = gp[s][i];
                        if (g.rho_out)
                            *reinterpret_cast<float2 *>(static_cast<float *>(g.rho_out) + s * plane + yx) =
                                make_float2(rho0[s], rho1[s]);
                        sum[s] += rho0[s] + rho1[s];
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

template <int Q, int S, int H, int K, int NW, int NS, int MINB, bool BATCH, int RK = -1>
struct HalfPairKernel {
    static constexpr size_t smem = (size_t)NW * NS * S * (72 * 4 + (Q - 1) * 72 * 2);
    static cudaError_t get(unsigned *full) {
        auto kern = step_half_pair_kernel<Q, S, H, K, NW, NS, MINB, BATCH, RK>;
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
cudaError_t launch_half_pair_rk(const StepArgs &a, cudaStream_t st) {
    constexpr int WO = HalfPairGeom<K>::WO;
    using HK = HalfPairKernel<Q, S, H, K, NW, NS, MINB, false, RK>;
    unsigned full = 0;
    cudaError_t e = HK::get(&full);
    if (e != cudaSuccess) return e;
    const int64_t nstrips = (a.nx + WO - 1) / WO;
    const int64_t nwarps = (int64_t)full * NW;
    const int64_t nb = choose_bands(K, nstrips, a.ny, nwarps);
    const int64_t band = (a.ny + nb - 1) / nb, nbands = (a.ny + band - 1) / band;
    const int64_t units = nstrips * nbands;
    const unsigned grid = units < nwarps ? (unsigned)((units + NW - 1) / NW) : full;
    step_half_pair_kernel<Q, S, H, K, NW, NS, MINB, false, RK>
        <<<grid, NW * 32, HK::smem, st>>>(a, nstrips, nbands, band, nullptr, 0, 0, a.rho_out != nullptr);
    return cudaGetLastError();
}

// nx a multiple of 8 (16-byte chunks of 16-bit values never straddle the
// seam); two-species Gray-Scott grids run the form with the reaction fixed at
// compile time.
template <int Q, int S, int H, int K, int NW, int NS, int MINB>
cudaError_t launch_half_pair(const StepArgs &a, cudaStream_t st) {
    if (a.nx % 8 != 0 || a.pitch % 8 != 0) return cudaErrorInvalidValue;
    if constexpr (S == 2)
        if (a.rkind == kGrayScott) return launch_half_pair_rk<Q, S, H, K, NW, NS, MINB, kGrayScott>(a, st);
    return launch_half_pair_rk<Q, S, H, K, NW, NS, MINB, -1>(a, st);
}

}  // namespace
}  // namespace lbrd
