// Tiled fused 55-point substep, two points per thread, packed FP32x2
// arithmetic, output planes finished three planes behind the in-plane work.
//
// The pipeline is that of the two-point kernel (one TMA copy per plane of
// all fields into a ring of shared-memory slots, u-tilde by a second TMA
// ring, paired shared loads, the thread's z-column in registers).  What
// differs is where the Eq. 8 terms that pair z with x or y take their
// in-plane differences from:
//
//   D_xz f(z) = sum_k MX_k [h_k(z+k) - h_k(z-k)],  h_k = f(x+k) - f(x-k),
//   D_yz f(z) = sum_k MX_k [g_k(z+k) - g_k(z-k)],  g_k = f(y+k) - f(y-k).
//
// h_k and g_k of u_x, u_y, u_z on a plane are exactly the x and y arm
// differences that plane's own first-derivative stencils form when it is the
// centre plane.  So each plane is read from shared memory once: when it is
// the centre, its arm differences go into running sums of the six output
// planes around it (plus to the planes below it, for which it is z + k;
// minus to those above, for which it is z - k), and output plane o is
// complete once plane o + 3 has been the centre.  Its right-hand side without
// those terms waits three planes, in registers or (TM, the default) in tensor
// memory; the state of its column is already held for the z stencils.  The
// three halo planes below and above a z-chunk are never centres: their arm
// differences come from loads of their own.
//
// Per output plane and thread this reads 92 shared pairs (5 column values,
// 50 x/y arms of the five fields, 32 for the two (x, y) cross terms, 5 of
// u-tilde; 96 with the halo planes of 40-plane chunks) where loading the
// arms of each arriving plane takes 116.
#pragma once

#include "tcgen05.cuh"
#include "tiled2_impl.cuh"

namespace gbfd {
namespace tiled4 {

using tiled2::PairOps;

// With TM, the pending right-hand sides wait in tensor memory instead of
// registers: a ring of 4 slots of 16 FP32 columns (one lane per thread, the
// 2 NF values of its two points), written once and read once per plane.
constexpr int kTmSlotCols = 16;
constexpr int kTmCols = 4 * kTmSlotCols;

// Warp-collective 32x32b accesses of n consecutive columns of the thread's
// own lane, each waiting for its own completion in the same statement.  They
// are .sync.aligned: the warp is reconverged first, since the bounded
// mbarrier spins before them exit lane by lane (without it, a register-capped
// build of this kernel read back wrong values).
__device__ __forceinline__ void tm_st8(uint32_t ta, const float2 *v)
{
    __syncwarp();
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n\t"
                 "tcgen05.wait::st.sync.aligned;" ::"r"(ta),
                 "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y),
                 "f"(v[3].x), "f"(v[3].y)
                 : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t ta, float2 *v)
{
    __syncwarp();
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x),
                   "=f"(v[2].y), "=f"(v[3].x), "=f"(v[3].y)
                 : "r"(ta)
                 : "memory");
}

// The five-field pending right-hand side (8 + 2 columns) in one round trip:
// both accesses issued, then one wait (two waits in a row cost 0.6% of the
// default kernel's time at 256^3 and 512^3).
__device__ __forceinline__ void tm_st10(uint32_t ta, const float2 *v)
{
    __syncwarp();
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n\t"
                 "tcgen05.st.sync.aligned.32x32b.x2.b32 [%9], {%10, %11};\n\t"
                 "tcgen05.wait::st.sync.aligned;" ::"r"(ta),
                 "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y),
                 "f"(v[3].x), "f"(v[3].y), "r"(ta + 8), "f"(v[4].x), "f"(v[4].y)
                 : "memory");
}
__device__ __forceinline__ void tm_ld10(uint32_t ta, float2 *v)
{
    __syncwarp();
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%10];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%11];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x),
                   "=f"(v[2].y), "=f"(v[3].x), "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y)
                 : "r"(ta), "r"(ta + 8)
                 : "memory");
}

// Shared-memory carve-up: NS state-plane slots, NW u-tilde slots, barriers.
template <class TW, int NF, int TX, int TY, int NS, int U>
struct RingL : tiled2::Ring<float, TW, NF, TX, TY, NS, U + 2> {
    using Base = tiled2::Ring<float, TW, NF, TX, TY, NS, U + 2>;
    static constexpr int TM_OFF = (Base::BYTES + 15) / 16 * 16;  // TMEM address word
    static constexpr int BYTES = TM_OFF + 16;
};

// One z-chunk of one column; same contract as the two-point kernel's column
// routine (barrier phases continue across calls through jrun / wrun; false
// when a bounded wait gave up).
// STG >= 0 fixes the RK3 substep (0, 1, 2) at compile time, FULL says that
// every tile lies inside the grid; both only drop run-time tests.
template <class TW, class TA, int NF, int TX, int TY, int NS, int U, bool ICVT, bool FORCE, bool TM,
          class CoefT, bool SHFL = false, int STG = -1, bool FULL = false>
__device__ __forceinline__ bool run_column(const CUtensorMap *tmap, const CUtensorMap *wmap,
                                           float *__restrict__ out, TW *__restrict__ w,
                                           const Layout &Ls, const Layout &Lw, const CoefT &c,
                                           const TA alpha, const TA beta, const TA dt,
                                           const bool first_arg, const bool last_arg, const int x0,
                                           const int y0, const int z0, const int nout, int &jrun,
                                           int &wrun, unsigned char *smem, int *dev_error,
                                           const int skip_plane, const Forcing *fo,
                                           const uint32_t tmem)
{
    using RG = RingL<TW, NF, TX, TY, NS, U>;
    using tiled::mbar_wait;
    using P = PairOps<float>;
    using V = float2;
    using VW = typename tiled2::V2<TW>::t;
    constexpr int BX = RG::BX, FSTRIDE = RG::FSTRIDE, SLOT_ELEMS = RG::SLOT_ELEMS;
    constexpr int NW = RG::NW;
    constexpr int NTX = TX / 2;
    constexpr bool UP32 = std::is_same<TA, float>::value && std::is_same<TW, float>::value;
    // the prologue holds local planes 0..5 at once; each step reads its
    // centre plane and the plane three above it
    static_assert(NS >= 6 && NS >= U + 4, "ring too short");
    static_assert(U >= 1 && U <= 2, "one or two steps per loop iteration");
    const float *sm = reinterpret_cast<const float *>(smem);
    unsigned char *wsm = smem + RG::W_OFF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF);
    uint64_t *wbars = bars + NS;

    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const int nz = Ls.nz;
    const int nplanes = nout + 2 * R;
    const int x = x0 + 2 * tx, y = y0 + ty;
    const bool first = STG >= 0 ? STG == 0 : first_arg;
    const bool last = STG >= 0 ? STG == 2 : last_arg;
    const bool valid0 = FULL || ((x < Ls.nx) && (y < Ls.ny));  // nx % 4 == 0: x+1 valid with x
    const int toff = (ty + GY) * BX + (2 * tx + GX);
    const bool need_w = !first;
    float2 fxy0 = make_float2(0.f, 0.f), fxy1 = make_float2(0.f, 0.f);
    if constexpr (FORCE) {
        // the column's x-y phase factor of the forcing, Re/Im of tx[x] ty[y]
        if (valid0) {
            const float2 a0 = __ldg(fo->tx32 + x), a1 = __ldg(fo->tx32 + x + 1);
            const float2 b = __ldg(fo->ty32 + y);
            fxy0 = make_float2(a0.x * b.x - a0.y * b.y, a0.x * b.y + a0.y * b.x);
            fxy1 = make_float2(a1.x * b.x - a1.y * b.y, a1.x * b.y + a1.y * b.x);
        }
    }

    __syncthreads();

    // local state plane j is grid plane z0 - 3 + j (wrapped), copy jrun + j
    // of this CTA: slot (jrun + j) % NS, phase ((jrun + j) / NS) & 1
    int issued = 0, wissued = 0;
    auto issue = [&](int j) {
        if (j == skip_plane)  // fault injection for the bounded-wait test
            return;
        int z = z0 - R + j;
        z = zplane(Ls, z) + Ls.gz;  // TMA z coordinate
        const int slot = (jrun + j) % NS;
        tiled::mbar_expect_tx(&bars[slot], RG::SLOT_BYTES);
        tiled::tma_load_4d(smem + slot * RG::SLOT_PITCH, tmap, &bars[slot], x0, y0, z, 0);
    };
    auto issue_w = [&](int o) {
        const int slot = (wrun + o) % NW;
        tiled::mbar_expect_tx(&wbars[slot], RG::WSLOT_BYTES);
        tiled::tma_load_4d(wsm + slot * RG::WSLOT_PITCH, wmap, &wbars[slot], x0 + GX, y0 + GY,
                           z0 + o, 0);
    };
    if (threadIdx.x == 0) {
        tiled::fence_proxy_async();
#pragma unroll 1
        for (int j = 0; j < NS && j < nplanes; ++j)
            issue(j);
        issued = min(NS, nplanes);
        if (need_w) {
#pragma unroll 1
            for (int o = 0; o < NW && o < nout; ++o)
                issue_w(o);
            wissued = min(NW, nout);
        }
    }

    // Register windows, relative to the first step `s0` of the current loop
    // iteration (step s works on local plane s, output plane s - 3):
    //   colv[f][k]  field f of both points at local plane s0 - 3 + k
    //   acx/acy/acz[m]  the z-paired Eq. 8 terms of output plane s0 - 6 + m
    //                   for the x (D_xz u_z), y (D_yz u_z) and z (D_xz u_x +
    //                   D_yz u_y) components
    //   pr[f][m]    the rest of the right-hand side of output plane s0 - 6 + m
    constexpr int W = 6 + U;
    V colv[NF][W];
    V acx[W], acy[W], acz[W];
    V pr[NF][TM ? 1 : 3 + U];
    // this thread's TMEM lane (the warp's 32-lane quarter), column 0
    const uint32_t trow = tmem + ((uint32_t)(threadIdx.x & ~31) << 16);
    (void)trow;
#pragma unroll
    for (int m = 0; m < W; ++m)
        acx[m] = acy[m] = acz[m] = P::bc(0.f);

    const V NEG1 = P::bc(-1.f);
    // add the arm differences d[k-1] of one plane, ac index MC, with weights
    // MX(pair, k): plus to the outputs below it, minus to those above
    auto spread = [&](V *ac, const V *d, int pair, auto mcc) {
        constexpr int MC = decltype(mcc)::value;
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const float mk = c.MX(pair, k);
            if (MC - k >= 0)
                ac[MC - k] = P::fma(P::bc(mk), d[k - 1], ac[MC - k]);
            if (MC + k < W)
                ac[MC + k] = P::fma(P::bc(-mk), d[k - 1], ac[MC + k]);
        }
    };
    // x-differences h_k (k = 1..3) of both points from the pairs of a row at
    // x offsets -4, -2, +2, +4 and the centre pair (of the outer pairs only
    // m4.y and p4.x enter, here and in the second derivative)
    auto xdiff = [&](V m4, V m2, V cc, V p2, V p4, V *h) {
        h[0] = P::mk(cc.y - m2.y, p2.x - cc.x);
        h[1] = P::fma(m2, NEG1, p2);
        h[2] = P::mk(p2.y - m4.y, p4.x - m2.x);
    };
    // the x-neighbour pairs of the centre pair cc at shared-memory index fb
    // (the pair's own element): SHFL takes them from the lanes that hold them
    // (a row is NTX consecutive lanes), and the two lanes at each end of the
    // row the missing ones from one 16-byte load of the four halo values on
    // their side; otherwise four paired shared loads
    auto xnb = [&](int fb, V cc, V &m4, V &m2, V &p2, V &p4) {
        if constexpr (SHFL) {
            static_assert(NTX == 16 || NTX == 32, "a row within one warp");
            static_assert(GX == 4 && RG::BX % 4 == 0 && RG::FSTRIDE % 4 == 0 &&
                              RG::SLOT_ELEMS % 4 == 0,
                          "16-byte aligned halo quads");
            constexpr unsigned ALL = 0xffffffffu;
            m2.x = __shfl_up_sync(ALL, cc.x, 1, NTX);
            m2.y = __shfl_up_sync(ALL, cc.y, 1, NTX);
            m4.y = __shfl_up_sync(ALL, cc.y, 2, NTX);
            p2.x = __shfl_down_sync(ALL, cc.x, 1, NTX);
            p2.y = __shfl_down_sync(ALL, cc.y, 1, NTX);
            p4.x = __shfl_down_sync(ALL, cc.x, 2, NTX);
            m4.x = p4.y = 0.f;
            const bool lo = tx < 2, hi = tx >= NTX - 2;
            if (lo || hi) {
                // the row's halo columns: x offsets -4..-1 or TX..TX+3 of the tile
                const int rb = fb - 2 * tx - GX + (lo ? 0 : GX + TX);
                const float4 e = *reinterpret_cast<const float4 *>(sm + rb);
                if (tx == 0) {
                    m4.y = e.y;
                    m2 = make_float2(e.z, e.w);
                } else if (tx == 1) {
                    m4.y = e.w;
                } else if (tx == NTX - 1) {
                    p2 = make_float2(e.x, e.y);
                    p4.x = e.z;
                } else {
                    p4.x = e.x;
                }
            }
        } else {
            m4 = *reinterpret_cast<const V *>(sm + fb - 4);
            m2 = *reinterpret_cast<const V *>(sm + fb - 2);
            p2 = *reinterpret_cast<const V *>(sm + fb + 2);
            p4 = *reinterpret_cast<const V *>(sm + fb + 4);
        }
    };
    // a plane that is not a centre (the halo planes of the chunk): its arm
    // differences alone, from its own loads; centre pairs from colv[.][MC]
    auto arms = [&](int base, auto mcc) {
        constexpr int MC = decltype(mcc)::value;
        auto at = [&](int f, int dy, int dx) -> V {
            return *reinterpret_cast<const V *>(sm + base + f * FSTRIDE + dy * BX + dx);
        };
        V h[3], gd[3], m4, m2, p2, p4;
        // u_x: x-differences -> z component
        xnb(base + FSTRIDE, colv[1][MC], m4, m2, p2, p4);
        xdiff(m4, m2, colv[1][MC], p2, p4, h);
        spread(acz, h, 1, mcc);
        // u_y: y-differences -> z component
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            gd[k - 1] = P::fma(at(2, -k, 0), NEG1, at(2, k, 0));
        spread(acz, gd, 2, mcc);
        // u_z: x-differences -> x component, y-differences -> y component
        xnb(base + 3 * FSTRIDE, colv[3][MC], m4, m2, p2, p4);
        xdiff(m4, m2, colv[3][MC], p2, p4, h);
        spread(acx, h, 1, mcc);
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            gd[k - 1] = P::fma(at(3, -k, 0), NEG1, at(3, k, 0));
        spread(acy, gd, 2, mcc);
    };

    bool timeout = false;
    // prologue: local planes 0..5 into the column window; the three halo
    // planes below the chunk (local 0..2) give their arm differences
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        const int q = jrun + j;
        if (!mbar_wait(&bars[q % NS], (q / NS) & 1))
            timeout = true;
        const int base = (q % NS) * SLOT_ELEMS + toff;
#pragma unroll
        for (int f = 0; f < NF; ++f)
            colv[f][j] = *reinterpret_cast<const V *>(sm + base + f * FSTRIDE);
        if (j == 0)
            arms(base, std::integral_constant<int, 0>{});
        else if (j == 1)
            arms(base, std::integral_constant<int, 1>{});
        else if (j == 2)
            arms(base, std::integral_constant<int, 2>{});
    }
    int waited = 2 * R, wwaited = 0;

    // global offsets of point (x, y) in the next output plane to finish
    long long go_s = (long long)z0 * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
    long long go_w = (long long)z0 * Lw.plane + (long long)(y + GY) * Lw.P + (x + GX);
    long long gdx = 0, gdy = 0;
    if (x < GX)
        gdx = Ls.nx;
    else if (x >= Ls.nx - GX)
        gdx = -Ls.nx;
    if (y < GY)
        gdy = (long long)Ls.ny * Ls.P;
    else if (y >= Ls.ny - GY)
        gdy = -(long long)Ls.ny * Ls.P;

    // centre step S of the iteration: local plane s (slot offset cb), output
    // plane s - 3; everything of the right-hand side but the z-paired Eq. 8
    // terms into prn, its arm differences into the accumulators
    auto centre = [&](const int cb, auto sc, V *prn) {
        constexpr int S = decltype(sc)::value;
        constexpr int MC = S + 3;
        auto C = [&](int f, int k) -> V & { return colv[f][S + k]; };
        auto ld2 = [&](int f, int dy, int dx) -> V {
            return *reinterpret_cast<const V *>(sm + cb + f * FSTRIDE + dy * BX + dx);
        };
        V g[3], d2[3], h[3], gd[3], y1p, y1m;
        auto axial = [&](int f, bool second) {
            const V cc = C(f, 3);
            V m4, m2, p2, p4;
            xnb(cb + f * FSTRIDE, cc, m4, m2, p2, p4);
            xdiff(m4, m2, cc, p2, p4, h);
            g[0] = P::fma(P::bc(c.D1(0, 3)), h[2],
                          P::fma(P::bc(c.D1(0, 2)), h[1], P::mul(P::bc(c.D1(0, 1)), h[0])));
            if (second) {
                const V s1 = P::mk(cc.y + m2.y, p2.x + cc.x);
                const V s3 = P::mk(p2.y + m4.y, p4.x + m2.x);
                d2[0] = P::fma(P::bc(c.D2(0, 3)), s3,
                               P::fma(P::bc(c.D2(0, 2)), P::add(p2, m2),
                                      P::fma(P::bc(c.D2(0, 1)), s1, P::mul(P::bc(c.D2c(0)), cc))));
            }
            V gy, by, gz, bz;
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                const V yp = ld2(f, k, 0), ym = ld2(f, -k, 0);
                if (k == 1) {
                    y1p = yp;
                    y1m = ym;
                }
                const V zp = C(f, 3 + k), zm = C(f, 3 - k);
                const V dyv = P::fma(ym, NEG1, yp), dzv = P::fma(zm, NEG1, zp);
                gd[k - 1] = dyv;
                gy = k == 1 ? P::mul(P::bc(c.D1(1, k)), dyv) : P::fma(P::bc(c.D1(1, k)), dyv, gy);
                gz = k == 1 ? P::mul(P::bc(c.D1(2, k)), dzv) : P::fma(P::bc(c.D1(2, k)), dzv, gz);
                if (second) {
                    if (k == 1) {
                        by = P::mul(P::bc(c.D2c(1)), C(f, 3));
                        bz = P::mul(P::bc(c.D2c(2)), C(f, 3));
                    }
                    by = P::fma(P::bc(c.D2(1, k)), P::add(yp, ym), by);
                    bz = P::fma(P::bc(c.D2(2, k)), P::add(zp, zm), bz);
                }
            }
            g[1] = gy;
            g[2] = gz;
            if (second) {
                d2[1] = by;
                d2[2] = bz;
            }
        };
        // Eq. 8 in the (x, y) plane: D_xy f = sum_k MX_k [h_k(y+k) - h_k(y-k)];
        // the centre pairs of rows y+-1 are those of the y arm just loaded
        auto mix_xy = [&](int f) -> V {
            V a;
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                V hh[2];
#pragma unroll
                for (int sgn = 0; sgn < 2; ++sgn) {
                    const int dy = sgn ? -k : k;
                    const V m2 = ld2(f, dy, -2), p2 = ld2(f, dy, 2);
                    if (k == 1) {
                        const V cc = sgn ? y1m : y1p;
                        hh[sgn] = P::mk(cc.y - m2.y, p2.x - cc.x);
                    } else if (k == 2) {
                        hh[sgn] = P::fma(m2, NEG1, p2);
                    } else {
                        const V m4 = ld2(f, dy, -4), p4 = ld2(f, dy, 4);
                        hh[sgn] = P::mk(p2.y - m4.y, p4.x - m2.x);
                    }
                }
                const V d = P::fma(hh[1], NEG1, hh[0]);
                a = k == 1 ? P::mul(P::bc(c.MX(0, k)), d) : P::fma(P::bc(c.MX(0, k)), d, a);
            }
            return a;
        };
        const V NU = P::bc(c.nu), NU3 = P::bc(c.nu3);
        const V uc[3] = {C(1, 3), C(2, 3), C(3, 3)};
        V acc[4], gl[3];
        V dv = P::bc(0.f);
        axial(0, false);
        gl[0] = g[0];
        gl[1] = g[1];
        gl[2] = g[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            axial(1 + i, true);
            // the arm differences of this plane, in the same order as a halo plane's
            if (i == 0) {
                spread(acz, h, 1, std::integral_constant<int, MC>{});
            } else if (i == 1) {
                spread(acz, gd, 2, std::integral_constant<int, MC>{});
            } else {
                spread(acx, h, 1, std::integral_constant<int, MC>{});
                spread(acy, gd, 2, std::integral_constant<int, MC>{});
            }
            V adv = P::mul(uc[0], g[0]);
            adv = P::fma(uc[1], g[1], adv);
            adv = P::fma(uc[2], g[2], adv);
            const V lap = P::add(P::add(d2[0], d2[1]), d2[2]);
            V sg = P::mul(g[0], gl[0]);
            sg = P::fma(g[1], gl[1], sg);
            sg = P::fma(g[2], gl[2], sg);
            V ai = P::mul(NU, P::add(lap, sg));
            if (i > 0)
                ai = P::add(ai, acc[1 + i]);
            ai = P::fma(adv, NEG1, ai);
            ai = P::fma(NU3, d2[i], ai);
            acc[1 + i] = ai;
            const V nugl = P::mul(NU, gl[i]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == i)
                    acc[1 + a] = P::fma(g[a], nugl, acc[1 + a]);
                else if (a > i && i == 0)
                    acc[1 + a] = P::mul(g[a], nugl);  // first contribution
                else
                    acc[1 + a] = P::fma(g[a], nugl, acc[1 + a]);
            }
            dv = P::add(dv, g[i]);
            if (i == 0)
                acc[2] = P::fma(NU3, mix_xy(1), acc[2]);  // D_xy u_x -> y
            else if (i == 1)
                acc[1] = P::fma(NU3, mix_xy(2), acc[1]);  // D_xy u_y -> x
        }
        if constexpr (NF == 5) {
            axial(4, false);
            V t = P::mul(uc[0], g[0]);
            t = P::fma(uc[1], g[1], t);
            t = P::fma(uc[2], g[2], t);
            prn[4] = P::mul(t, NEG1);
        }
        V ug = P::mul(uc[0], gl[0]);
        ug = P::fma(uc[1], gl[1], ug);
        ug = P::fma(uc[2], gl[2], ug);
        prn[0] = P::mul(P::add(ug, dv), NEG1);
        const V NCS2 = P::bc(-c.cs2);
        const V t = P::mul(P::bc(-c.nu23), dv);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            prn[1 + a] = P::fma(t, gl[a], P::fma(NCS2, gl[a], acc[1 + a]));
    };

    // output plane o (window index S): add the z-paired terms and the
    // forcing, apply Eq. 10, store the state (and ghost copies) and u-tilde
    auto finish = [&](const int o, auto sc) {
        constexpr int S = decltype(sc)::value;
        V prv[NF];
        if constexpr (TM) {
            const uint32_t ta = trow + (uint32_t)((o & 3) * kTmSlotCols);
            if constexpr (NF == 5)
                tm_ld10(ta, prv);
            else
                tm_ld8(ta, prv);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                prv[f] = pr[f][S];
        }
        if (need_w) {
            const int qw = wrun + o;
            if (!mbar_wait(&wbars[qw % NW], (qw / NW) & 1))
                timeout = true;
            wwaited = o + 1;
        }
        if (valid0) {
            VW wv[NF];
            if (need_w) {
                const TW *ws = reinterpret_cast<const TW *>(wsm + ((wrun + o) % NW) * RG::WSLOT_PITCH) +
                               ty * TX + 2 * tx;
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    wv[f] = *reinterpret_cast<const VW *>(ws + f * TX * TY);
            }
            const V NU3 = P::bc(c.nu3);
            V r[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f)
                r[f] = prv[f];
            r[1] = P::fma(NU3, acx[S], r[1]);
            r[2] = P::fma(NU3, acy[S], r[2]);
            r[3] = P::fma(NU3, acz[S], r[3]);
            if constexpr (FORCE) {
                // f_i = amp_i cos(k.x + phi)
                const float2 cz = __ldg(fo->tz32 + z0 + o);
                const V fc = P::mk(fxy0.x * cz.x - fxy0.y * cz.y, fxy1.x * cz.x - fxy1.y * cz.y);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    r[1 + a] = P::fma(P::bc(fo->amp32[a]), fc, r[1 + a]);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const V u0 = colv[f][S];
                V o2;
                if constexpr (UP32) {
                    const V DT = P::bc(dt), ALPHA = P::bc(alpha), BETA = P::bc(beta);
                    const V wn = first ? P::mul(DT, r[f]) : P::fma(DT, r[f], P::mul(ALPHA, wv[f]));
                    o2 = P::fma(BETA, wn, u0);
                    if (!last)
                        *reinterpret_cast<V *>(w + f * Lw.fpitch + go_w) = wn;
                } else if constexpr (std::is_same<TA, ffloat>::value) {
                    // the precision form in float-float arithmetic
                    static_assert(std::is_same<TW, float>::value, "u-tilde stored in FP32");
                    float wo[2] = {first ? 0.f : wv[f].x, first ? 0.f : wv[f].y};
                    float on[2];
                    rk3_update_ff(first, alpha, beta, dt, r[f].x, u0.x, wo[0], on[0]);
                    rk3_update_ff(first, alpha, beta, dt, r[f].y, u0.y, wo[1], on[1]);
                    o2 = make_float2(on[0], on[1]);
                    if (!last)
                        *reinterpret_cast<V *>(w + f * Lw.fpitch + go_w) = make_float2(wo[0], wo[1]);
                } else {
                    static_assert(std::is_same<TA, double>::value, "FP64 update");
                    TW wo[2] = {first ? (TW)0 : wv[f].x, first ? (TW)0 : wv[f].y};
                    float on[2];
                    rk3_update_f64<ICVT, TW>(first, alpha, beta, dt, r[f].x, u0.x, wo[0], on[0]);
                    rk3_update_f64<ICVT, TW>(first, alpha, beta, dt, r[f].y, u0.y, wo[1], on[1]);
                    o2 = make_float2(on[0], on[1]);
                    if (!last) {
                        VW tw;
                        tw.x = wo[0];
                        tw.y = wo[1];
                        *reinterpret_cast<VW *>(w + f * Lw.fpitch + go_w) = tw;
                    }
                }
                float *op = out + f * Ls.fpitch + go_s;
                *reinterpret_cast<V *>(op) = o2;
                if (gdx)
                    *reinterpret_cast<V *>(op + gdx) = o2;
                if (gdy) {
                    *reinterpret_cast<V *>(op + gdy) = o2;
                    if (gdx)
                        *reinterpret_cast<V *>(op + gdy + gdx) = o2;
                }
            }
        }
        go_s += Ls.plane;
        go_w += Lw.plane;
    };

    // main-loop step s (window index S): the column value of local plane
    // s + 3, the centre work on local plane s (output plane s - 3), then
    // output plane s - 6 when there is one
    auto step = [&](const int s, auto sc) {
        constexpr int S = decltype(sc)::value;
        const int cb = (int)((unsigned)(jrun + s) % NS) * SLOT_ELEMS + toff;
        const int qn = jrun + s + R;
        if (!mbar_wait(&bars[qn % NS], (qn / NS) & 1))
            timeout = true;
        waited = s + R + 1;
        const int nb = (qn % NS) * SLOT_ELEMS + toff;
#pragma unroll
        for (int f = 0; f < NF; ++f)
            colv[f][S + 6] = *reinterpret_cast<const V *>(sm + nb + f * FSTRIDE);
        // every lane computes (the tile box is in shared memory whatever the
        // grid extent); only the stores of finish() look at valid0
        V prn[NF];
        centre(cb, sc, prn);
        if constexpr (TM) {
            const uint32_t ta = trow + (uint32_t)(((s - R) & 3) * kTmSlotCols);
            if constexpr (NF == 5)
                tm_st10(ta, prn);
            else
                tm_st8(ta, prn);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                pr[f][S + 3] = prn[f];
        }
        if (s >= 2 * R)
            finish(s - 2 * R, sc);
    };
    // slide every window by SH steps
    auto shift = [&](auto shc) {
        constexpr int SH = decltype(shc)::value;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
#pragma unroll
            for (int k = 0; k + SH < W; ++k)
                colv[f][k] = colv[f][k + SH];
            if constexpr (!TM) {
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    pr[f][m] = pr[f][m + SH];
            }
        }
#pragma unroll
        for (int m = 0; m < W; ++m) {
            acx[m] = m + SH < W ? acx[m + SH] : P::bc(0.f);
            acy[m] = m + SH < W ? acy[m + SH] : P::bc(0.f);
            acz[m] = m + SH < W ? acz[m + SH] : P::bc(0.f);
        }
    };
    // all threads are done with the steps before s0: slots of local planes
    // below s0 and u-tilde slots of outputs below s0 - 6 are free; returns
    // true (for every thread) when some thread's wait gave up
    auto top = [&](const int s0) -> bool {
        if (__syncthreads_or(timeout))
            return true;
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            const int jend = min(s0 + NS, nplanes);
#pragma unroll 1
            for (int j = issued; j < jend; ++j)
                issue(j);
            issued = max(issued, jend);
            if (need_w) {
                const int tend = min(s0 - 2 * R + NW, nout);
#pragma unroll 1
                for (int t = wissued; t < tend; ++t)
                    issue_w(t);
                wissued = max(wissued, tend);
            }
        }
        return false;
    };

    int s0 = R;
    bool stop = false;
#pragma unroll 1
    for (; s0 + U <= nout + R; s0 += U) {
        if (top(s0)) {
            stop = true;
            break;
        }
        step(s0, std::integral_constant<int, 0>{});
        if constexpr (U > 1)
            step(s0 + 1, std::integral_constant<int, 1>{});
        shift(std::integral_constant<int, U>{});
    }
    if constexpr (U > 1) {
        // an odd number of output planes: one centre step left
        if (!stop && s0 < nout + R) {
            if (top(s0)) {
                stop = true;
            } else {
                step(s0, std::integral_constant<int, 0>{});
                shift(std::integral_constant<int, 1>{});
                ++s0;
            }
        }
    }
    // the last u-tilde copies (the state planes are all issued by now)
    if (!stop && top(s0))
        stop = true;
    if (!stop) {
        // the three halo planes above the chunk (local s0 .. s0 + 2, all in
        // the ring already): their arm differences finish the last outputs
        auto tail = [&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const int s = s0 + E;
            arms((int)((unsigned)(jrun + s) % NS) * SLOT_ELEMS + toff,
                 std::integral_constant<int, E + 3>{});
            if (s >= 2 * R)
                finish(s - 2 * R, ec);
        };
        tail(std::integral_constant<int, 0>{});
        tail(std::integral_constant<int, 1>{});
        tail(std::integral_constant<int, 2>{});
    }
    const bool bad = __syncthreads_or(timeout);
    if (bad && threadIdx.x == 0) {
        atomicExch(dev_error, 1);
        // drain the copies still in flight into this CTA's shared memory
        // (the copy that fault injection skipped never lands: not waited for)
        for (int j = waited; j < issued; ++j)
            if (j != skip_plane)
                (void)mbar_wait(&bars[(jrun + j) % NS], ((jrun + j) / NS) & 1);
        for (int o = wwaited; o < wissued; ++o)
            (void)mbar_wait(&wbars[(wrun + o) % NW], ((wrun + o) / NW) & 1);
    }
    jrun += nplanes;
    wrun += need_w ? nout : 0;
    return !bad;
}

// Single box: one CTA per (tile, z-chunk).
// CoefT: Coef<float>, or CubicCoef<float> when the grid spacing is the same on
// every axis (10 stencil weights instead of 30, few enough to stay in uniform
// registers).
template <class TW, class TA, int NF, int TX, int TY, int NS, int U, int MINB, bool ICVT,
          bool FORCE, bool TM, class CoefT, bool SHFL, int STG = -1, bool FULL = false>
__global__ void __launch_bounds__((TX / 2) * TY, MINB) k_substep_lag(
    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap wmap,
    float *__restrict__ out, TW *__restrict__ w, const Layout Ls, const Layout Lw,
    const CoefT c, const RKStage st, const int zc, const int tiles_x,
    int *__restrict__ dev_error, const int skip_plane)
{
    using RG = RingL<TW, NF, TX, TY, NS, U>;
    extern __shared__ __align__(128) unsigned char smem[];
    tiled2::init_barriers(reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF), NS + RG::NW);
    uint32_t tmem = 0;
    if constexpr (TM) {
        // warp 0 allocates the CTA's columns; every thread reads the address
        uint32_t *slot = reinterpret_cast<uint32_t *>(smem + RG::TM_OFF);
        if (threadIdx.x < 32)
            tc::tmem_alloc(slot, kTmCols);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = *reinterpret_cast<volatile uint32_t *>(slot);
    }
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nout = min(zc, Ls.nz - z0);
    int jrun = 0, wrun = 0;
    run_column<TW, TA, NF, TX, TY, NS, U, ICVT, FORCE, TM, CoefT, SHFL, STG, FULL>(
        &tmap, &wmap, out, w, Ls, Lw, c, (TA)st.alpha, (TA)st.beta, (TA)st.dt, st.first != 0,
        st.last != 0, x0, y0, z0, nout, jrun, wrun, smem, dev_error,
        blockIdx.x == 0 && blockIdx.y == 0 ? skip_plane : -1, &st.fo, tmem);
    if constexpr (TM) {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x < 32)
            tc::tmem_dealloc(tmem, kTmCols);
    }
}

}  // namespace tiled4

// Launch of the lagged-output kernel for the 55-point form (form 0 only).
template <class TW, class TA, int TX, int TY, int NS, int U, bool TM = false, int MINB = 1,
          bool ICVT = false, bool SHFL = false>
cudaError_t launch_lag_cfg(const StateBufs &b, const Coef<float> &c, const RKStage &st, int nf,
                           int zc, int cfg_key, int *dev_error, TmapCache *cache,
                           cudaStream_t stream, int *launches)
{
    const int skip_plane = st.fault_skip_plane;
    CUtensorMap *map = nullptr, *wmap = nullptr;
    if (!get_state_tmap(cache, b.in, b.Ls, nf, TX, TY, cfg_key, &map))
        return cudaErrorInvalidValue;
    if (!get_tile_tmap(cache, b.w, b.Lw, nf, TX, TY, cfg_key, &wmap))
        return cudaErrorInvalidValue;
    const int tiles_x = (b.Ls.nx + TX - 1) / TX;
    const int tiles_y = (b.Ls.ny + TY - 1) / TY;
    const dim3 grid(tiles_x * tiles_y, (b.Ls.nz + zc - 1) / zc);
    const dim3 block((TX / 2) * TY);
    float *out = (float *)b.out;
    TW *w = (TW *)b.w;
    cudaError_t e;
    // equal spacing on every axis: the isotropic weights (same values)
    const bool iso = TM && coef_is_cubic(c);
    const CubicCoef<float> cc = cubic_of(c);
#define GBFD_LAUNCH_LAG_C(NFV, FRC, CT, CV)                                                       \
    do {                                                                                          \
        auto kern = tiled4::k_substep_lag<TW, TA, NFV, TX, TY, NS, U, MINB, ICVT, FRC, TM, CT,    \
                                          SHFL>;                                                  \
        constexpr int sm = tiled4::RingL<TW, NFV, TX, TY, NS, U>::BYTES;                          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, *wmap, out, w, b.Ls, b.Lw, CV, st, zc, tiles_x,   \
                                          dev_error, skip_plane);                                 \
    } while (0)
#define GBFD_LAUNCH_LAG(NFV, FRC)                                                                 \
    do {                                                                                          \
        if constexpr (TM) {                                                                       \
            if (iso) {                                                                            \
                GBFD_LAUNCH_LAG_C(NFV, FRC, CubicCoef<float>, cc);                                \
                break;                                                                            \
            }                                                                                     \
        }                                                                                         \
        GBFD_LAUNCH_LAG_C(NFV, FRC, Coef<float>, c);                                              \
    } while (0)
    // the five-field isotropic case on whole tiles (forced steps in FP32
    // arithmetic included): the substep is a template argument and the
    // grid-extent test goes
    constexpr bool SPEC = TM && MINB == 1 && !ICVT && !SHFL && std::is_same<TW, float>::value &&
                          (std::is_same<TA, float>::value || std::is_same<TA, ffloat>::value);
    const bool full = b.Ls.nx % TX == 0 && b.Ls.ny % TY == 0;
    if constexpr (SPEC) {
        // forced steps too, in FP32 arithmetic (the forcing is a compile-time
        // switch of the same kernel)
        const bool frc_ok = !st.fo.on || std::is_same<TA, float>::value;
        if (nf == 5 && frc_ok && iso && full && st.s >= 0 && st.s <= 2) {
#define GBFD_LAUNCH_LAG_S(FRC, SV)                                                                \
    do {                                                                                          \
        auto kern = tiled4::k_substep_lag<TW, TA, 5, TX, TY, NS, U, MINB, ICVT, FRC, TM,          \
                                          CubicCoef<float>, SHFL, SV, true>;                      \
        constexpr int sm = tiled4::RingL<TW, 5, TX, TY, NS, U>::BYTES;                            \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, *wmap, out, w, b.Ls, b.Lw, cc, st, zc, tiles_x,   \
                                          dev_error, skip_plane);                                 \
    } while (0)
#define GBFD_LAUNCH_LAG_SS(FRC)                                                                   \
    do {                                                                                          \
        if (st.s == 0)                                                                            \
            GBFD_LAUNCH_LAG_S(FRC, 0);                                                            \
        else if (st.s == 1)                                                                       \
            GBFD_LAUNCH_LAG_S(FRC, 1);                                                            \
        else                                                                                      \
            GBFD_LAUNCH_LAG_S(FRC, 2);                                                            \
    } while (0)
            if (!st.fo.on) {
                GBFD_LAUNCH_LAG_SS(false);
            } else {
                if constexpr (std::is_same<TA, float>::value)
                    GBFD_LAUNCH_LAG_SS(true);
            }
#undef GBFD_LAUNCH_LAG_SS
#undef GBFD_LAUNCH_LAG_S
            *launches += 1;
            return cudaGetLastError();
        }
    }
    if (nf == 5) {
        if (st.fo.on)
            GBFD_LAUNCH_LAG(5, true);
        else
            GBFD_LAUNCH_LAG(5, false);
    } else {
        if (st.fo.on)
            GBFD_LAUNCH_LAG(4, true);
        else
            GBFD_LAUNCH_LAG(4, false);
    }
#undef GBFD_LAUNCH_LAG
#undef GBFD_LAUNCH_LAG_C
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
