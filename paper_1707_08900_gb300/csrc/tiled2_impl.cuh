// Tiled fused substep, two points per thread (x, x+1).
//
// Pipeline of one CTA over one column of a box (tile x0..x0+TX, y0..y0+TY,
// output planes z0..z0+nout):
// * each z-plane of all NF fields, tile plus 3-cell halo, arrives by ONE 4D
//   TMA copy into a ring of NS shared-memory slots (per-slot mbarrier);
// * u-tilde of the output plane (no halo) arrives by a second TMA ring of 3
//   slots, two planes ahead, so the loop has no global loads at all;
// * every shared-memory read fetches an aligned pair (float2 / double2) that
//   serves both points' stencil arms; the thread's own z-column slides
//   through registers;
// * the barrier phases run on per-CTA counters, so a persistent CTA can
//   stream many columns (of many boxes) through the same ring.
//
// The right-hand side of Eqs. 1-3 is accumulated field by field so that only
// the running sums stay live:
//   grad lnrho first; then for each velocity component u_i with gradient g:
//     rhs_i += -u.g + nu (lap u_i + g.grad lnrho) + (nu/3) D2_i u_i
//     rhs_j += nu g_j d_i lnrho                  (the d_i u_j d_j lnrho half of
//                                                  2 S.grad lnrho, for all j)
//     rhs_j += (nu/3) D_ij u_i  (j != i, 55-point grad div, Eq. 8)
//     div   += g_i
//   finally rhs_i += -c_s^2 d_i lnrho - (2/3) nu div d_i lnrho,
//   rhs_lnrho = -u.grad lnrho - div, rhs_s = -u.grad s.
// This is Eq. 2 with 2 (S.grad lnrho)_i written out from Eq. 3.
#pragma once

#include <type_traits>

#include "tiled_impl.cuh"

namespace gbfd {
namespace tiled2 {

template <class T>
struct V2;
template <>
struct V2<float> {
    using t = float2;
};
template <>
struct V2<double> {
    using t = double2;
};

// Values of one field along x in one row: e[i] = f(x - 4 + i), i = 0..9,
// filled only where loaded.
template <class T>
struct Row {
    T e[10];
};

// Operations on the pair (point x, point x+1).  For FP32 these are the
// packed two-lane instructions of sm_100+ (one instruction, two results);
// for FP64 they fall back to two scalar operations.
template <class T>
struct PairOps;
template <>
struct PairOps<float> {
    using V = float2;
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V bc(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct PairOps<double> {
    using V = double2;
    static __device__ __forceinline__ V fma(V a, V b, V c)
    {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ V bc(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
};

// Shared-memory carve-up of the pipeline.
template <class TS, class TW, int NF, int TX, int TY, int NS, int NW_ = 3>
struct Ring {
    static constexpr int BX = TX + 2 * GX;
    static constexpr int BY = TY + 2 * GY;
    static constexpr int FSTRIDE = BX * BY;
    static constexpr int SLOT_BYTES = NF * FSTRIDE * (int)sizeof(TS);
    static constexpr int SLOT_PITCH = (SLOT_BYTES + 127) / 128 * 128;
    static constexpr int SLOT_ELEMS = SLOT_PITCH / (int)sizeof(TS);
    static constexpr int NW = NW_;
    static constexpr int WSLOT_BYTES = NF * TX * TY * (int)sizeof(TW);
    static constexpr int WSLOT_PITCH = (WSLOT_BYTES + 127) / 128 * 128;
    static constexpr int W_OFF = NS * SLOT_PITCH;
    static constexpr int BAR_OFF = W_OFF + NW * WSLOT_PITCH;
    static constexpr int BYTES = BAR_OFF + (NS + NW) * 8;
};

__device__ __forceinline__ void init_barriers(uint64_t *bars, int n)
{
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int i = 0; i < n; ++i)
            tiled::mbar_init(&bars[i], 1);
        tiled::fence_mbar_init();
    }
    __syncthreads();
}

// One column of one box.  jrun / wrun count the state-plane and u-tilde
// copies this CTA has made before (they continue the barrier phases) and are
// advanced on return.  Returns false when a bounded wait gave up (after
// recording it and draining the copies in flight).
// STG >= 0 fixes the RK3 substep (0, 1, 2) at compile time, FULL says that
// every tile lies inside the grid; both only drop run-time tests.
template <class TS, class TW, class TA, int NF, bool MIXED, int TX, int TY, int NS, bool PK,
          int U, bool WG, bool ICVT = false, bool FORCE = false, class CoefT, int STG = -1,
          bool FULL = false>
__device__ __forceinline__ bool run_column(const CUtensorMap *tmap, const CUtensorMap *wmap,
                                           TS *__restrict__ out, TW *__restrict__ w,
                                           TS *__restrict__ divf, const Layout &Ls,
                                           const Layout &Lw, const CoefT &c, const TA alpha,
                                           const TA beta, const TA dt, const bool first_arg,
                                           const bool last_arg, const int x0, const int y0,
                                           const int z0, const int nout, int &jrun, int &wrun,
                                           unsigned char *smem, int *dev_error,
                                           const int skip_plane = -1,
                                           const Forcing *fo = nullptr)
{
    // WG: u-tilde read straight from global memory (no u-tilde ring)
    static_assert(!WG || PK, "global u-tilde reads only in the packed form");
    using RG = Ring<TS, TW, NF, TX, TY, NS, WG ? 0 : U + 2>;
    using tiled::mbar_wait;
    using V = typename V2<TS>::t;
    using VW = typename V2<TW>::t;
    constexpr int BX = RG::BX, FSTRIDE = RG::FSTRIDE, SLOT_ELEMS = RG::SLOT_ELEMS;
    constexpr int NW = RG::NW;
    constexpr int NTX = TX / 2;
    const TS *sm = reinterpret_cast<const TS *>(smem);
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
    // element offset of point (x, y) in a field of a slot; even, so pairs align
    const int toff = (ty + GY) * BX + (2 * tx + GX);
    const bool need_w = !first;
    // FORCE: the body force of Eq. 2 (Sect. 6); the column's x-y phase factor
    // Re/Im of tx[x] ty[y] for both points, times tz[z] per plane
    float2 fxy0 = make_float2(0.f, 0.f), fxy1 = make_float2(0.f, 0.f);
    if constexpr (FORCE) {
        if (valid0) {
            const float2 a0 = __ldg(fo->tx32 + x), a1 = __ldg(fo->tx32 + x + 1);
            const float2 b = __ldg(fo->ty32 + y);
            fxy0 = make_float2(a0.x * b.x - a0.y * b.y, a0.x * b.y + a0.y * b.x);
            fxy1 = make_float2(a1.x * b.x - a1.y * b.y, a1.x * b.y + a1.y * b.x);
        }
    }

    // every thread is done with the previous column's slots
    __syncthreads();

    // local state plane j is grid plane z0 - 3 + j (wrapped); it is copy
    // jrun + j of this CTA: slot (jrun + j) % NS, phase (jrun + j) / NS
    int issued = 0, wissued = 0;
    auto issue = [&](int j) {
        // fault injection for the bounded-wait test: never copy this plane
        if (j == skip_plane)
            return;
        int z = z0 - R + j;
        z = zplane(Ls, z) + Ls.gz;  // TMA z coordinate
        const int slot = (jrun + j) % NS;
        tiled::mbar_expect_tx(&bars[slot], RG::SLOT_BYTES);
        tiled::tma_load_4d(smem + slot * RG::SLOT_PITCH, tmap, &bars[slot], x0, y0, z, 0);
    };
    auto issue_w = [&](int o) {
        if constexpr (!WG) {
            const int slot = (wrun + o) % NW;
            tiled::mbar_expect_tx(&wbars[slot], RG::WSLOT_BYTES);
            tiled::tma_load_4d(wsm + slot * RG::WSLOT_PITCH, wmap, &wbars[slot], x0 + GX, y0 + GY,
                               z0 + o, 0);
        }
    };
    // The forward-accumulated and 19-point forms read only the centre plane
    // and the arriving plane from shared memory, so the ring need not keep
    // the three planes below the centre (LAG); the unpacked 55-point form
    // reads all seven.
    constexpr bool FWD = PK && MIXED;
    constexpr int LAG = (MIXED && !FWD) ? 0 : R;
    static_assert(NS >= 4 && NS >= (LAG ? U + 3 : U + 6), "ring too short for the planes in use");
    if (threadIdx.x == 0) {
        tiled::fence_proxy_async();
#pragma unroll 1
        for (int j = 0; j < NS && j < nplanes; ++j)
            issue(j);
        issued = min(NS, nplanes);
        if (need_w && !WG) {
#pragma unroll 1
            for (int o = 0; o < NW && o < nout; ++o)
                issue_w(o);
            wissued = min(NW, nout);
        }
    }

    // z-column window of both points: colv[f][k] = (point x, point x+1) of
    // field f at local plane o + k (output plane o - 3 + k), o the first
    // output plane of the current group of U
    constexpr int W = 6 + U;
    V colv[NF][W];

    // Packed 55-point form: the Eq. 8 terms that pair z with x or y,
    //   D_xz f(z) = sum_k MX_k [h_k(z+k) - h_k(z-k)],  h_k = f(x+k) - f(x-k),
    //   D_yz f(z) = sum_k MX_k [g_k(z+k) - g_k(z-k)],  g_k = f(y+k) - f(y-k),
    // are accumulated forward: each plane, when it arrives, adds its h_k /
    // g_k to the pending outputs k planes below and subtracts them from those
    // k planes above.  acx/acy/acz[m] hold the terms of output plane o+m for
    // the x (D_xz u_z), y (D_yz u_z) and z (D_xz u_x + D_yz u_y) components.
    V acx[FWD ? W : 1], acy[FWD ? W : 1], acz[FWD ? W : 1];
    if constexpr (FWD) {
#pragma unroll
        for (int m = 0; m < W; ++m)
            acx[m] = acy[m] = acz[m] = PairOps<TS>::bc((TS)0);
    }
    // plane at element offset `base` (slot + toff), its column values in
    // colv[.][Q + 3]; it is output plane o + Q
    auto absorb = [&](int base, auto qc) {
        if constexpr (FWD) {
            using P = PairOps<TS>;
            constexpr int Q = decltype(qc)::value;
            const V NEG1 = P::bc((TS)-1);
            auto at = [&](int f, int dy, int dx) -> V {
                return *reinterpret_cast<const V *>(sm + base + f * FSTRIDE + dy * BX + dx);
            };
            // x-differences of u_x (field 1) and u_z (field 3)
            V hx[2][3];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int f = u ? 3 : 1;
                const V m4 = at(f, 0, -4), m2 = at(f, 0, -2), p2 = at(f, 0, 2), p4 = at(f, 0, 4);
                const V cc = colv[f][Q + 3];
                hx[u][0] = P::mk(cc.y - m2.y, p2.x - cc.x);
                hx[u][1] = P::fma(m2, NEG1, p2);
                hx[u][2] = P::mk(p2.y - m4.y, p4.x - m2.x);
            }
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                // y-differences of u_y (field 2) and u_z (field 3)
                const V gy = P::fma(at(2, -k, 0), NEG1, at(2, k, 0));
                const V gz = P::fma(at(3, -k, 0), NEG1, at(3, k, 0));
                const V MX1 = P::bc(c.MX(1, k)), MX2 = P::bc(c.MX(2, k));
                const V tx = P::mul(MX1, hx[1][k - 1]);
                const V ty = P::mul(MX2, gz);
                const V tz = P::fma(MX2, gy, P::mul(MX1, hx[0][k - 1]));
                if (Q - k >= 0) {
                    acx[Q - k] = P::add(acx[Q - k], tx);
                    acy[Q - k] = P::add(acy[Q - k], ty);
                    acz[Q - k] = P::add(acz[Q - k], tz);
                }
                if (Q + k < W) {
                    acx[Q + k] = P::fma(tx, NEG1, acx[Q + k]);
                    acy[Q + k] = P::fma(ty, NEG1, acy[Q + k]);
                    acz[Q + k] = P::fma(tz, NEG1, acz[Q + k]);
                }
            }
        }
    };

    bool timeout = false;
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        if (j == NS) {
            // a ring shorter than the six leading planes: the first ones are
            // consumed, their slots take the rest
            __syncthreads();
            if (threadIdx.x == 0) {
                tiled::fence_proxy_async();
#pragma unroll 1
                for (int jj = NS; jj < 2 * R; ++jj)
                    issue(jj);
                issued = 2 * R;
            }
        }
        const int q = jrun + j;
        if (!mbar_wait(&bars[q % NS], (q / NS) & 1))
            timeout = true;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            colv[f][j] = *reinterpret_cast<const V *>(sm + (q % NS) * SLOT_ELEMS + f * FSTRIDE + toff);
        }
        if constexpr (FWD) {
            const int base = (q % NS) * SLOT_ELEMS + toff;
            switch (j) {
            case 0: absorb(base, std::integral_constant<int, -3>{}); break;
            case 1: absorb(base, std::integral_constant<int, -2>{}); break;
            case 2: absorb(base, std::integral_constant<int, -1>{}); break;
            case 3: absorb(base, std::integral_constant<int, 0>{}); break;
            case 4: absorb(base, std::integral_constant<int, 1>{}); break;
            default: absorb(base, std::integral_constant<int, 2>{}); break;
            }
        }
    }

    // global offsets of point (x, y, z0): advanced by one plane per iteration
    long long go_s = (long long)z0 * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
    long long go_w = (long long)z0 * Lw.plane + (long long)(y + GY) * Lw.P + (x + GX);
    // periodic ghost copies this thread's points own (x even, nx % 4 == 0:
    // both points share the x-ghost condition)
    long long gdx = 0, gdy = 0;
    if (x < GX)
        gdx = Ls.nx;
    else if (x >= Ls.nx - GX)
        gdx = -Ls.nx;
    if (y < GY)
        gdy = (long long)Ls.ny * Ls.P;
    else if (y >= Ls.ny - GY)
        gdy = -(long long)Ls.ny * Ls.P;

    int waited = 2 * R, wwaited = 0;
    int slot0 = jrun % NS;  // slot of local plane oo (the output plane being computed)

    // output plane oo = o + S of the current group
    auto plane = [&](const int oo, auto sc) {
        constexpr int S = decltype(sc)::value;
        auto C = [&](int f, int k) -> V & { return colv[f][S + k]; };
        const int qn = jrun + oo + 2 * R;
        if (!mbar_wait(&bars[qn % NS], (qn / NS) & 1))
            timeout = true;
        waited = oo + 2 * R + 1;
        V wg[WG ? NF : 1];
        (void)wg;
        if constexpr (WG) {
            // u-tilde of this plane from global memory, issued before the
            // stencil work so its latency overlaps it
            if (need_w && valid0) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    wg[f] = *reinterpret_cast<const V *>(w + f * Lw.fpitch + go_w);
            }
        } else if (need_w) {
            const int qw = wrun + oo;
            if (!mbar_wait(&wbars[qw % NW], (qw / NW) & 1))
                timeout = true;
            wwaited = oo + 1;
        }
        int so[7];  // element offsets of the slots of local planes oo..oo+6
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            // slot0 < NS and NS >= 4, so two wraps cover k <= 6
            int sl = slot0 + k;
            sl = sl >= NS ? sl - NS : sl;
            sl = sl >= NS ? sl - NS : sl;
            so[k] = sl * SLOT_ELEMS + toff;
        }
        slot0 = slot0 + 1 == NS ? 0 : slot0 + 1;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            C(f, 6) = *reinterpret_cast<const V *>(sm + so[6] + f * FSTRIDE);
        }
        absorb(so[6], std::integral_constant<int, S + 3>{});

            // pair of field f at plane offset dz, row offset dy, x offset dx (even)
            auto ld2 = [&](int f, int dz, int dy, int dx) -> V {
                return *reinterpret_cast<const V *>(sm + so[dz + 3] + f * FSTRIDE + dy * BX + dx);
            };
            // the x row of field f at (dz, dy): pairs at -4, -2, 2, 4 (+ centre)
            auto row = [&](int f, int dz, int dy, bool centre, bool outer) {
                Row<TS> r;
                V a;
                if (outer) {
                    a = ld2(f, dz, dy, -4);
                    r.e[0] = a.x;
                    r.e[1] = a.y;
                }
                a = ld2(f, dz, dy, -2);
                r.e[2] = a.x;
                r.e[3] = a.y;
                if (centre) {
                    a = ld2(f, dz, dy, 0);
                    r.e[4] = a.x;
                    r.e[5] = a.y;
                }
                a = ld2(f, dz, dy, 2);
                r.e[6] = a.x;
                r.e[7] = a.y;
                if (outer) {
                    a = ld2(f, dz, dy, 4);
                    r.e[8] = a.x;
                    r.e[9] = a.y;
                }
                return r;
            };

            if constexpr (PK) {
                // stencil arithmetic in TS on point pairs (packed FP32x2 for
                // FP32, pairs of scalar operations for FP64); the Eq. 10
                // update in TA, u-tilde stored as TW: in TS when all three
                // agree, else the precision form (FP32 storage, FP64 update)
                constexpr bool UP32 = std::is_same<TA, TS>::value && std::is_same<TW, TS>::value;
                static_assert(UP32 || std::is_same<TS, float>::value,
                              "FP64 update only with FP32 storage");
                using P = PairOps<TS>;
                if (valid0) {
                    const int zo = z0 + oo;
                    const V NEG1 = P::bc((TS)-1);
                    VW wv[NF];
                    if constexpr (WG) {
    #pragma unroll
                        for (int f = 0; f < NF; ++f)
                            wv[f] = wg[f];
                    } else if (need_w) {
                        const TW *ws = reinterpret_cast<const TW *>(wsm + ((wrun + oo) % NW) * RG::WSLOT_PITCH) +
                                       ty * TX + 2 * tx;
    #pragma unroll
                        for (int f = 0; f < NF; ++f)
                            wv[f] = *reinterpret_cast<const VW *>(ws + f * TX * TY);
                    }
                    // first (and second) derivatives of field f along x, y, z:
                    // x per point from the loaded row, y and z on the pair
                    V g[3], d2[3];
                    auto axial = [&](int f, bool second) {
                        // the x row as pairs at -4, -2, 0, +2, +4: the +-2
                        // arms of both points line up with the pairs (packed),
                        // the odd +-1 and +-3 arms do not (per point)
                        const V m4 = ld2(f, 0, 0, -4), m2 = ld2(f, 0, 0, -2);
                        const V p2 = ld2(f, 0, 0, 2), p4 = ld2(f, 0, 0, 4);
                        const V cc = C(f, 3);
                        const TS e1 = m4.y, e2 = m2.x, e3 = m2.y, e4 = cc.x, e5 = cc.y;
                        const TS e6 = p2.x, e7 = p2.y, e8 = p4.x;
                        const V ax = P::mk(c.D1(0, 1) * (e5 - e3) + c.D1(0, 3) * (e7 - e1),
                                           c.D1(0, 1) * (e6 - e4) + c.D1(0, 3) * (e8 - e2));
                        g[0] = P::fma(P::bc(c.D1(0, 2)), P::fma(m2, NEG1, p2), ax);
                        if (second) {
                            const V bx = P::mk(c.D2c(0) * e4 + c.D2(0, 1) * (e5 + e3) + c.D2(0, 3) * (e7 + e1),
                                               c.D2c(0) * e5 + c.D2(0, 1) * (e6 + e4) + c.D2(0, 3) * (e8 + e2));
                            d2[0] = P::fma(P::bc(c.D2(0, 2)), P::add(p2, m2), bx);
                        }
                        V gy, by, gz, bz;
    #pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const V yp = ld2(f, 0, k, 0), ym = ld2(f, 0, -k, 0);
                            const V zp = C(f, 3 + k), zm = C(f, 3 - k);
                            const V dyv = P::fma(ym, NEG1, yp), dzv = P::fma(zm, NEG1, zp);
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
                    // Eq. 8 in the (x, y) plane: D_xy f = sum_k MX_k [h_k(y+k) - h_k(y-k)]
                    // with h_k the x-difference f(x+k) - f(x-k) of a row; h_2 is
                    // packed, h_1 and h_3 straddle the pairs
                    auto mix_xy = [&](int f) -> V {
                        V a;
    #pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            V h[2];
    #pragma unroll
                            for (int sgn = 0; sgn < 2; ++sgn) {
                                const int dy = sgn ? -k : k;
                                const V m2 = ld2(f, 0, dy, -2), p2 = ld2(f, 0, dy, 2);
                                if (k == 1) {
                                    const V cc = ld2(f, 0, dy, 0);
                                    h[sgn] = P::mk(cc.y - m2.y, p2.x - cc.x);
                                } else if (k == 2) {
                                    h[sgn] = P::fma(m2, NEG1, p2);
                                } else {
                                    const V m4 = ld2(f, 0, dy, -4), p4 = ld2(f, 0, dy, 4);
                                    h[sgn] = P::mk(p2.y - m4.y, p4.x - m2.x);
                                }
                            }
                            const V d = P::fma(h[1], NEG1, h[0]);
                            a = k == 1 ? P::mul(P::bc(c.MX(0, k)), d) : P::fma(P::bc(c.MX(0, k)), d, a);
                        }
                        return a;
                    };
                    const V NU = P::bc(c.nu), NU3 = P::bc(c.nu3);
                    const V uc[3] = {C(1, 3), C(2, 3), C(3, 3)};
                    V acc[4], gl[3];
                    V dv = P::bc((TS)0);
                    axial(0, false);
                    gl[0] = g[0];
                    gl[1] = g[1];
                    gl[2] = g[2];
    #pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        axial(1 + i, true);
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
                        if (MIXED)
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
                        if (MIXED) {
                            // D_ij u_i enters d_j (div u) for j != i; the pairs
                            // with z come from the forward accumulators
                            if (i == 0)
                                acc[2] = P::fma(NU3, mix_xy(1), acc[2]);  // D_xy u_x -> y
                            else if (i == 1)
                                acc[1] = P::fma(NU3, mix_xy(2), acc[1]);  // D_xy u_y -> x
                        }
                    }
                    if constexpr (MIXED) {
                        acc[1] = P::fma(NU3, acx[S], acc[1]);  // D_xz u_z
                        acc[2] = P::fma(NU3, acy[S], acc[2]);  // D_yz u_z
                        acc[3] = P::fma(NU3, acz[S], acc[3]);  // D_xz u_x + D_yz u_y
                    }
                    V rs = P::bc((TS)0);
                    if (NF == 5) {
                        axial(4, false);
                        V t = P::mul(uc[0], g[0]);
                        t = P::fma(uc[1], g[1], t);
                        t = P::fma(uc[2], g[2], t);
                        rs = P::mul(t, NEG1);
                    }
                    {
                        V ug = P::mul(uc[0], gl[0]);
                        ug = P::fma(uc[1], gl[1], ug);
                        ug = P::fma(uc[2], gl[2], ug);
                        acc[0] = P::mul(P::add(ug, dv), NEG1);
                        const V NCS2 = P::bc(-c.cs2);
                        const V t = P::mul(P::bc(-c.nu23), dv);
    #pragma unroll
                        for (int a = 0; a < 3; ++a)
                            acc[1 + a] = P::fma(t, gl[a], P::fma(NCS2, gl[a], acc[1 + a]));
                    }
                    if (!MIXED) {
                        const long long gi = (long long)zo * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
                        *reinterpret_cast<V *>(divf + gi) = dv;
                        if (gdx)
                            *reinterpret_cast<V *>(divf + gi + gdx) = dv;
                        if (gdy) {
                            *reinterpret_cast<V *>(divf + gi + gdy) = dv;
                            if (gdx)
                                *reinterpret_cast<V *>(divf + gi + gdy + gdx) = dv;
                        }
                    }
                    if constexpr (FORCE) {
                        // f_i = amp_i cos(k.x + phi)
                        const float2 cz = __ldg(fo->tz32 + zo);
                        const float czr = cz.x, czi = cz.y;
                        const V fc = P::mk(fxy0.x * czr - fxy0.y * czi, fxy1.x * czr - fxy1.y * czi);
    #pragma unroll
                        for (int a = 0; a < 3; ++a)
                            acc[1 + a] = P::fma(P::bc(fo->amp32[a]), fc, acc[1 + a]);
                    }
    #pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const V r = f < 4 ? acc[f] : rs;
                        V o2;
                        if constexpr (UP32) {
                            const V DT = P::bc(dt), ALPHA = P::bc(alpha), BETA = P::bc(beta);
                            const V wn = first ? P::mul(DT, r) : P::fma(DT, r, P::mul(ALPHA, wv[f]));
                            o2 = P::fma(BETA, wn, C(f, 3));
                            if (!last)
                                *reinterpret_cast<V *>(w + f * Lw.fpitch + go_w) = wn;
                        } else {
                            // Eq. 10 in TA for both points (the precision form)
                            static_assert(std::is_same<TA, double>::value, "FP64 update");
                            TW wo[2] = {first ? (TW)0 : wv[f].x, first ? (TW)0 : wv[f].y};
                            TS on[2];
                            rk3_update_f64<ICVT, TW>(first, alpha, beta, dt, r.x, C(f, 3).x, wo[0], on[0]);
                            rk3_update_f64<ICVT, TW>(first, alpha, beta, dt, r.y, C(f, 3).y, wo[1], on[1]);
                            o2 = make_float2(on[0], on[1]);
                            if (!last) {
                                VW t;
                                t.x = wo[0];
                                t.y = wo[1];
                                *reinterpret_cast<VW *>(w + f * Lw.fpitch + go_w) = t;
                            }
                        }
                        TS *op = out + f * Ls.fpitch + go_s;
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
            } else {
                if (valid0) {
                    const int zo = z0 + oo;
                    TW wv[NF][2];
                    if (need_w) {
                        const TW *ws = reinterpret_cast<const TW *>(wsm + ((wrun + oo) % NW) * RG::WSLOT_PITCH) +
                                       ty * TX + 2 * tx;
        #pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const VW t = *reinterpret_cast<const VW *>(ws + f * TX * TY);
                            wv[f][0] = t.x;
                            wv[f][1] = t.y;
                        }
                    }

                    // first derivatives along x, y, z of field f for both points, plus
                    // second derivatives when `second`; centre values from C(f, 3)
                    TS g[2][3], d2[2][3];
                    auto axial = [&](int f, bool second) {
                        Row<TS> r0 = row(f, 0, 0, false, true);
                        r0.e[4] = C(f, 3).x;
                        r0.e[5] = C(f, 3).y;
                        V yp[3], ym[3];
        #pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            yp[k - 1] = ld2(f, 0, k, 0);
                            ym[k - 1] = ld2(f, 0, -k, 0);
                        }
        #pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const TS cc = j ? C(f, 3).y : C(f, 3).x;
                            TS ax = (TS)0, ay = (TS)0, az = (TS)0;
                            TS bx = c.D2c(0) * cc, by = c.D2c(1) * cc, bz = c.D2c(2) * cc;
        #pragma unroll
                            for (int k = 1; k <= 3; ++k) {
                                const TS xp = r0.e[4 + j + k], xm = r0.e[4 + j - k];
                                const TS ypv = j ? yp[k - 1].y : yp[k - 1].x;
                                const TS ymv = j ? ym[k - 1].y : ym[k - 1].x;
                                const TS zp = j ? C(f, 3 + k).y : C(f, 3 + k).x;
                                const TS zm = j ? C(f, 3 - k).y : C(f, 3 - k).x;
                                ax += c.D1(0, k) * (xp - xm);
                                ay += c.D1(1, k) * (ypv - ymv);
                                az += c.D1(2, k) * (zp - zm);
                                if (second) {
                                    bx += c.D2(0, k) * (xp + xm);
                                    by += c.D2(1, k) * (ypv + ymv);
                                    bz += c.D2(2, k) * (zp + zm);
                                }
                            }
                            g[j][0] = ax;
                            g[j][1] = ay;
                            g[j][2] = az;
                            d2[j][0] = bx;
                            d2[j][1] = by;
                            d2[j][2] = bz;
                        }
                    };
                    // Eq. 8 in the (x, y) plane (in_y) or the (x, z) plane: rows or
                    // planes at +-k, x offsets +-k, for both points
                    auto mix_x = [&](int f, bool in_y, TS *res) {
                        Row<TS> rp[3], rm[3];
        #pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const int dz = in_y ? 0 : k, dy = in_y ? k : 0;
                            rp[k - 1] = row(f, dz, dy, false, k == 3);
                            rm[k - 1] = row(f, -dz, -dy, false, k == 3);
                        }
                        // k = 1 also needs the centre pair: x+1 for point 0, x for point 1
                        if (in_y) {
                            V a = ld2(f, 0, 1, 0);
                            rp[0].e[4] = a.x;
                            rp[0].e[5] = a.y;
                            a = ld2(f, 0, -1, 0);
                            rm[0].e[4] = a.x;
                            rm[0].e[5] = a.y;
                        } else {
                            rp[0].e[4] = C(f, 4).x;
                            rp[0].e[5] = C(f, 4).y;
                            rm[0].e[4] = C(f, 2).x;
                            rm[0].e[5] = C(f, 2).y;
                        }
        #pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            TS a = (TS)0;
        #pragma unroll
                            for (int k = 1; k <= 3; ++k) {
                                const TS pp = rp[k - 1].e[4 + j + k], mp = rp[k - 1].e[4 + j - k];
                                const TS mm = rm[k - 1].e[4 + j - k], pm = rm[k - 1].e[4 + j + k];
                                a += c.MX(in_y ? 0 : 1, k) * ((pp - mp) + (mm - pm));
                            }
                            res[j] = a;
                        }
                    };
                    // Eq. 8 in the (y, z) plane: pairs at (dz, dy) = (+-k, +-k)
                    auto mix_yz = [&](int f, TS *res) {
                        TS a0 = (TS)0, a1 = (TS)0;
        #pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const V pp = ld2(f, k, k, 0), mp = ld2(f, k, -k, 0);
                            const V mm = ld2(f, -k, -k, 0), pm = ld2(f, -k, k, 0);
                            a0 += c.MX(2, k) * ((pp.x - mp.x) + (mm.x - pm.x));
                            a1 += c.MX(2, k) * ((pp.y - mp.y) + (mm.y - pm.y));
                        }
                        res[0] = a0;
                        res[1] = a1;
                    };

                    TS uc[2][3], gl[2][3], acc[2][4], dv[2];
        #pragma unroll
                    for (int j = 0; j < 2; ++j) {
        #pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            uc[j][i] = j ? C(1 + i, 3).y : C(1 + i, 3).x;
                            acc[j][1 + i] = (TS)0;
                        }
                        dv[j] = (TS)0;
                    }
                    // grad lnrho
                    axial(0, false);
        #pragma unroll
                    for (int j = 0; j < 2; ++j)
        #pragma unroll
                        for (int a = 0; a < 3; ++a)
                            gl[j][a] = g[j][a];
                    // velocity components
        #pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        axial(1 + i, true);
        #pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const TS adv = uc[j][0] * g[j][0] + uc[j][1] * g[j][1] + uc[j][2] * g[j][2];
                            const TS lap = d2[j][0] + d2[j][1] + d2[j][2];
                            const TS sg = g[j][0] * gl[j][0] + g[j][1] * gl[j][1] + g[j][2] * gl[j][2];
                            acc[j][1 + i] += c.nu * (lap + sg) - adv;
                            if (MIXED)
                                acc[j][1 + i] += c.nu3 * d2[j][i];
        #pragma unroll
                            for (int a = 0; a < 3; ++a)
                                acc[j][1 + a] += c.nu * g[j][a] * gl[j][i];
                            dv[j] += g[j][i];
                        }
                        if (MIXED) {
                            // D_ij u_i enters d_j (div u) for j != i
                            TS m[2];
                            if (i == 0) {
                                mix_x(1, true, m);  // D_xy u_x -> y
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][2] += c.nu3 * m[j];
                                mix_x(1, false, m);  // D_xz u_x -> z
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][3] += c.nu3 * m[j];
                            } else if (i == 1) {
                                mix_x(2, true, m);  // D_xy u_y -> x
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][1] += c.nu3 * m[j];
                                mix_yz(2, m);  // D_yz u_y -> z
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][3] += c.nu3 * m[j];
                            } else {
                                mix_x(3, false, m);  // D_xz u_z -> x
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][1] += c.nu3 * m[j];
                                mix_yz(3, m);  // D_yz u_z -> y
        #pragma unroll
                                for (int j = 0; j < 2; ++j)
                                    acc[j][2] += c.nu3 * m[j];
                            }
                        }
                    }
                    TS rs[2] = {(TS)0, (TS)0};
                    if (NF == 5) {
                        axial(4, false);
        #pragma unroll
                        for (int j = 0; j < 2; ++j)
                            rs[j] = -(uc[j][0] * g[j][0] + uc[j][1] * g[j][1] + uc[j][2] * g[j][2]);
                    }
        #pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        acc[j][0] = -(uc[j][0] * gl[j][0] + uc[j][1] * gl[j][1] + uc[j][2] * gl[j][2]) - dv[j];
        #pragma unroll
                        for (int a = 0; a < 3; ++a)
                            acc[j][1 + a] += -c.cs2 * gl[j][a] - c.nu23 * dv[j] * gl[j][a];
                    }
                    if (!MIXED) {
                        V dvv;
                        dvv.x = dv[0];
                        dvv.y = dv[1];
                        const long long gi = (long long)zo * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
                        *reinterpret_cast<V *>(divf + gi) = dvv;
                        if (gdx)
                            *reinterpret_cast<V *>(divf + gi + gdx) = dvv;
                        if (gdy) {
                            *reinterpret_cast<V *>(divf + gi + gdy) = dvv;
                            if (gdx)
                                *reinterpret_cast<V *>(divf + gi + gdy + gdx) = dvv;
                        }
                    }
        #pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        TS ov[2];
                        TW wn[2];
        #pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const TS r = f < 4 ? acc[j][f] : rs[j];
                            TW wo = first ? (TW)0 : wv[f][j];
                            rk3_update<TA, TW, TS>(first, alpha, beta, dt, (TA)r,
                                                   j ? C(f, 3).y : C(f, 3).x, wo, ov[j]);
                            wn[j] = wo;
                        }
                        if (!last) {
                            VW t;
                            t.x = wn[0];
                            t.y = wn[1];
                            *reinterpret_cast<VW *>(w + f * Lw.fpitch + go_w) = t;
                        }
                        V o2;
                        o2.x = ov[0];
                        o2.y = ov[1];
                        TS *op = out + f * Ls.fpitch + go_s;
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
            }
        go_s += Ls.plane;
        go_w += Lw.plane;
    };

#pragma unroll 1
    for (int o = 0; o < nout; o += U) {
        // all threads are done with the previous group: the slots of planes
        // below the oldest one still read are free, and a timeout seen by
        // any thread ends the CTA for everyone
        if (__syncthreads_or(timeout))
            break;
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            const int jend = min(o + LAG + NS, nplanes);
#pragma unroll 1
            for (int j = issued; j < jend; ++j)
                issue(j);
            issued = max(issued, jend);
            if (need_w && !WG) {
                const int tend = min(o + NW, nout);
#pragma unroll 1
                for (int t = wissued; t < tend; ++t)
                    issue_w(t);
                wissued = max(wissued, tend);
            }
        }
        plane(o, std::integral_constant<int, 0>{});
        if constexpr (U > 1) {
            if (o + 1 < nout)
                plane(o + 1, std::integral_constant<int, 1>{});
        }
        if constexpr (U > 2) {
            if (o + 2 < nout)
                plane(o + 2, std::integral_constant<int, 2>{});
        }
        static_assert(U >= 1 && U <= 3, "one to three output planes per iteration");
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                colv[f][k] = colv[f][k + U];
        if constexpr (FWD) {
#pragma unroll
            for (int m = 0; m < W; ++m) {
                acx[m] = m + U < W ? acx[m + U] : PairOps<TS>::bc((TS)0);
                acy[m] = m + U < W ? acy[m + U] : PairOps<TS>::bc((TS)0);
                acz[m] = m + U < W ? acz[m + U] : PairOps<TS>::bc((TS)0);
            }
        }
    }
    const bool bad = __syncthreads_or(timeout);
    if (bad && threadIdx.x == 0) {
        atomicExch(dev_error, 1);
        // drain the copies still in flight into this CTA's shared memory
        // (the copy that fault injection skipped never lands: not waited for)
        for (int j = waited; j < issued; ++j)
            if (j != skip_plane)
                (void)mbar_wait(&bars[(jrun + j) % NS], ((jrun + j) / NS) & 1);
        if constexpr (!WG) {
            for (int o = wwaited; o < wissued; ++o)
                (void)mbar_wait(&wbars[(wrun + o) % NW], ((wrun + o) / NW) & 1);
        }
    }
    jrun += nplanes;
    wrun += need_w ? nout : 0;
    return !bad;
}

// Single box: one CTA per (tile, z-chunk).
template <class TS, class TW, class TA, int NF, bool MIXED, int TX, int TY, int NS, bool PK, int U,
          int MINB, bool WG, bool ICVT, bool FORCE, class CoefT = Coef<TS>, int STG = -1,
          bool FULL = false>
__global__ void __launch_bounds__((TX / 2) * TY, MINB) k_substep_px2(
    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap wmap,
    TS *__restrict__ out, TW *__restrict__ w, TS *__restrict__ divf, const Layout Ls,
    const Layout Lw, const CoefT c, const RKStage st, const int zc, const int tiles_x,
    int *__restrict__ dev_error, const int skip_plane)
{
    using RG = Ring<TS, TW, NF, TX, TY, NS, WG ? 0 : U + 2>;
    extern __shared__ __align__(128) unsigned char smem[];
    init_barriers(reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF), NS + RG::NW);
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nout = min(zc, Ls.nz - z0);
    int jrun = 0, wrun = 0;
    run_column<TS, TW, TA, NF, MIXED, TX, TY, NS, PK, U, WG, ICVT, FORCE, CoefT, STG, FULL>(
        &tmap, &wmap, out, w, divf, Ls, Lw, c,
                                                  (TA)st.alpha, (TA)st.beta, (TA)st.dt,
                                                  st.first != 0, st.last != 0, x0, y0, z0, nout,
                                                  jrun, wrun, smem, dev_error,
                                                  blockIdx.x == 0 && blockIdx.y == 0 ? skip_plane : -1, &st.fo);
}

}  // namespace tiled2

// ISO_OK (bit 0: 19-point form, bit 1: 55-point form): with equal spacing on
// every axis, launch the instantiation that takes the isotropic weights
// (CubicCoef: 10 stencil weights instead of 30).
template <class TS, class TW, class TA, int TX, int TY, int NS, bool PK = false, int U = 1,
          int MINB = 1, bool WG = false, bool ICVT = false, bool FORCE_OK = false,
          int ISO_OK = 0>
cudaError_t launch_px2_cfg(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                           int form, int zc, int cfg_key, int *dev_error, TmapCache *cache,
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
    TS *out = (TS *)b.out;
    TW *w = (TW *)b.w;
    TS *divf = (TS *)b.div;
    cudaError_t e;
    // a forced step needs the forcing instantiation (FORCE_OK variants only)
    if (st.fo.on && !FORCE_OK)
        return cudaErrorNotSupported;
    const bool iso = ISO_OK != 0 && coef_is_cubic(c);
    const CubicCoef<TS> cc = cubic_of(c);
#define GBFD_LAUNCH2_KC(NFV, MIX, FRC, CT, CV)                                                    \
    do {                                                                                          \
        auto kern = tiled2::k_substep_px2<TS, TW, TA, NFV, MIX, TX, TY, NS, PK, U, MINB, WG,     \
                                          ICVT, FRC, CT>;                                         \
        constexpr int sm = tiled2::Ring<TS, TW, NFV, TX, TY, NS, WG ? 0 : U + 2>::BYTES;          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, *wmap, out, w, divf, b.Ls, b.Lw, CV, st, zc,      \
                                          tiles_x, dev_error, skip_plane);                        \
    } while (0)
#define GBFD_LAUNCH2_K(NFV, MIX, FRC)                                                             \
    do {                                                                                          \
        if constexpr ((ISO_OK & ((MIX) ? 2 : 1)) != 0) {                                          \
            if (iso) {                                                                            \
                GBFD_LAUNCH2_KC(NFV, MIX, FRC, CubicCoef<TS>, cc);                                \
                break;                                                                            \
            }                                                                                     \
        }                                                                                         \
        GBFD_LAUNCH2_KC(NFV, MIX, FRC, Coef<TS>, c);                                              \
    } while (0)
#define GBFD_LAUNCH2(NFV, MIX)                                                                    \
    do {                                                                                          \
        if constexpr (FORCE_OK) {                                                                 \
            if (st.fo.on) {                                                                       \
                GBFD_LAUNCH2_K(NFV, MIX, true);                                                   \
                break;                                                                            \
            }                                                                                     \
        }                                                                                         \
        GBFD_LAUNCH2_K(NFV, MIX, false);                                                          \
    } while (0)
    // the 19-point form's first pass in FP32, five fields (forced or not),
    // equal spacing, whole tiles: the substep is a template argument and the
    // grid-extent test goes (one instantiation per RK3 substep)
    constexpr bool SPEC = PK && !WG && !ICVT && (ISO_OK & 1) != 0 &&
                          std::is_same<TS, float>::value && std::is_same<TW, float>::value &&
                          std::is_same<TA, float>::value;
    if constexpr (SPEC) {
        if (form == 1 && nf == 5 && iso && b.Ls.nx % TX == 0 && b.Ls.ny % TY == 0 &&
            st.s >= 0 && st.s <= 2) {
#define GBFD_LAUNCH2_S(FRC, SV)                                                                   \
    do {                                                                                          \
        auto kern = tiled2::k_substep_px2<TS, TW, TA, 5, false, TX, TY, NS, PK, U, MINB, WG,     \
                                          ICVT, FRC, CubicCoef<TS>, SV, true>;                    \
        constexpr int sm = tiled2::Ring<TS, TW, 5, TX, TY, NS, U + 2>::BYTES;                     \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, *wmap, out, w, divf, b.Ls, b.Lw, cc, st, zc,      \
                                          tiles_x, dev_error, skip_plane);                        \
    } while (0)
#define GBFD_LAUNCH2_SS(FRC)                                                                      \
    do {                                                                                          \
        if (st.s == 0)                                                                            \
            GBFD_LAUNCH2_S(FRC, 0);                                                               \
        else if (st.s == 1)                                                                       \
            GBFD_LAUNCH2_S(FRC, 1);                                                               \
        else                                                                                      \
            GBFD_LAUNCH2_S(FRC, 2);                                                               \
    } while (0)
            if (!st.fo.on) {
                GBFD_LAUNCH2_SS(false);
            } else {
                // FORCE_OK: the forced step was accepted above
                if constexpr (FORCE_OK)
                    GBFD_LAUNCH2_SS(true);
            }
#undef GBFD_LAUNCH2_SS
#undef GBFD_LAUNCH2_S
            *launches += 1;
            return cudaGetLastError();
        }
    }
    if (form == 0) {
        if (nf == 5)
            GBFD_LAUNCH2(5, true);
        else
            GBFD_LAUNCH2(4, true);
    } else {
        if (nf == 5)
            GBFD_LAUNCH2(5, false);
        else
            GBFD_LAUNCH2(4, false);
    }
#undef GBFD_LAUNCH2
#undef GBFD_LAUNCH2_K
#undef GBFD_LAUNCH2_KC
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
