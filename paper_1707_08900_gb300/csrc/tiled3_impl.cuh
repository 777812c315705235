// Tiled fused 55-point substep in FP32 with the in-plane stencil work done
// when a plane arrives and its results carried to the output plane through
// tensor memory (TMEM).
//
// Pipeline of one CTA over one column (tile x0..x0+TX, y0..y0+TY, output
// planes z0..z0+nout), two points per thread (x, x+1), packed FP32x2
// arithmetic:
// * each z-plane of all NF fields, tile plus 3-cell halo, arrives by one 4D
//   TMA copy into a ring of NS shared-memory slots; u-tilde of the output
//   plane arrives by a second ring;
// * when plane p arrives, every thread reads its x rows and y rows from
//   shared memory ONCE and forms from them
//     - the x and y first derivatives of every field and the x and y second
//       derivatives of the velocity (Eqs. 6-7),
//     - the (x, y) cross derivatives of u_x and u_y (Eq. 8),
//     - the per-plane differences h_k = f(x+k) - f(x-k), g_k = f(y+k) -
//       f(y-k) of the z-paired cross terms, accumulated forward into the
//       register windows of the outputs k planes below and above,
//   and from these the whole part of the right-hand side (Eqs. 1-3) that
//   needs no z derivative; it stores that part and the five in-plane
//   quantities the z part multiplies (20 floats for its two points) into
//   its own TMEM lane (a ring of four plane slots);
// * three planes later plane p is the centre of output plane p: the thread
//   loads them back from TMEM, takes the z derivatives from its register
//   column window, completes the right-hand side and applies the RK3
//   update (Eq. 10).
// Shared memory therefore holds only the arriving planes, and each row of
// the halo box is read once per plane instead of twice.
#pragma once

#include "tcgen05.cuh"
#include "tiled2_impl.cuh"

namespace gbfd {
namespace tiled3 {

using tiled2::PairOps;

// Warp-collective TMEM accesses of the 32x32b shape: each thread moves n
// consecutive 32-bit columns of its own lane.  Each statement also waits for
// its own completion, so the compiler never sees a load's destination (or a
// store's source) registers before the hardware is done with them.
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {"
                 "%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16"
                 "};\n\t"
                 "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
                 : "memory");
}

__device__ __forceinline__ void tm_st4(uint32_t taddr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {"
                 "%1, %2, %3, %4"
                 "};\n\t"
                 "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3]))
                 : "memory");
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, float *v)
{
    uint32_t u[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {"
                 "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15"
                 "}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                   "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]),
                   "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void tm_ld4(uint32_t taddr, float *v)
{
    uint32_t u[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {"
                 "%0, %1, %2, %3"
                 "}, [%4];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i)
        v[i] = __uint_as_float(u[i]);
}


// TMEM columns: per plane slot, for one thread's two points (pairs), the
// part of the right-hand side that needs no z derivative and the in-plane
// quantities the z part multiplies:
//   P_f (f < NF) at 2f, d_x lnrho at 10, d_y lnrho at 12, the in-plane
//   divergence d_x u_x + d_y u_y at 14, d_x u_z at 16, d_y u_z at 18.
// Four slots of 32 columns.
struct TmLayout {
    static constexpr int FLOATS = 20;
    static constexpr int GLX = 10, GLY = 12, DIV = 14, DZX = 16, DZY = 18;
    static constexpr int SLOT_COLS = 32;
    static constexpr int NSLOT = 4;
    static constexpr int COLS = 128;  // allocation: a power of two >= NSLOT * SLOT_COLS
};

// Shared memory: the two-point ring (state slots, u-tilde slots, mbarriers)
// plus the TMEM address written by the allocating warp.
template <int NF, int TX, int TY, int NS>
struct RingTm {
    using RG = tiled2::Ring<float, float, NF, TX, TY, NS, 3>;
    static constexpr int TM_OFF = (RG::BYTES + 15) / 16 * 16;
    static constexpr int BYTES = TM_OFF + 16;
};

template <int NF, int TX, int TY, int NS>
__device__ __forceinline__ bool run_column_tm(const CUtensorMap *tmap, const CUtensorMap *wmap,
                                              float *__restrict__ out, float *__restrict__ w,
                                              const Layout &Ls, const Layout &Lw,
                                              const Coef<float> &c, const float alpha,
                                              const float beta, const float dt, const bool first,
                                              const bool last, const int x0, const int y0,
                                              const int z0, const int nout, int &jrun, int &wrun,
                                              unsigned char *smem, const uint32_t tmem,
                                              int *dev_error, const int skip_plane = -1)
{
    using RG = tiled2::Ring<float, float, NF, TX, TY, NS, 3>;
    using TL = TmLayout;
    using V = float2;
    using P = PairOps<float>;
    using tiled::mbar_wait;
    constexpr int BX = RG::BX, FSTRIDE = RG::FSTRIDE, SLOT_ELEMS = RG::SLOT_ELEMS;
    constexpr int NW = RG::NW;
    constexpr int NTX = TX / 2;
    const float *sm = reinterpret_cast<const float *>(smem);
    unsigned char *wsm = smem + RG::W_OFF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF);
    uint64_t *wbars = bars + NS;

    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const int nz = Ls.nz;
    const int nplanes = nout + 2 * R;
    const int x = x0 + 2 * tx, y = y0 + ty;
    const bool valid0 = (x < Ls.nx) && (y < Ls.ny);  // nx % 4 == 0: x+1 valid with x
    const int toff = (ty + GY) * BX + (2 * tx + GX);
    const bool need_w = !first;
    // this warp's 32 TMEM lanes (one per thread)
    const uint32_t trow = tmem + ((uint32_t)(threadIdx.x & ~31) << 16);

    // every thread is done with the previous column's slots
    __syncthreads();

    int issued = 0, wissued = 0;
    auto issue = [&](int j) {
        // fault injection for the bounded-wait test: never copy this plane
        if (j == skip_plane)
            return;
        int z = z0 - R + j;
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
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
    }

    // z-column window: colv[f][k] = (point x, point x+1) of field f at local
    // plane j - 6 + k during the iteration that receives local plane j
    V colv[NF][7];
    // forward accumulators of the z-paired Eq. 8 terms; position m is output
    // plane (j - 6) + m: x (D_xz u_z), y (D_yz u_z), z (D_xz u_x + D_yz u_y)
    V acx[7], acy[7], acz[7];
#pragma unroll
    for (int m = 0; m < 7; ++m)
        acx[m] = acy[m] = acz[m] = P::bc(0.f);

    // global offsets of point (x, y, z0): advanced by one plane per output
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

    const V NEG1 = P::bc(-1.f);
    bool timeout = false;
    int waited = 0, wwaited = 0;
#pragma unroll 1
    for (int j = 0; j < nplanes; ++j) {
        // all threads are done with plane j-1: its slot is free, and a
        // timeout seen by any thread ends the CTA for everyone
        if (__syncthreads_or(timeout))
            break;
        const int o = j - 2 * R;  // output plane finished in this iteration, if >= 0
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            const int jend = min(j + NS, nplanes);
#pragma unroll 1
            for (int jj = issued; jj < jend; ++jj)
                issue(jj);
            issued = max(issued, jend);
            if (need_w) {
                const int tend = min(o + NW, nout);
#pragma unroll 1
                for (int t = wissued; t < tend; ++t)
                    issue_w(t);
                wissued = max(wissued, tend);
            }
        }
        const int q = jrun + j;
        if (!mbar_wait(&bars[q % NS], (q / NS) & 1))
            timeout = true;
        waited = j + 1;
        const int base = (q % NS) * SLOT_ELEMS + toff;
        auto at = [&](int f, int dy, int dx) -> V {
            return *reinterpret_cast<const V *>(sm + base + f * FSTRIDE + dy * BX + dx);
        };
#pragma unroll
        for (int f = 0; f < NF; ++f)
            colv[f][6] = at(f, 0, 0);

        // ---- arrival of local plane j (output plane j - 3 relative to z0)
        const bool centre = j >= R && j < nout + R;
        const V NU = P::bc(c.nu), NU3 = P::bc(c.nu3);
        {
            // in-plane (x, y) derivatives of each field, combined at once into
            // the part of the right-hand side they fix (Eqs. 1-3 with
            // 2 S.grad lnrho written out); u_x, u_y of this plane are its
            // own column values
            const V ux = colv[1][6], uy = colv[2][6];
            const V NU43 = P::bc(c.nu + c.nu3), NU2 = P::bc(2.f * c.nu);
            V Pf[5], glx, gly, dvxy, dzx, dzy;
            V hxx[3];  // x-differences of u_x, kept for the z-paired term
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const bool vel = f >= 1 && f <= 3;
                const V cc = colv[f][6];
                const bool need_x = centre || f == 1 || f == 3;
                const bool need_y = centre || f == 2 || f == 3;
                V d1x, d1y, d2x, d2y, dxy;
                if (need_x) {
                    const V m4 = at(f, 0, -4), m2 = at(f, 0, -2), p2 = at(f, 0, 2), p4 = at(f, 0, 4);
                    // h_k = f(x+k) - f(x-k) for both points; h_2 lines up
                    // with the pairs, h_1 and h_3 straddle them
                    const V h1 = P::mk(cc.y - m2.y, p2.x - cc.x);
                    const V h2 = P::fma(m2, NEG1, p2);
                    const V h3 = P::mk(p2.y - m4.y, p4.x - m2.x);
                    if (centre) {
                        d1x = P::mul(P::bc(c.D1(0, 1)), h1);
                        d1x = P::fma(P::bc(c.D1(0, 2)), h2, d1x);
                        d1x = P::fma(P::bc(c.D1(0, 3)), h3, d1x);
                        if (vel) {
                            const V s1 = P::mk(cc.y + m2.y, p2.x + cc.x);
                            const V s3 = P::mk(p2.y + m4.y, p4.x + m2.x);
                            d2x = P::mul(P::bc(c.D2c(0)), cc);
                            d2x = P::fma(P::bc(c.D2(0, 1)), s1, d2x);
                            d2x = P::fma(P::bc(c.D2(0, 2)), P::add(p2, m2), d2x);
                            d2x = P::fma(P::bc(c.D2(0, 3)), s3, d2x);
                        }
                    }
                    if (f == 1) {
                        hxx[0] = h1;
                        hxx[1] = h2;
                        hxx[2] = h3;
                    } else if (f == 3) {
                        // D_xz u_z -> x component
                        const V hz[3] = {h1, h2, h3};
#pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const V t = P::mul(P::bc(c.MX(1, k)), hz[k - 1]);
                            acx[3 - k] = P::add(acx[3 - k], t);
                            acx[3 + k] = P::fma(t, NEG1, acx[3 + k]);
                        }
                    }
                }
                if (need_y) {
                    V yp[3], ym[3], gk[3];
#pragma unroll
                    for (int k = 1; k <= 3; ++k) {
                        yp[k - 1] = at(f, k, 0);
                        ym[k - 1] = at(f, -k, 0);
                        gk[k - 1] = P::fma(ym[k - 1], NEG1, yp[k - 1]);
                    }
                    if (centre) {
                        d1y = P::mul(P::bc(c.D1(1, 1)), gk[0]);
                        d1y = P::fma(P::bc(c.D1(1, 2)), gk[1], d1y);
                        d1y = P::fma(P::bc(c.D1(1, 3)), gk[2], d1y);
                        if (vel) {
                            d2y = P::mul(P::bc(c.D2c(1)), cc);
#pragma unroll
                            for (int k = 1; k <= 3; ++k)
                                d2y = P::fma(P::bc(c.D2(1, k)), P::add(yp[k - 1], ym[k - 1]), d2y);
                        }
                        if (f == 1 || f == 2) {
                            // D_xy f = sum_k MX_k [h_k(y+k) - h_k(y-k)], rows y+-k
#pragma unroll
                            for (int k = 1; k <= 3; ++k) {
                                V h[2];
#pragma unroll
                                for (int sg = 0; sg < 2; ++sg) {
                                    const int dy = sg ? -k : k;
                                    const V m2 = at(f, dy, -2), p2 = at(f, dy, 2);
                                    if (k == 1) {
                                        const V ce = sg ? ym[0] : yp[0];
                                        h[sg] = P::mk(ce.y - m2.y, p2.x - ce.x);
                                    } else if (k == 2) {
                                        h[sg] = P::fma(m2, NEG1, p2);
                                    } else {
                                        const V m4 = at(f, dy, -4), p4 = at(f, dy, 4);
                                        h[sg] = P::mk(p2.y - m4.y, p4.x - m2.x);
                                    }
                                }
                                const V dd = P::fma(h[1], NEG1, h[0]);
                                dxy = k == 1 ? P::mul(P::bc(c.MX(0, k)), dd)
                                             : P::fma(P::bc(c.MX(0, k)), dd, dxy);
                            }
                        }
                    }
                    if (f == 2) {
                        // D_xz u_x + D_yz u_y -> z component
#pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const V t = P::fma(P::bc(c.MX(2, k)), gk[k - 1],
                                               P::mul(P::bc(c.MX(1, k)), hxx[k - 1]));
                            acz[3 - k] = P::add(acz[3 - k], t);
                            acz[3 + k] = P::fma(t, NEG1, acz[3 + k]);
                        }
                    } else if (f == 3) {
                        // D_yz u_z -> y component
#pragma unroll
                        for (int k = 1; k <= 3; ++k) {
                            const V t = P::mul(P::bc(c.MX(2, k)), gk[k - 1]);
                            acy[3 - k] = P::add(acy[3 - k], t);
                            acy[3 + k] = P::fma(t, NEG1, acy[3 + k]);
                        }
                    }
                }
                if (centre) {
                    // -u_x d_x f - u_y d_y f: the in-plane advection of every field
                    const V adv = P::fma(uy, d1y, P::mul(ux, d1x));
                    if (f == 0) {
                        glx = d1x;
                        gly = d1y;
                        Pf[0] = P::mul(adv, NEG1);
                    } else if (f == 1) {
                        // u_x: nu (4/3 D_xx + D_yy) u_x (Laplacian and the diagonal of
                        // grad div), nu (2 d_x u_x d_x lnrho + d_y u_x d_y lnrho)
                        Pf[0] = P::fma(d1x, NEG1, Pf[0]);
                        dvxy = d1x;
                        V p = P::fma(NU43, d2x, P::fma(NU, d2y, P::mul(adv, NEG1)));
                        p = P::fma(NU2, P::mul(d1x, glx), p);
                        Pf[1] = P::fma(NU, P::mul(d1y, gly), p);
                        // into u_y: nu d_y u_x d_x lnrho + (nu/3) D_xy u_x
                        Pf[2] = P::fma(NU, P::mul(d1y, glx), P::mul(NU3, dxy));
                    } else if (f == 2) {
                        Pf[0] = P::fma(d1y, NEG1, Pf[0]);
                        dvxy = P::add(dvxy, d1y);
                        V p = P::fma(NU, d2x, P::fma(NU43, d2y, P::fma(adv, NEG1, Pf[2])));
                        p = P::fma(NU, P::mul(d1x, glx), p);
                        Pf[2] = P::fma(NU2, P::mul(d1y, gly), p);
                        // into u_x: nu d_x u_y d_y lnrho + (nu/3) D_xy u_y
                        Pf[1] = P::fma(NU, P::mul(d1x, gly), P::fma(NU3, dxy, Pf[1]));
                    } else if (f == 3) {
                        V p = P::fma(NU, P::add(d2x, d2y), P::mul(adv, NEG1));
                        p = P::fma(NU, P::mul(d1x, glx), p);
                        Pf[3] = P::fma(NU, P::mul(d1y, gly), p);
                        dzx = d1x;
                        dzy = d1y;
                    } else {
                        Pf[4] = P::mul(adv, NEG1);
                    }
                }
            }
            if (centre) {
                // -c_s^2 d_i lnrho - (2/3) nu (d_x u_x + d_y u_y) d_i lnrho, i = x, y
                const V NCS2 = P::bc(-c.cs2), N23 = P::bc(-c.nu23);
                Pf[1] = P::fma(NCS2, glx, P::fma(P::mul(N23, dvxy), glx, Pf[1]));
                Pf[2] = P::fma(NCS2, gly, P::fma(P::mul(N23, dvxy), gly, Pf[2]));
                if (NF == 4)
                    Pf[4] = P::bc(0.f);
                float r[TL::FLOATS];
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    r[2 * f] = Pf[f].x;
                    r[2 * f + 1] = Pf[f].y;
                }
                const V rest[5] = {glx, gly, dvxy, dzx, dzy};
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    r[TL::GLX + 2 * i] = rest[i].x;
                    r[TL::GLX + 2 * i + 1] = rest[i].y;
                }
                // slot j % 4 last held plane j - 4, read in iteration j - 1
                const uint32_t ta = trow + (uint32_t)((j % TL::NSLOT) * TL::SLOT_COLS);
                __syncwarp();  // the TMEM accesses are warp-collective
                tm_st16(ta, r);
                tm_st4(ta + 16, r + 16);
            }
        }

        // ---- output plane o (centre: local plane o + 3, stored 3 iterations ago)
        if (o >= 0) {
            float qv[TL::FLOATS];
            {
                __syncwarp();
                const uint32_t ta = trow + (uint32_t)(((o + R) % TL::NSLOT) * TL::SLOT_COLS);
                tm_ld16(ta, qv);
                tm_ld4(ta + 16, qv + 16);
            }
            V wv[NF];
            if (need_w) {
                const int qw = wrun + o;
                if (!mbar_wait(&wbars[qw % NW], (qw / NW) & 1))
                    timeout = true;
                wwaited = o + 1;
                const float *ws = reinterpret_cast<const float *>(wsm + (qw % NW) * RG::WSLOT_PITCH) +
                                  ty * TX + 2 * tx;
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    wv[f] = *reinterpret_cast<const V *>(ws + f * TX * TY);
            }
            auto pair = [&](int i) { return P::mk(qv[i], qv[i + 1]); };
            // z derivatives from the column window (centre at position 3)
            auto dz1 = [&](int f) {
                V gz;
#pragma unroll
                for (int k = 1; k <= 3; ++k) {
                    const V dzv = P::fma(colv[f][3 - k], NEG1, colv[f][3 + k]);
                    gz = k == 1 ? P::mul(P::bc(c.D1(2, k)), dzv) : P::fma(P::bc(c.D1(2, k)), dzv, gz);
                }
                return gz;
            };
            auto dz2 = [&](int f) {
                V bz = P::mul(P::bc(c.D2c(2)), colv[f][3]);
#pragma unroll
                for (int k = 1; k <= 3; ++k)
                    bz = P::fma(P::bc(c.D2(2, k)), P::add(colv[f][3 + k], colv[f][3 - k]), bz);
                return bz;
            };
            const V uz = colv[3][3];
            const V glx = pair(TL::GLX), gly = pair(TL::GLY);
            const V glz = dz1(0);
            const V gzx = dz1(1), gzy = dz1(2), gzz = dz1(3);
            const V NU2 = P::bc(2.f * c.nu), N23 = P::bc(-c.nu23);
            const V div = P::add(pair(TL::DIV), gzz);
            V rr[5];
            // lnrho: -u_z d_z lnrho - d_z u_z
            rr[0] = P::fma(uz, P::mul(glz, NEG1), P::fma(gzz, NEG1, pair(0)));
            // u_x, u_y: -u_z d_z u_i + nu D_zz u_i + nu (d_z u_i + d_i u_z) d_z lnrho
            //           - (2/3) nu d_z u_z d_i lnrho + (nu/3) (D_iz u_z)
            {
                V p = P::fma(uz, P::mul(gzx, NEG1), pair(2));
                p = P::fma(NU, dz2(1), p);
                p = P::fma(NU, P::mul(P::add(gzx, pair(TL::DZX)), glz), p);
                p = P::fma(P::mul(N23, gzz), glx, p);
                rr[1] = P::fma(NU3, acx[0], p);
            }
            {
                V p = P::fma(uz, P::mul(gzy, NEG1), pair(4));
                p = P::fma(NU, dz2(2), p);
                p = P::fma(NU, P::mul(P::add(gzy, pair(TL::DZY)), glz), p);
                p = P::fma(P::mul(N23, gzz), gly, p);
                rr[2] = P::fma(NU3, acy[0], p);
            }
            // u_z: -u_z d_z u_z - c_s^2 d_z lnrho + (4/3) nu D_zz u_z + (nu/3) (D_xz u_x
            //      + D_yz u_y) + 2 nu d_z u_z d_z lnrho + nu (d_z u_x d_x lnrho
            //      + d_z u_y d_y lnrho) - (2/3) nu div u d_z lnrho
            {
                V p = P::fma(uz, P::mul(gzz, NEG1), pair(6));
                p = P::fma(P::bc(-c.cs2), glz, p);
                p = P::fma(P::bc(c.nu + c.nu3), dz2(3), p);
                p = P::fma(NU3, acz[0], p);
                p = P::fma(NU2, P::mul(gzz, glz), p);
                p = P::fma(NU, P::fma(gzy, gly, P::mul(gzx, glx)), p);
                rr[3] = P::fma(P::mul(N23, div), glz, p);
            }
            if (NF == 5)
                rr[4] = P::fma(uz, P::mul(dz1(4), NEG1), pair(8));
            if (valid0) {
                const V DT = P::bc(dt), ALPHA = P::bc(alpha), BETA = P::bc(beta);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const V wn = first ? P::mul(DT, rr[f]) : P::fma(DT, rr[f], P::mul(ALPHA, wv[f]));
                    const V o2 = P::fma(BETA, wn, colv[f][3]);
                    if (!last)
                        *reinterpret_cast<V *>(w + f * Lw.fpitch + go_w) = wn;
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
        }

        // advance the windows by one plane
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                colv[f][k] = colv[f][k + 1];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            acx[m] = acx[m + 1];
            acy[m] = acy[m + 1];
            acz[m] = acz[m + 1];
        }
        acx[6] = acy[6] = acz[6] = P::bc(0.f);
    }
    const bool bad = __syncthreads_or(timeout);
    if (bad && threadIdx.x == 0) {
        atomicExch(dev_error, 1);
        // drain the copies still in flight into this CTA's shared memory
        for (int j = waited; j < issued; ++j)
            (void)mbar_wait(&bars[(jrun + j) % NS], ((jrun + j) / NS) & 1);
        for (int o = wwaited; o < wissued; ++o)
            (void)mbar_wait(&wbars[(wrun + o) % NW], ((wrun + o) / NW) & 1);
    }
    jrun += nplanes;
    wrun += need_w ? nout : 0;
    return !bad;
}

// TMEM for the CTA: warp 0 allocates and frees; the address is shared.
__device__ __forceinline__ uint32_t tmem_acquire(uint32_t *slot)
{
    if (threadIdx.x < 32)
        tc::tmem_alloc(slot, TmLayout::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *reinterpret_cast<volatile uint32_t *>(slot);
}

__device__ __forceinline__ void tmem_release(uint32_t tmem)
{
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32)
        tc::tmem_dealloc(tmem, TmLayout::COLS);
}

// Single box: one CTA per (tile, z-chunk).
template <int NF, int TX, int TY, int NS>
__global__ void __launch_bounds__((TX / 2) * TY) k_substep_tm(
    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap wmap,
    float *__restrict__ out, float *__restrict__ w, const Layout Ls, const Layout Lw,
    const Coef<float> c, const RKStage st, const int zc, const int tiles_x,
    int *__restrict__ dev_error, const int skip_plane)
{
    using RT = RingTm<NF, TX, TY, NS>;
    using RG = typename RT::RG;
    extern __shared__ __align__(128) unsigned char smem[];
    tiled2::init_barriers(reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF), NS + RG::NW);
    const uint32_t tmem = tmem_acquire(reinterpret_cast<uint32_t *>(smem + RT::TM_OFF));
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nout = min(zc, Ls.nz - z0);
    int jrun = 0, wrun = 0;
    run_column_tm<NF, TX, TY, NS>(&tmap, &wmap, out, w, Ls, Lw, c, (float)st.alpha,
                                  (float)st.beta, (float)st.dt, st.first != 0, st.last != 0, x0,
                                  y0, z0, nout, jrun, wrun, smem, tmem, dev_error,
                                  blockIdx.x == 0 && blockIdx.y == 0 ? skip_plane : -1);
    tmem_release(tmem);
}

}  // namespace tiled3

// Launch of the TMEM-carried 55-point kernel (FP32 storage and arithmetic).
// Each CTA holds 128 TMEM columns, so the four CTAs an SM could hold at most
// fit in its 512 columns and tcgen05.alloc never waits for another CTA.
// (Registers, about 240 per thread, allow two.)
template <int TX, int TY, int NS>
cudaError_t launch_tm_cfg(const StateBufs &b, const Coef<float> &c, const RKStage &st, int nf,
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
    static_assert(4 * tiled3::TmLayout::COLS <= 512, "TMEM columns per CTA");
    cudaError_t e;
#define GBFD_LAUNCH_TM(NFV)                                                                       \
    do {                                                                                          \
        auto kern = tiled3::k_substep_tm<NFV, TX, TY, NS>;                                        \
        constexpr int sm = tiled3::RingTm<NFV, TX, TY, NS>::BYTES;                                \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, *wmap, (float *)b.out, (float *)b.w, b.Ls, b.Lw,  \
                                          c, st, zc, tiles_x, dev_error, skip_plane);             \
    } while (0)
    if (nf == 5)
        GBFD_LAUNCH_TM(5);
    else
        GBFD_LAUNCH_TM(4);
#undef GBFD_LAUNCH_TM
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
