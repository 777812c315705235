// FP64 fused 55-point substep (Algorithm 2), one point per thread, output
// planes finished three planes behind the in-plane work: the scheme of the
// FP32 default (tiled4_impl.cuh) in scalar FP64, where the FP64 pipe, not the
// issue rate, is the bound.
//
// What it changes against the one-point FP64 kernel (tiled_impl.cuh):
//   * fewer FP64 operations.  The Eq. 8 terms that pair z with x or y,
//       D_xz f(z) = sum_k MX_k [h_k(z+k) - h_k(z-k)],  h_k = f(x+k) - f(x-k),
//     take their in-plane differences h_k (and the y differences g_k) from
//     the first-derivative stencils of each plane when it is the centre, and
//     spread them into the running sums of the six output planes around it:
//     6 fused multiply-adds per term and plane instead of 12 operations
//     (3 differences per side, their difference, the weighted sum);
//   * a shorter ring.  A step reads only its centre plane (the in-plane arms)
//     and the plane three above it (its own z-column value), so the ring of
//     full planes holds planes s .. s+3 plus one in flight: 5 slots of
//     13.4 KB (16 x 8 tile, 3-cell halo, 5 fields), three CTAs per SM where
//     the 7-plane ring of the one-point kernel allows two.  u-tilde comes
//     from global memory, loaded at the start of the step that uses it.
// Output plane o waits three planes for its z-paired terms; the rest of its
// right-hand side waits in tensor memory (4 slots, 2 columns per FP64 value).
#pragma once

#include "tcgen05.cuh"
#include "tiled2_impl.cuh"

namespace gbfd {
namespace tiled6 {

constexpr int kTmSlotCols = 16;
constexpr int kTmCols = 4 * kTmSlotCols;

// Shared-memory carve-up: NS full-plane slots, barriers, TMEM address word.
template <int NF, int TX, int TY, int NS>
struct Ring64 {
    static constexpr int BX = TX + 2 * GX;
    static constexpr int BY = TY + 2 * GY;
    static constexpr int FSTRIDE = BX * BY;
    static constexpr int SLOT_BYTES = NF * FSTRIDE * 8;
    static constexpr int SLOT_PITCH = (SLOT_BYTES + 127) / 128 * 128;
    static constexpr int SLOT_ELEMS = SLOT_PITCH / 8;
    static constexpr int BAR_OFF = NS * SLOT_PITCH;
    static constexpr int TM_OFF = (BAR_OFF + NS * 8 + 15) / 16 * 16;
    static constexpr int BYTES = TM_OFF + 16;
};

// The NF FP64 values of one pending slot to / from the thread's TMEM lane
// (value f in columns 2 f, 2 f + 1).  Warp-collective: the warp is
// reconverged first (the bounded mbarrier spins before exit lane by lane).
template <int NF>
__device__ __forceinline__ void tm_put(uint32_t ta, const double *v)
{
    uint32_t u[10];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        u[2 * f] = (uint32_t)__double2loint(v[f]);
        u[2 * f + 1] = (uint32_t)__double2hiint(v[f]);
    }
    __syncwarp();
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
                 "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]),
                 "r"(u[7])
                 : "memory");
    if constexpr (NF == 5)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(ta + 8),
                     "r"(u[8]), "r"(u[9])
                     : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
template <int NF>
__device__ __forceinline__ void tm_get(uint32_t ta, double *v)
{
    uint32_t u[10];
    __syncwarp();
    if constexpr (NF == 5)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%10];\n\t"
                     "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%11];\n\t"
                     "tcgen05.wait::ld.sync.aligned;"
                     : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                       "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9])
                     : "r"(ta), "r"(ta + 8)
                     : "memory");
    else
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                     "tcgen05.wait::ld.sync.aligned;"
                     : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                       "=r"(u[6]), "=r"(u[7])
                     : "r"(ta)
                     : "memory");
#pragma unroll
    for (int f = 0; f < NF; ++f)
        v[f] = __hiloint2double((int)u[2 * f + 1], (int)u[2 * f]);
}

// One CTA per (tile, z-chunk).  Local plane j is grid plane z0 - 3 + j
// (wrapped), j = 0 .. nout + 5; step s (s = 3 .. nout + 2) takes the value of
// plane s + 3 on the thread's z-column, does the centre work of plane s
// (output plane s - 3) and finishes output plane s - 6.
template <int NF, int TX, int TY, int NS, int MINB, bool FORCE, class CoefT>
__global__ void __launch_bounds__(TX *TY, MINB) k_substep_lag64(
    const __grid_constant__ CUtensorMap tmap, double *__restrict__ out, double *__restrict__ w,
    const Layout Ls, const Layout Lw, const CoefT c, const RKStage st, const int zc,
    const int tiles_x, int *__restrict__ dev_error, const int skip_plane_arg)
{
    using RG = Ring64<NF, TX, TY, NS>;
    using tiled::mbar_wait;
    constexpr int BX = RG::BX, FSTRIDE = RG::FSTRIDE, SLOT_ELEMS = RG::SLOT_ELEMS;
    constexpr int W = 7;  // windows: planes (outputs) s-3 .. s+3 around step s
    static_assert(NS >= 5, "the centre plane, the three above it and one in flight");
    extern __shared__ __align__(128) unsigned char smem[];
    const double *sm = reinterpret_cast<const double *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF);
    tiled2::init_barriers(bars, NS);
    // warp 0 allocates the CTA's TMEM columns; every thread reads the address
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + RG::TM_OFF);
    if (threadIdx.x < 32)
        tc::tmem_alloc(tslot, kTmCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    const uint32_t trow = tmem + ((uint32_t)(threadIdx.x & ~31) << 16);

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nout = min(zc, Ls.nz - z0);
    const int nplanes = nout + 2 * R;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = (x < Ls.nx) && (y < Ls.ny);
    const int toff = (ty + GY) * BX + (tx + GX);
    const bool first = st.first != 0, last = st.last != 0;
    const double alpha = st.alpha, beta = st.beta, dt = st.dt;
    const int skip_plane = blockIdx.x == 0 && blockIdx.y == 0 ? skip_plane_arg : -1;

    int issued = 0;
    auto issue = [&](int j) {
        if (j == skip_plane)  // fault injection for the bounded-wait test
            return;
        const int z = zplane(Ls, z0 - R + j) + Ls.gz;  // TMA z coordinate
        const int slot = j % NS;
        tiled::mbar_expect_tx(&bars[slot], RG::SLOT_BYTES);
        tiled::tma_load_4d(smem + slot * RG::SLOT_PITCH, &tmap, &bars[slot], x0, y0, z, 0);
    };
    auto issue_upto = [&](int jend) {
        jend = min(jend, nplanes);
#pragma unroll 1
        for (int j = issued; j < jend; ++j)
            issue(j);
        issued = max(issued, jend);
    };
    int waited = 0;
    bool timeout = false;
    auto wait = [&](int j) {
        if (!mbar_wait(&bars[j % NS], (j / NS) & 1))
            timeout = true;
        waited = j + 1;
    };
    if (threadIdx.x == 0) {
        tiled::fence_proxy_async();
        issue_upto(NS);
    }

    // colv[f][k]: field f on the thread's z-column at local plane s - 3 + k;
    // acx/acy/acz[m]: the z-paired Eq. 8 terms of output plane s - 6 + m for
    // the x (D_xz u_z), y (D_yz u_z) and z (D_xz u_x + D_yz u_y) components
    double colv[NF][W];
    double acx[W], acy[W], acz[W];
#pragma unroll
    for (int m = 0; m < W; ++m)
        acx[m] = acy[m] = acz[m] = 0.0;

    // add the differences d[k-1] of one plane (accumulator index MC) with
    // weights MX(pair, k): plus to the outputs below it, minus to those above
    auto spread = [&](double *ac, const double *d, int pair, auto mcc) {
        constexpr int MC = decltype(mcc)::value;
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const double mk = c.MX(pair, k);
            if (MC - k >= 0)
                ac[MC - k] = fma(mk, d[k - 1], ac[MC - k]);
            if (MC + k < W)
                ac[MC + k] = fma(-mk, d[k - 1], ac[MC + k]);
        }
    };
    // a plane that is not a centre (the halo planes of the chunk): its
    // x and y differences of u_x, u_y, u_z alone
    auto arms = [&](int base, auto mcc) {
        auto at = [&](int f, int dy, int dx) -> double {
            return sm[base + f * FSTRIDE + dy * BX + dx];
        };
        double d[3];
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            d[k - 1] = at(1, 0, k) - at(1, 0, -k);
        spread(acz, d, 1, mcc);
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            d[k - 1] = at(2, k, 0) - at(2, -k, 0);
        spread(acz, d, 2, mcc);
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            d[k - 1] = at(3, 0, k) - at(3, 0, -k);
        spread(acx, d, 1, mcc);
#pragma unroll
        for (int k = 1; k <= 3; ++k)
            d[k - 1] = at(3, k, 0) - at(3, -k, 0);
        spread(acy, d, 2, mcc);
    };

    // prologue: local planes 0..5 into the column window (the ring holds NS
    // at a time: planes 0..2 first, then their slots go to planes NS..); the
    // three halo planes below the chunk give their differences
#pragma unroll
    for (int j = 0; j < R; ++j) {
        wait(j);
        const int base = (j % NS) * SLOT_ELEMS + toff;
#pragma unroll
        for (int f = 0; f < NF; ++f)
            colv[f][j] = sm[base + f * FSTRIDE];
        if (j == 0)
            arms(base, std::integral_constant<int, 0>{});
        else if (j == 1)
            arms(base, std::integral_constant<int, 1>{});
        else
            arms(base, std::integral_constant<int, 2>{});
    }
    if (__syncthreads_or(timeout)) {
        timeout = true;
    } else {
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            issue_upto(R + NS);
        }
#pragma unroll
        for (int j = R; j < 2 * R; ++j) {
            wait(j);
            const int base = (j % NS) * SLOT_ELEMS + toff;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                colv[f][j] = sm[base + f * FSTRIDE];
        }
    }

    // global offsets of the point in the next output plane to finish, and of
    // its periodic ghost copies
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
    const bool need_w = !first;

    // centre work on the plane in the slot at cb (output plane s - 3): the
    // right-hand side without the z-paired Eq. 8 terms into prn, the plane's
    // x/y differences of u_x, u_y, u_z into the accumulators (index 3)
    auto centre = [&](const int cb, double *prn) {
        using MC3 = std::integral_constant<int, 3>;
        auto ld = [&](int f, int dy, int dx) -> double {
            return sm[cb + f * FSTRIDE + dy * BX + dx];
        };
        double g[3], d2[3], hx[3], hy[3];
        // Eqs. 6-7 along x, y, z for field f; hx, hy keep the differences
        auto axial = [&](int f, bool second) {
            const double cc = colv[f][3];
            double ax, ay, az, bx, by, bz;
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                const double xp = ld(f, 0, k), xm = ld(f, 0, -k);
                const double yp = ld(f, k, 0), ym = ld(f, -k, 0);
                const double zp = colv[f][3 + k], zm = colv[f][3 - k];
                hx[k - 1] = xp - xm;
                hy[k - 1] = yp - ym;
                const double dz = zp - zm;
                if (k == 1) {
                    ax = c.D1(0, 1) * hx[0];
                    ay = c.D1(1, 1) * hy[0];
                    az = c.D1(2, 1) * dz;
                } else {
                    ax = fma(c.D1(0, k), hx[k - 1], ax);
                    ay = fma(c.D1(1, k), hy[k - 1], ay);
                    az = fma(c.D1(2, k), dz, az);
                }
                if (second) {
                    if (k == 1) {
                        bx = c.D2c(0) * cc;
                        by = c.D2c(1) * cc;
                        bz = c.D2c(2) * cc;
                    }
                    bx = fma(c.D2(0, k), xp + xm, bx);
                    by = fma(c.D2(1, k), yp + ym, by);
                    bz = fma(c.D2(2, k), zp + zm, bz);
                }
            }
            g[0] = ax;
            g[1] = ay;
            g[2] = az;
            if (second) {
                d2[0] = bx;
                d2[1] = by;
                d2[2] = bz;
            }
        };
        // Eq. 8 in the (x, y) plane
        auto mix_xy = [&](int f) -> double {
            double a;
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                const double d = (ld(f, k, k) - ld(f, k, -k)) - (ld(f, -k, k) - ld(f, -k, -k));
                a = k == 1 ? c.MX(0, 1) * d : fma(c.MX(0, k), d, a);
            }
            return a;
        };
        const double NU = c.nu, NU3 = c.nu3;
        const double uc[3] = {colv[1][3], colv[2][3], colv[3][3]};
        double acc[4], gl[3];
        double dv = 0.0;
        axial(0, false);
        gl[0] = g[0];
        gl[1] = g[1];
        gl[2] = g[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            axial(1 + i, true);
            // this plane's differences: D_xz u_x and D_yz u_y -> z component,
            // D_xz u_z -> x, D_yz u_z -> y
            if (i == 0) {
                spread(acz, hx, 1, MC3{});
            } else if (i == 1) {
                spread(acz, hy, 2, MC3{});
            } else {
                spread(acx, hx, 1, MC3{});
                spread(acy, hy, 2, MC3{});
            }
            double adv = uc[0] * g[0];
            adv = fma(uc[1], g[1], adv);
            adv = fma(uc[2], g[2], adv);
            const double lap = d2[0] + d2[1] + d2[2];
            double sg = g[0] * gl[0];
            sg = fma(g[1], gl[1], sg);
            sg = fma(g[2], gl[2], sg);
            double ai = NU * (lap + sg);
            if (i > 0)
                ai += acc[1 + i];
            ai -= adv;
            ai = fma(NU3, d2[i], ai);
            acc[1 + i] = ai;
            // the d_a u_i d_i lnrho half of 2 S.grad lnrho, for every component a
            const double nugl = NU * gl[i];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a > i && i == 0)
                    acc[1 + a] = g[a] * nugl;  // first contribution
                else
                    acc[1 + a] = fma(g[a], nugl, acc[1 + a]);
            }
            dv += g[i];
            if (i == 0)
                acc[2] = fma(NU3, mix_xy(1), acc[2]);  // D_xy u_x -> y
            else if (i == 1)
                acc[1] = fma(NU3, mix_xy(2), acc[1]);  // D_xy u_y -> x
        }
        if constexpr (NF == 5) {
            axial(4, false);
            double t = uc[0] * g[0];
            t = fma(uc[1], g[1], t);
            t = fma(uc[2], g[2], t);
            prn[4] = -t;
        }
        double ug = uc[0] * gl[0];
        ug = fma(uc[1], gl[1], ug);
        ug = fma(uc[2], gl[2], ug);
        prn[0] = -(ug + dv);
        const double t = -c.nu23 * dv;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            prn[1 + a] = fma(t, gl[a], fma(-c.cs2, gl[a], acc[1 + a]));
    };

    // u-tilde of the next output plane to finish (before the work that hides
    // the loads)
    auto load_w = [&](double *wv) {
        if (need_w && valid) {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                wv[f] = w[f * Lw.fpitch + go_w];
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                wv[f] = 0.0;
        }
    };
    // output plane o (accumulator and window index I): add the z-paired
    // terms, apply Eq. 10, store the state (and ghost copies) and u-tilde
    auto finish = [&](const int o, auto ic, const double *wv) {
        constexpr int I = decltype(ic)::value;
        double r[NF];
        tm_get<NF>(trow + (uint32_t)((o & 3) * kTmSlotCols), r);
        r[1] = fma(c.nu3, acx[I], r[1]);
        r[2] = fma(c.nu3, acy[I], r[2]);
        r[3] = fma(c.nu3, acz[I], r[3]);
        if (valid) {
            if constexpr (FORCE) {
                // f_i = amp_i cos(k.x + phi) (Sect. 6, Eqs. 20-21)
                const double fc = forcing_cos<double>(st.fo, x, y, z0 + o);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    r[1 + a] = fma(st.fo.amp[a], fc, r[1 + a]);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const double wn = first ? dt * r[f] : fma(alpha, wv[f], dt * r[f]);
                const double ov = fma(beta, wn, colv[f][I]);
                if (!last)
                    w[f * Lw.fpitch + go_w] = wn;
                double *op = out + f * Ls.fpitch + go_s;
                *op = ov;
                if (gdx)
                    op[gdx] = ov;
                if (gdy) {
                    op[gdy] = ov;
                    if (gdx)
                        op[gdy + gdx] = ov;
                }
            }
        }
        go_s += Ls.plane;
        go_w += Lw.plane;
    };
    // all threads are done with the steps before s: the slots of planes
    // below s are free; true (for every thread) when some wait gave up
    auto top = [&](const int s) -> bool {
        if (__syncthreads_or(timeout))
            return true;
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            issue_upto(s + NS);
        }
        return false;
    };

    int s = R;
    bool stop = timeout;
    if (!stop) {
#pragma unroll 1
        for (; s < nout + R; ++s) {
            if (top(s)) {
                stop = true;
                break;
            }
            double wv[NF];
            const bool fin = s >= 2 * R;
            if (fin)
                load_w(wv);
            // the column value of plane s + 3
            wait(s + R);
            const int nb = ((s + R) % NS) * SLOT_ELEMS + toff;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                colv[f][6] = sm[nb + f * FSTRIDE];
            double prn[NF];
            centre((s % NS) * SLOT_ELEMS + toff, prn);
            tm_put<NF>(trow + (uint32_t)(((s - R) & 3) * kTmSlotCols), prn);
            if (fin)
                finish(s - 2 * R, std::integral_constant<int, 0>{}, wv);
            // slide the windows by one plane
#pragma unroll
            for (int f = 0; f < NF; ++f) {
#pragma unroll
                for (int k = 0; k + 1 < W; ++k)
                    colv[f][k] = colv[f][k + 1];
            }
#pragma unroll
            for (int m = 0; m < W; ++m) {
                acx[m] = m + 1 < W ? acx[m + 1] : 0.0;
                acy[m] = m + 1 < W ? acy[m + 1] : 0.0;
                acz[m] = m + 1 < W ? acz[m + 1] : 0.0;
            }
        }
    }
    if (!stop && top(s))
        stop = true;
    if (!stop) {
        // the three halo planes above the chunk (local s .. s + 2, waited for
        // as column values already): their differences finish the last outputs
        auto tail = [&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const int j = s + E;
            arms((j % NS) * SLOT_ELEMS + toff, std::integral_constant<int, E + 3>{});
            if (j >= 2 * R) {
                double wv[NF];
                load_w(wv);
                finish(j - 2 * R, ec, wv);
            }
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
                (void)mbar_wait(&bars[j % NS], (j / NS) & 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32)
        tc::tmem_dealloc(tmem, kTmCols);
}

}  // namespace tiled6

// Launch of the FP64 lagged-output kernel (55-point form).
template <int TX, int TY, int NS, int MINB>
cudaError_t launch_lag64_cfg(const StateBufs &b, const Coef<double> &c, const RKStage &st, int nf,
                             int zc, int cfg_key, int *dev_error, TmapCache *cache,
                             cudaStream_t stream, int *launches)
{
    CUtensorMap *map = nullptr;
    if (!get_state_tmap(cache, b.in, b.Ls, nf, TX, TY, cfg_key, &map))
        return cudaErrorInvalidValue;
    const int tiles_x = (b.Ls.nx + TX - 1) / TX;
    const int tiles_y = (b.Ls.ny + TY - 1) / TY;
    const dim3 grid(tiles_x * tiles_y, (b.Ls.nz + zc - 1) / zc);
    const dim3 block(TX * TY);
    double *out = (double *)b.out;
    double *w = (double *)b.w;
    const int skip_plane = st.fault_skip_plane;
    cudaError_t e;
    const bool iso = coef_is_cubic(c);
    const CubicCoef<double> cc = cubic_of(c);
#define GBFD_LAUNCH_L64_F(NFV, FRC, CT, CV)                                                       \
    do {                                                                                          \
        auto kern = tiled6::k_substep_lag64<NFV, TX, TY, NS, MINB, FRC, CT>;                      \
        constexpr int sm = tiled6::Ring64<NFV, TX, TY, NS>::BYTES;                                \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e == cudaSuccess)                                                                     \
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,        \
                                     (int)cudaSharedmemCarveoutMaxShared);                        \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, out, w, b.Ls, b.Lw, CV, st, zc, tiles_x,          \
                                          dev_error, skip_plane);                                 \
    } while (0)
#define GBFD_LAUNCH_L64(NFV, CT, CV)                                                              \
    do {                                                                                          \
        if (st.fo.on)                                                                             \
            GBFD_LAUNCH_L64_F(NFV, true, CT, CV);                                                 \
        else                                                                                      \
            GBFD_LAUNCH_L64_F(NFV, false, CT, CV);                                                \
    } while (0)
    if (nf == 5) {
        if (iso)
            GBFD_LAUNCH_L64(5, CubicCoef<double>, cc);
        else
            GBFD_LAUNCH_L64(5, Coef<double>, c);
    } else {
        if (iso)
            GBFD_LAUNCH_L64(4, CubicCoef<double>, cc);
        else
            GBFD_LAUNCH_L64(4, Coef<double>, c);
    }
#undef GBFD_LAUNCH_L64
#undef GBFD_LAUNCH_L64_F
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
